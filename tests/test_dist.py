"""Replica coordination over world_size 2 with the gloo backend on CPU: the host logic that
bench.py runs under torchrun (barrier, slowest-rank time, whole-job rate, disjoint seeds)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2212_14191_gb300 import replicas as R


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port),
                       "WORLD_SIZE": str(ws), "RANK": str(rank), "LOCAL_RANK": str(rank)})
    got_ws, got_rank, _ = R.dist_env()
    R.init(got_ws, "gloo")
    R.barrier(got_ws, cuda=False)
    elapsed = 1.0 + rank          # rank 1 is the slower one
    slowest = R.max_over_ranks(elapsed, got_ws, device="cpu")
    rate = R.whole_job_rate(100, got_ws, slowest)
    R.barrier(got_ws, cuda=False)
    R.finish(got_ws)
    q.put((got_rank, got_ws, slowest, rate, R.rank_seed(1234, got_rank)))


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1]
    assert all(r[1] == 2 for r in res)
    assert all(r[2] == 2.0 for r in res)          # both see the slowest rank's time
    assert all(r[3] == 100.0 for r in res)        # 2 ranks x 100 units / 2 s
    assert res[0][4] != res[1][4]                 # disjoint input seeds


def test_single_process_defaults(monkeypatch):
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert R.dist_env() == (1, 0, 0)
    assert R.max_over_ranks(3.5, 1) == 3.5
    assert R.whole_job_rate(10, 1, 2.0) == 5.0
    with pytest.raises(ValueError):
        R.whole_job_rate(10, 1, 0.0)

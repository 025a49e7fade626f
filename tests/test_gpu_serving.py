"""Serving loop: every request's result is identical whether it is served alone (a
single-request library call) or batched with others in the continuous-batching loop, and the
loop respects its HBM budget."""
import numpy as np
import pytest

from oracle import params as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fhe():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_14191_gb300 import fhe as f
    return f


def test_results_identical_alone_and_in_mix(fhe):
    import torch
    from paper_2212_14191_gb300 import serving as S
    qs, ps = P.default_moduli(10, 4)
    logns = (12, 13)
    ctxs = {lg: fhe.Context(lg, qs, ps, alpha=4) for lg in logns}
    dnum = -(-len(qs) // 4)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(3)
    evks = {lg: torch.randint(0, 1 << 29, (dnum, 2, len(qs) + len(ps), 1 << lg), dtype=torch.int32,
                              device="cuda", generator=gen) for lg in logns}

    def make_inputs(kind, logN, nl, rid):
        n = 1 << logN
        if kind == S.KEYSWITCH:
            return (torch.randint(0, 1 << 29, (nl, 1, n), dtype=torch.int32, device="cuda", generator=gen),)
        k = 2 if kind == S.HMULT else 1
        return tuple(torch.randint(0, 1 << 29, (2, nl, 1, n), dtype=torch.int32, device="cuda", generator=gen)
                     for _ in range(k))

    reqs = S.poisson_requests(9, 80, 20000.0, [S.HMULT, S.RESCALE, S.KEYSWITCH], logns, (2, 10), make_inputs)
    budget = 256 << 20
    server = S.Server(ctxs, evks, budget_bytes=budget, n_streams=3, max_batch=8)
    stats = server.run(reqs)
    torch.cuda.synchronize()
    assert stats["requests"] == 80 and stats["peak_footprint_bytes"] <= budget
    assert stats["mean_batch"] > 1.0          # requests were actually batched together
    for r in reqs:
        alone = server._launch([r.__class__(r.rid, r.kind, r.logN, r.nl, 0.0, r.inputs)],
                               torch.cuda.current_stream())
        torch.cuda.synchronize()
        assert torch.equal(alone["reqs"][0].out, r.out), (r.rid, r.kind)
    for c in ctxs.values():
        fhe.fhe_device_status(c.handle, 1)
        c.close()

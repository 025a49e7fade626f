"""Host logic of the serving loop on the CPU, with the GPU calls replaced by fakes: admission
by footprint under the budget, continuous batching to completion, rejection under overload
once a request's admission deadline passes, the stall watchdog (a batch that never completes
stops the run with an error instead of hanging it) and the device-status check after the run.
No kernel runs and no GPU is touched."""
import pytest

from paper_2212_14191_gb300 import serving as S


class FakeClock:
    """Deterministic seconds: every reading advances by `step`."""

    def __init__(self, step=0.001):
        self.t, self.step = 0.0, step

    def __call__(self):
        self.t += self.step
        return self.t


class FakeEvent:
    def __init__(self, clock, done_at):
        self.clock, self.done_at = clock, done_at

    def query(self):
        return self.clock.t >= self.done_at


class FakeServer(S.Server):
    """The loop of S.Server with launches that complete `latency` seconds later (never, for
    latency None) and a device check that only records that it ran."""

    def __init__(self, clock, latency, budget, stall_s=0.5, footprint=10, n_streams=2, max_batch=3,
                 admit_timeout_s=None):
        self.ctx, self.evk = {}, {}
        self.budget, self.streams, self.max_batch, self.stall_s = budget, list(range(n_streams)), max_batch, stall_s
        self.admit_timeout_s = admit_timeout_s
        self.clock, self.latency, self.fp = clock, latency, footprint
        self.checked, self.launched, self.max_used = False, [], 0

    def footprint(self, r):
        return self.fp

    def _launch(self, reqs, stream):
        self.launched.append(len(reqs))
        done_at = float("inf") if self.latency is None else self.clock.t + self.latency
        return {"reqs": reqs, "event": FakeEvent(self.clock, done_at), "keep": None, "stream": stream}

    def check_device(self):
        self.checked = True

    def _producer_event(self):
        return None


def requests(n, gap=0.0005, kinds=(S.HMULT, S.RESCALE)):
    return [S.Request(i, kinds[i % len(kinds)], 15, 4, i * gap, ()) for i in range(n)]


def test_all_requests_complete_within_the_budget():
    clock = FakeClock()
    srv = FakeServer(clock, latency=0.01, budget=45)
    reqs = requests(40)
    res = srv.run(reqs, clock=clock)
    assert res["requests"] == 40 and res["completed"] == 40 and res["rejected"] == 0 and srv.checked
    assert all(r.t_done is not None and r.t_done >= r.t_launch >= r.t_admit >= r.arrival for r in reqs)
    assert res["peak_footprint_bytes"] <= 45                    # at most 4 of 10 bytes admitted at once
    assert max(srv.launched) <= 3 and sum(srv.launched) == 40
    assert res["p50_ms"] <= res["p99_ms"] <= res["max_ms"]


def test_a_request_larger_than_the_budget_still_runs_alone():
    clock = FakeClock()
    srv = FakeServer(clock, latency=0.01, budget=5, footprint=10)
    res = srv.run(requests(3), clock=clock)
    assert res["requests"] == 3 and res["peak_footprint_bytes"] == 10


def test_a_batch_that_never_completes_stops_the_run():
    clock = FakeClock()
    srv = FakeServer(clock, latency=None, budget=1000, stall_s=0.2)
    with pytest.raises(RuntimeError, match="no batch completed"):
        srv.run(requests(5), clock=clock)
    assert not srv.checked


def test_overload_rejects_after_the_admission_deadline():
    """One request fits the budget at a time and each batch takes 50 ms while requests arrive
    every 0.5 ms: those that wait more than 10 ms for memory are rejected, never launched, and
    the rest complete; the counts add up and the latency statistics cover completed ones."""
    clock = FakeClock()
    srv = FakeServer(clock, latency=0.05, budget=10, n_streams=1, max_batch=1, admit_timeout_s=0.01)
    reqs = requests(30)
    res = srv.run(reqs, clock=clock)
    assert 0 < res["rejected"] < 30 and res["completed"] + res["rejected"] == 30
    assert sum(srv.launched) == res["completed"] and srv.checked
    for r in reqs:
        if r.rejected:
            assert r.t_admit is None and r.t_launch is None and r.t_done is None
        else:
            assert r.t_done >= r.t_launch >= r.t_admit >= r.arrival
    assert res["peak_footprint_bytes"] <= 10

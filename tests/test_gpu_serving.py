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


def _serve_and_compare(fhe, logns, n_q, n_p, alpha, nl_range, n_req, rate, budget, n_streams, max_batch, seed):
    """Serve a seeded Poisson stream of HMULT / RESCALE / KEYSWITCH requests whose operands are
    written by torch on the current stream right before the run, with no synchronisation in
    between (the server orders its streams after that one), then compare every result with
    the same request launched alone."""
    import torch
    from paper_2212_14191_gb300 import serving as S
    qs, ps = P.default_moduli(n_q, n_p)
    ctxs = {lg: fhe.Context(lg, qs, ps, alpha=alpha) for lg in logns}
    dnum = -(-len(qs) // alpha)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    evks = {lg: torch.randint(0, 1 << 29, (dnum, 2, len(qs) + len(ps), 1 << lg), dtype=torch.int32,
                              device="cuda", generator=gen) for lg in logns}

    def make_inputs(kind, logN, nl, rid):
        n = 1 << logN
        if kind == S.KEYSWITCH:
            return (torch.randint(0, 1 << 29, (nl, 1, n), dtype=torch.int32, device="cuda", generator=gen),)
        k = 2 if kind == S.HMULT else 1
        return tuple(torch.randint(0, 1 << 29, (2, nl, 1, n), dtype=torch.int32, device="cuda", generator=gen)
                     for _ in range(k))

    reqs = S.poisson_requests(seed + 6, n_req, rate, [S.HMULT, S.RESCALE, S.KEYSWITCH], logns, nl_range, make_inputs)
    server = S.Server(ctxs, evks, budget_bytes=budget, n_streams=n_streams, max_batch=max_batch)
    stats = server.run(reqs)
    torch.cuda.synchronize()
    assert stats["requests"] == n_req and stats["completed"] == n_req and stats["peak_footprint_bytes"] <= budget
    assert stats["mean_batch"] > 1.0          # requests were actually batched together
    for r in reqs:
        alone = server._launch([r.__class__(r.rid, r.kind, r.logN, r.nl, 0.0, r.inputs)],
                               torch.cuda.current_stream())
        torch.cuda.synchronize()
        assert torch.equal(alone["reqs"][0].out, r.out), (r.rid, r.kind)
    for c in ctxs.values():
        fhe.fhe_device_status(c.handle, 1)
        c.close()


def test_results_identical_alone_and_in_mix(fhe):
    """N = 2^12 and 2^13, 2..10 limbs: many small requests per batch."""
    _serve_and_compare(fhe, (12, 13), 10, 4, 4, (2, 10), 80, 20000.0, 256 << 20, 3, 8, 3)


def test_results_identical_alone_and_in_mix_n32768(fhe):
    """The serving workload's ring degree N = 2^15 with 3..24 limbs (24 ciphertext primes, 8
    special primes, alpha = 8): the two-pass NTT kernels and up to three key-switching slices
    inside the batched calls."""
    _serve_and_compare(fhe, (15,), 24, 8, 8, (3, 24), 160, 20000.0, 2 << 30, 4, 8, 11)

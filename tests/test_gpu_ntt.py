"""GPU parity of the batched negacyclic NTT/INTT against the CPU oracle (bit-exact)."""
import numpy as np
import pytest

from oracle import ntt as ON
from oracle import params as P
from paper_2212_14191_gb300 import inputs as I

pytestmark = pytest.mark.gpu

QS, PS = P.default_moduli(44, 8)
MODS = QS + PS
PATHS = ["u32", "tc"]


@pytest.fixture(scope="module")
def fhe():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_14191_gb300 import fhe as f
    return f


@pytest.fixture(scope="module")
def ctx(fhe):
    c = fhe.Context(16, QS, PS, alpha=8)
    yield c
    c.close()


def _path(fhe, name):
    return {"u32": fhe.FHE_NTT_U32, "tc": fhe.FHE_NTT_TC}[name]


def psis(mods, n):
    return [P.psi(m, n) for m in mods]


@pytest.mark.parametrize("variant", list(range(32)))
@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("logn", [10, 11, 12, 13, 14, 15, 16])
def test_fwd_inv_match_oracle(fhe, ctx, logn, path, variant):
    import torch
    if path == "tc" and variant > 0:
        pytest.skip("kernel shapes apply to the 32-bit path")
    try:
        fhe.fhe_ntt_set_variant(ctx.handle, logn, variant)
    except fhe.FheError:
        pytest.skip("no such shape at this N")
    n = 1 << logn
    first, nl, batch = 42, 4, 3          # limbs q_42, q_43, p_0, p_1: crosses the q/p boundary
    mods = MODS[first:first + nl]
    x = I.uniform_residues(logn, mods, batch, n)
    d = fhe.to_device(x)
    ctx.ntt_fwd(d, logn, first_limb=first, path=_path(fhe, path))
    torch.cuda.synchronize()
    want, _ = ON.ntt_batch(x, mods, psis(mods, n))
    assert (fhe.to_host(d) == want).all()
    ctx.ntt_inv(d, logn, first_limb=first, path=_path(fhe, path))
    assert (fhe.to_host(d) == x).all()
    # inverse on fresh random input against the oracle's inverse
    y = I.uniform_residues(100 + logn, mods, batch, n)
    e = fhe.to_device(y)
    ctx.ntt_inv(e, logn, first_limb=first, path=_path(fhe, path))
    want, _ = ON.ntt_batch(y, mods, psis(mods, n), inverse=True)
    assert (fhe.to_host(e) == want).all()
    fhe.fhe_ntt_set_variant(ctx.handle, logn, 0)


@pytest.mark.parametrize("choice", [32, 33])
@pytest.mark.parametrize("logn", [10, 11, 12, 13, 14, 15, 16])
def test_tensor_core_choices(fhe, ctx, logn, choice):
    """The tensor-core path as the choice of FHE_NTT_DEFAULT (variant ids FHE_NTT_VARIANT_TC64 /
    TC32: output tiles of 64 or 32 columns, the latter with its own 32-row constant-matrix tensor
    maps where the matrices are 64 or more columns wide): bit-exact forward and inverse, the
    explicit FHE_NTT_TC path taking the same tile width, and FHE_NTT_U32 keeping its plain
    variant."""
    import torch
    keep = (fhe.fhe_ntt_get_variant(ctx.handle, logn, 0), fhe.fhe_ntt_get_variant(ctx.handle, logn, 1))
    fhe.fhe_ntt_set_variant(ctx.handle, logn, choice, choice)
    assert fhe.fhe_ntt_get_variant(ctx.handle, logn, 0) == choice
    n = 1 << logn
    first, nl, batch = 40, 6, 5
    mods = MODS[first:first + nl]
    x = I.uniform_residues(900 + logn + choice, mods, batch, n)
    want, _ = ON.ntt_batch(x, mods, psis(mods, n))
    for path in (fhe.FHE_NTT_DEFAULT, fhe.FHE_NTT_TC, fhe.FHE_NTT_U32):
        d = fhe.to_device(x)
        ctx.ntt_fwd(d, logn, first_limb=first, path=path)
        torch.cuda.synchronize()
        assert (fhe.to_host(d) == want).all(), path
        ctx.ntt_inv(d, logn, first_limb=first, path=path)
        torch.cuda.synchronize()
        assert (fhe.to_host(d) == x).all(), path
    fhe.fhe_device_status(ctx.handle, 1)
    fhe.fhe_ntt_set_variant(ctx.handle, logn, keep[0], keep[1])


@pytest.mark.parametrize("path", PATHS)
def test_plain_ntt_config_n4096(fhe, path):
    """N = 2^12, one prime q_0, 16 polynomials uniform in [0, q), seed 0."""
    import torch
    logn, n = 12, 1 << 12
    q = QS[0]
    c = fhe.Context(12, [q])
    x = I.uniform_residues(0, [q], 16, n)
    d = fhe.to_device(x)
    c.ntt_fwd(d, logn, path=_path(fhe, path))
    torch.cuda.synchronize()
    A = fhe.to_host(d)
    psi = P.psi(q, n)
    want, _ = ON.ntt_batch(x, [q], [psi])
    assert (A == want).all()
    assert (A[0, 0] == ON.ntt_brute(x[0, 0], q, psi)).all()
    # convolution theorem: INTT(NTT(a) . NTT(b)) equals the schoolbook product mod X^N + 1
    prod = (A[0, 0::2].astype(np.uint64) * A[0, 1::2].astype(np.uint64)) % q
    p = fhe.to_device(prod.astype(np.uint32)[None])
    c.ntt_inv(p, logn, path=_path(fhe, path))
    got = fhe.to_host(p)[0]
    for i in range(8):
        assert (got[i] == ON.negacyclic_mul(x[0, 2 * i], x[0, 2 * i + 1], q)).all()
    c.close()


@pytest.mark.parametrize("path", PATHS)
def test_full_size_ckks_batch(fhe, ctx, path):
    """N = 2^16, 44 limbs q_0..q_43, 64 polynomials (704 MiB), one call per direction.

    Sampled rows are checked against the oracle; the round trip is checked in full.
    """
    import torch
    logn, n, nl, batch = 16, 1 << 16, 44, 64
    x = I.uniform_residues(7, QS, batch, n)
    d = fhe.to_device(x)
    ctx.ntt_fwd(d, logn, path=_path(fhe, path))
    torch.cuda.synchronize()
    rng = np.random.default_rng(1)
    rows = [(l, b) for l in range(nl) for b in (0, batch - 1)] + \
           [(int(l), int(b)) for l, b in zip(rng.integers(0, nl, 8), rng.integers(0, batch, 8))]
    got = fhe.to_host(d)
    for l, b in rows:
        assert (got[l, b] == ON.ntt(x[l, b], QS[l], P.psi(QS[l], n))).all(), (l, b)
    ctx.ntt_inv(d, logn, path=_path(fhe, path))
    xd = fhe.to_device(x)
    assert torch.equal(d, xd)


@pytest.mark.parametrize("variant", list(range(32)))
@pytest.mark.parametrize("logn", [14, 15, 16])
def test_many_rows_cross_limbs(fhe, ctx, logn, variant):
    """More rows than resident clusters, a ragged batch, and limb boundaries inside every
    persistent CTA's row range: the per-modulus twiddle refresh and the row iteration."""
    import torch
    keep = fhe.fhe_ntt_get_variant(ctx.handle, logn)
    try:
        fhe.fhe_ntt_set_variant(ctx.handle, logn, variant)
    except fhe.FheError:
        pytest.skip("no such shape at this N")
    n = 1 << logn
    first, nl = 3, 5
    batch = {14: 61, 15: 29, 16: 23}[logn]
    mods = MODS[first:first + nl]
    x = I.uniform_residues(900 + logn, mods, batch, n)
    d = fhe.to_device(x)
    ctx.ntt_fwd(d, logn, first_limb=first)
    torch.cuda.synchronize()
    got = fhe.to_host(d)
    ps = psis(mods, n)
    for l in range(nl):
        for b in sorted({0, 1, batch // 2, batch - 2, batch - 1}):
            assert (got[l, b] == ON.ntt(x[l, b], mods[l], ps[l])).all(), (l, b)
    ctx.ntt_inv(d, logn, first_limb=first)
    assert torch.equal(d, fhe.to_device(x))
    fhe.fhe_ntt_set_variant(ctx.handle, logn, keep)


@pytest.mark.parametrize("path", PATHS)
def test_edge_values(fhe, ctx, path):
    import torch
    for logn in (10, 16):
        n = 1 << logn
        mods = QS[:2]
        for fill in ("zero", "max"):
            x = np.zeros((2, 2, n), dtype=np.uint32)
            if fill == "max":
                for l, m in enumerate(mods):
                    x[l] = m - 1
            d = fhe.to_device(x)
            ctx.ntt_fwd(d, logn, path=_path(fhe, path))
            torch.cuda.synchronize()
            want, _ = ON.ntt_batch(x, mods, psis(mods, n))
            assert (fhe.to_host(d) == want).all()
            ctx.ntt_inv(d, logn, path=_path(fhe, path))
            assert (fhe.to_host(d) == x).all()


@pytest.mark.parametrize("logn", [12, 16])
def test_autotune_keeps_results(fhe, ctx, logn):
    import torch
    n = 1 << logn
    x = I.uniform_residues(55, QS[:4], 8, n)
    d = fhe.to_device(x)
    fwd, inv = fhe.fhe_autotune_ntt(ctx.handle, logn, d.data_ptr(), 4, 8, reps=2,
                                    stream=torch.cuda.current_stream().cuda_stream)
    count = fhe.fhe_ntt_variant_count(ctx.handle, logn)
    assert len(fwd) == len(inv) == count
    valid = [i for i in range(count) if fwd[i] > 0]
    assert valid and valid == [i for i in range(count) if inv[i] > 0]
    assert all(fwd[i] == -1 and inv[i] == -1 for i in range(count) if i not in valid)
    for i in valid:                                     # exactly the variants the library accepts
        fhe.fhe_ntt_set_variant(ctx.handle, logn, i)
    for i in set(range(count)) - set(valid):
        with pytest.raises(fhe.FheError):
            fhe.fhe_ntt_set_variant(ctx.handle, logn, i)
    fwd, inv = fhe.fhe_autotune_ntt(ctx.handle, logn, d.data_ptr(), 4, 8, reps=2,
                                    stream=torch.cuda.current_stream().cuda_stream)
    assert fhe.fhe_ntt_get_variant(ctx.handle, logn, 0) == min(valid, key=lambda i: fwd[i])
    assert fhe.fhe_ntt_get_variant(ctx.handle, logn, 1) == min(valid, key=lambda i: inv[i])
    assert (fhe.to_host(d) == x).all()          # the round trips restore the input
    ctx.ntt_fwd(d, logn)
    want, _ = ON.ntt_batch(x, QS[:4], psis(QS[:4], n))
    assert (fhe.to_host(d) == want).all()
    fhe.fhe_ntt_set_variant(ctx.handle, logn, 0)


def test_device_status_clean(fhe, ctx):
    fhe.fhe_device_status(ctx.handle, 1)


def test_batch_zero_and_bad_args(fhe, ctx):
    import torch
    d = torch.zeros((1, 1, 1024), dtype=torch.int32, device="cuda")
    fhe.fhe_ntt_fwd(ctx.handle, 0, 10, d.data_ptr(), 0, 1, 0, 0)      # batch 0: no-op
    assert int(d.abs().sum()) == 0
    for args in ((0, 9, d.data_ptr(), 0, 1, 1), (0, 17, d.data_ptr(), 0, 1, 1),
                 (0, 10, d.data_ptr() + 4, 0, 1, 1), (0, 10, d.data_ptr(), 50, 3, 1),
                 (7, 10, d.data_ptr(), 0, 1, 1), (0, 10, 0, 0, 1, 1)):
        with pytest.raises(fhe.FheError) as e:
            fhe.fhe_ntt_fwd(ctx.handle, *args, 0)
        assert e.value.code == fhe.FHE_EINVAL
    small = fhe.Context(12, QS[:1])
    with pytest.raises(fhe.FheError):
        small.ntt_fwd(torch.zeros((1, 1, 1 << 13), dtype=torch.int32, device="cuda"), 13)
    small.close()


@pytest.mark.parametrize("variant", [6, 7])
@pytest.mark.parametrize("logn", [15, 16])
def test_two_pass_fused_and_chunked(fhe, ctx, logn, variant):
    """The two-pass variants with enough rows that every row's cross pass runs in its last
    local-pass CTA (the fused form; smaller calls elsewhere take the stand-alone cross
    launch, and RESCALE's small buffer many chunks)."""
    import torch
    keep = (fhe.fhe_ntt_get_variant(ctx.handle, logn, 0), fhe.fhe_ntt_get_variant(ctx.handle, logn, 1))
    fhe.fhe_ntt_set_variant(ctx.handle, logn, variant)
    n = 1 << logn
    nl, batch = {15: (8, 80), 16: (5, 64)}[logn]        # 640 / 320 rows: above the fusion threshold
    mods = MODS[:nl]
    x = I.uniform_residues(700 + logn + variant, mods, batch, n)
    d = fhe.to_device(x)
    ctx.ntt_fwd(d, logn)
    torch.cuda.synchronize()
    got = fhe.to_host(d)
    ps = psis(mods, n)
    for l in range(nl):
        for b in (0, batch // 3, batch - 1):
            assert (got[l, b] == ON.ntt(x[l, b], mods[l], ps[l])).all(), (l, b)
    ctx.ntt_inv(d, logn)
    assert torch.equal(d, fhe.to_device(x))
    fhe.fhe_ntt_set_variant(ctx.handle, logn, keep[0], keep[1])


@pytest.mark.parametrize("logn", [15, 16])
def test_rescale_two_pass_small_chunks(fhe, logn):
    """RESCALE at N >= 2^15 chunks its NTTs through its own 2-limb buffer (a few rows per
    chunk): bit-exact against the oracle."""
    import torch
    from oracle import ckks as C
    n, nl, batch = 1 << logn, 4, 3
    qs, ps = P.default_moduli(nl, 2)
    prm = C.Params(n, qs, ps, alpha=2)
    c = fhe.Context(logn, qs, ps, alpha=2)
    x = I.uniform_residues(800 + logn, qs, 2 * batch, n)
    ct = x.reshape(nl, 2, batch, n).transpose(1, 0, 2, 3).copy()
    out = c.rescale(fhe.to_device(ct), logn)
    torch.cuda.synchronize()
    got = fhe.to_host(out)
    for b in (0, batch - 1):
        assert (got[:, :, b] == C.rescale(prm, ct[:, :, b].astype(np.uint64))).all(), b
    c.close()


def test_tensor_core_polynomial_chunks(fhe, ctx):
    """N = 2^16 on the tensor-core path with more polynomials than one plane buffer holds (512):
    each limb runs as chunks of 512 and 88 polynomials, whose source rows skip the other chunk's
    polynomials and whose last row tiles run past the chunk. Rows on both sides of the split
    against the oracle; the round trip in full."""
    import torch
    logn, n, first, nl, batch = 16, 1 << 16, 5, 2, 600
    mods = MODS[first:first + nl]
    x = I.uniform_residues(17, mods, batch, n)
    d = fhe.to_device(x)
    ctx.ntt_fwd(d, logn, first_limb=first, path=fhe.FHE_NTT_TC)
    torch.cuda.synchronize()
    got = fhe.to_host(d)
    for l in range(nl):
        for b in (0, 1, 510, 511, 512, 513, 598, 599):
            assert (got[l, b] == ON.ntt(x[l, b], mods[l], P.psi(mods[l], n))).all(), (l, b)
    ctx.ntt_inv(d, logn, first_limb=first, path=fhe.FHE_NTT_TC)
    assert torch.equal(d, fhe.to_device(x))
    fhe.fhe_device_status(ctx.handle, 1)

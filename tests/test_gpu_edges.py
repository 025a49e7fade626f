"""Edge cases on the GPU: empty batches, the smallest and largest ring degrees with a single
polynomial of a single limb, the largest modulus count a context accepts (all limbs
transformed in one call), and the minimum limb counts of the CKKS calls."""
import numpy as np
import pytest

from oracle import ckks as C
from oracle import ntt as ON
from oracle import params as P
from paper_2212_14191_gb300 import inputs as I

pytestmark = pytest.mark.gpu
U64 = np.uint64


@pytest.fixture(scope="module")
def fhe():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_14191_gb300 import fhe as f
    return f


def test_empty_batches_do_nothing(fhe):
    import torch
    qs, ps = P.default_moduli(4, 2)
    ctx = fhe.Context(12, qs, ps, alpha=2)
    for path in (fhe.FHE_NTT_U32, fhe.FHE_NTT_TC):
        fhe.fhe_ntt_fwd(ctx.handle, path, 12, None, 0, 4, 0, 0)      # batch 0, NULL data: accepted
        fhe.fhe_ntt_inv(ctx.handle, path, 12, None, 0, 4, 0, 0)
    fhe.fhe_hmult(ctx.handle, 12, 4, 0, None, None, None, None, None, 0, 0)
    fhe.fhe_hrotate(ctx.handle, 12, 4, 0, 5, None, None, None, None, 0, 0)
    fhe.fhe_cmult(ctx.handle, 12, 4, 0, None, None, None, 0)
    fhe.fhe_hadd(ctx.handle, 12, 4, 0, None, None, None, 0)
    fhe.fhe_automorph(ctx.handle, 12, 0, 5, None, None, 0)
    torch.cuda.synchronize()
    fhe.fhe_device_status(ctx.handle, 1)
    ctx.close()


@pytest.mark.parametrize("logn", [10, 16])
@pytest.mark.parametrize("path", ["u32", "tc"])
def test_single_row_at_extreme_ring_degrees(fhe, logn, path):
    import torch
    n = 1 << logn
    qs = P.ntt_primes(3)
    ctx = fhe.Context(logn, qs)
    p = {"u32": fhe.FHE_NTT_U32, "tc": fhe.FHE_NTT_TC}[path]
    x = I.uniform_residues(logn, qs[2:], 1, n)                       # the last limb only
    d = fhe.to_device(x)
    ctx.ntt_fwd(d, logn, first_limb=2, path=p)
    torch.cuda.synchronize()
    assert (fhe.to_host(d)[0, 0] == ON.ntt(x[0, 0], qs[2], P.psi(qs[2], n))).all()
    ctx.ntt_inv(d, logn, first_limb=2, path=p)
    assert (fhe.to_host(d) == x).all()
    ctx.close()


def test_largest_modulus_count(fhe):
    """64 moduli (56 ciphertext + 8 special primes, the most a context takes), every limb of
    two polynomials at N = 2^16 in one call per direction; sampled rows against the oracle."""
    import torch
    n = 1 << 16
    qs, ps = P.default_moduli(56, 8)
    ctx = fhe.Context(16, qs, ps, alpha=8)
    mods = qs + ps
    x = I.uniform_residues(64, mods, 2, n)
    d = fhe.to_device(x)
    ctx.ntt_fwd(d, 16)
    torch.cuda.synchronize()
    got = fhe.to_host(d)
    for l in (0, 31, 55, 56, 63):
        assert (got[l, 1] == ON.ntt(x[l, 1], mods[l], P.psi(mods[l], n))).all(), l
    ctx.ntt_inv(d, 16)
    assert torch.equal(d, fhe.to_device(x))
    with pytest.raises(fhe.FheError):
        fhe.Context(16, P.default_moduli(57, 8)[0], ps, alpha=8)      # 65 moduli: rejected
    ctx.close()


def test_minimum_limb_counts(fhe):
    """HMULT / RESCALE at 2 limbs, key switching and HROTATE at 1 limb, bit-exact."""
    import torch
    logn = 10
    qs, ps = P.default_moduli(3, 2)
    prm = C.Params(1 << logn, qs, ps, alpha=1)
    s = I.ternary_secret(3, prm.N, hamming_weight=32)
    L = len(qs)
    ar = I.uniform_residues(4, qs + ps, prm.dnum(L), prm.N, dtype=np.uint64).transpose(1, 0, 2)
    evk = C.keygen_evk(prm, s, ar, I.gaussian_error(5, (prm.dnum(L), prm.N)))
    ctx = fhe.Context(logn, qs, ps, alpha=1)
    dev_evk = fhe.to_device(evk.astype(np.uint32))
    a = I.uniform_residues(6, qs[:2], 2, prm.N).reshape(2, 2, 1, prm.N).transpose(1, 0, 2, 3).copy()
    b = I.uniform_residues(7, qs[:2], 2, prm.N).reshape(2, 2, 1, prm.N).transpose(1, 0, 2, 3).copy()
    out = ctx.hmult(fhe.to_device(a), fhe.to_device(b), dev_evk, logn)
    d2 = I.uniform_residues(8, qs[:1], 1, prm.N)
    ks = ctx.keyswitch(fhe.to_device(d2), dev_evk, logn)
    ct1 = a[:, :1].copy()
    rot = ctx.hrotate(fhe.to_device(ct1), dev_evk, logn, 5)            # any key: parity only
    torch.cuda.synchronize()
    assert (fhe.to_host(out)[:, :, 0] == C.hmult(prm, 2, a[:, :, 0].astype(U64), b[:, :, 0].astype(U64), evk)).all()
    k0, k1 = C.keyswitch(prm, 1, d2[:, 0].astype(U64), evk)
    assert (fhe.to_host(ks)[0, :, 0] == k0).all() and (fhe.to_host(ks)[1, :, 0] == k1).all()
    assert (fhe.to_host(rot)[:, :, 0] == C.hrotate(prm, 1, ct1[:, :, 0].astype(U64), evk, 5)).all()
    fhe.fhe_device_status(ctx.handle, 1)
    ctx.close()


def test_expired_device_wait_is_reported_and_the_context_survives(fhe):
    """The failure path of the bounded device waits, without a fault: a kernel whose mbarrier
    wait can never complete gives up after its cycle limit and records FHE_ETIMEOUT; the host
    reads it through fhe_device_status (which clears it), and the same context then transforms
    correctly."""
    import torch
    qs, ps = P.default_moduli(2, 2)
    ctx = fhe.Context(12, qs, ps, alpha=1)
    fhe.fhe_device_status(ctx.handle, 1)
    fhe.fhe_selftest_wait_timeout(ctx.handle, 20_000_000)     # ~10 ms at the SM clock
    torch.cuda.synchronize()
    with pytest.raises(fhe.FheError) as e:
        fhe.fhe_device_status(ctx.handle, 1)
    assert e.value.code == fhe.FHE_ETIMEOUT
    fhe.fhe_device_status(ctx.handle, 0)                       # cleared by the read above
    with pytest.raises(fhe.FheError):
        fhe.fhe_selftest_wait_timeout(ctx.handle, 0)
    x = I.uniform_residues(21, qs, 3, 1 << 12)
    d = fhe.to_device(x)
    ctx.ntt_fwd(d, 12)
    ctx.ntt_inv(d, 12)
    torch.cuda.synchronize()
    assert (fhe.to_host(d) == x).all()
    fhe.fhe_device_status(ctx.handle, 1)
    ctx.close()


def test_hmult_at_the_largest_limb_count(fhe):
    """HMULT with 44 ciphertext limbs and 8 special primes (alpha = 8, dnum = 6): ModUp converts
    into 44 destination limbs, the largest count, on the CUDA cores and on the tensor cores
    (whose accumulators then take 176 of 256 TMEM columns); both equal the oracle."""
    import torch
    logn, nl, K, batch = 12, 44, 8, 1
    n = 1 << logn
    qs, ps = P.default_moduli(nl, K)
    prm = C.Params(n, qs, ps, alpha=8)
    s = I.ternary_secret(800, n, hamming_weight=64)
    arand = I.uniform_residues(801, prm.qs + prm.ps, prm.dnum(nl), n, dtype=np.uint64).transpose(1, 0, 2)
    evk = C.keygen_evk(prm, s, arand, I.gaussian_error(802, (prm.dnum(nl), n)))
    x = I.uniform_residues(803, qs, 4 * batch, n)
    A = x.reshape(nl, 2, 2, batch, n)[:, 0].transpose(1, 0, 2, 3).copy()
    B = x.reshape(nl, 2, 2, batch, n)[:, 1].transpose(1, 0, 2, 3).copy()
    want = C.hmult(prm, nl, A[:, :, 0].astype(U64), B[:, :, 0].astype(U64), evk)
    ctx = fhe.Context(logn, qs, ps, alpha=8)
    da, db, de = fhe.to_device(A), fhe.to_device(B), fhe.to_device(evk.astype(np.uint32))
    for path in (fhe.FHE_CONV_CUDA, fhe.FHE_CONV_TC):
        fhe.fhe_conv_set_path(ctx.handle, path)
        out = ctx.hmult(da, db, de, logn)
        torch.cuda.synchronize()
        assert (fhe.to_host(out)[:, :, 0] == want).all(), path
    fhe.fhe_device_status(ctx.handle, 1)
    ctx.close()

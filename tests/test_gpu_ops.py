"""GPU parity of the other ciphertext operations of Sec. II-B's table against the CPU
oracle: FrobeniusMap (X -> X^k), HROTATE / conjugation, hoisted HROTATE (several rotations
sharing one ModUp), CMULT and HADD, bit-exact on seeded inputs, plus CKKS decryption of a GPU
rotation. The full-size case uses the HMULT
configuration (N = 2^16, 24 + 8 limbs, dnum = 3) with sampled rows."""
import numpy as np
import pytest

from oracle import ckks as C
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


@pytest.fixture(scope="module")
def small(fhe):
    logn = 11
    qs, ps = P.default_moduli(12, 4)
    prm = C.Params(1 << logn, qs, ps, alpha=4)
    s = I.ternary_secret(8, prm.N, hamming_weight=64)
    ctx = fhe.Context(logn, qs, ps, alpha=4)
    yield logn, prm, s, ctx
    ctx.close()


def rot_key(prm, s, k, seed):
    L = len(prm.qs)
    arand = I.uniform_residues(seed, prm.qs + prm.ps, prm.dnum(L), prm.N, dtype=np.uint64).transpose(1, 0, 2)
    return C.keygen_rot(prm, s, k, arand, I.gaussian_error(seed + 1, (prm.dnum(L), prm.N)))


def batch_cts(prm, nl, batch, seed):
    x = I.uniform_residues(seed, prm.qs[:nl], 2 * batch, prm.N)
    return x.reshape(nl, 2, batch, prm.N).transpose(1, 0, 2, 3).copy()


@pytest.mark.parametrize("logn", [10, 13, 16])
def test_automorph_bitexact(fhe, logn):
    import torch
    n = 1 << logn
    mods = P.default_moduli(3, 1)[0]
    ctx = fhe.Context(logn, mods)
    x = I.uniform_residues(logn, mods, 2, n)
    for k in (5, 25, 2 * n - 1, C.galois_rotation(-7, n)):
        out = ctx.automorph(fhe.to_device(x), logn, k)
        torch.cuda.synchronize()
        got = fhe.to_host(out)
        for b in range(2):
            want = C.automorph(x[:, b].astype(U64), mods, [P.psi(q, n) for q in mods], k) if logn < 16 else None
            if want is None:   # 2^16: the permutation the oracle's NTT-domain map equals (pinned on CPU)
                perm = [(((2 * j + 1) * k) % (2 * n) - 1) // 2 for j in range(n)]
                want = x[:, b][:, perm]
            assert (got[:, b] == want).all(), (k, b)
    ctx.close()


@pytest.mark.parametrize("nl", [1, 4, 9, 12])
def test_hrotate_bitexact(fhe, small, nl):
    import torch
    logn, prm, s, ctx = small
    for k in (C.galois_rotation(3, prm.N), C.galois_conjugation(prm.N)):
        ksk = rot_key(prm, s, k, 100 + nl)
        ct = batch_cts(prm, nl, 3, 110 + nl)
        out = ctx.hrotate(fhe.to_device(ct), fhe.to_device(ksk.astype(np.uint32)), logn, k)
        torch.cuda.synchronize()
        got = fhe.to_host(out)
        for b in range(3):
            want = C.hrotate(prm, nl, ct[:, :, b].astype(U64), ksk, k)
            assert (got[:, :, b] == want).all(), (k, b)


@pytest.mark.parametrize("nl", [1, 5, 12])
def test_hrotate_hoisted_bitexact(fhe, small, nl):
    """Three rotations and the conjugation of a batch of two ciphertexts sharing one ModUp,
    against the oracle's hoisted rotation (its own parity definition), bit for bit."""
    import torch
    logn, prm, s, ctx = small
    ks = [C.galois_rotation(3, prm.N), C.galois_conjugation(prm.N), C.galois_rotation(-1, prm.N)]
    keys = [rot_key(prm, s, k, 130 + 2 * i) for i, k in enumerate(ks)]
    ct = batch_cts(prm, nl, 2, 140 + nl)
    out = ctx.hrotate_hoisted(fhe.to_device(ct), [fhe.to_device(k.astype(np.uint32)) for k in keys], logn, ks)
    torch.cuda.synchronize()
    got = fhe.to_host(out)
    assert got.shape == (len(ks), 2, nl, 2, prm.N)
    for b in range(2):
        want = C.hrotate_hoisted(prm, nl, ct[:, :, b].astype(U64), keys, ks)
        for r in range(len(ks)):
            assert (got[r, :, :, b] == want[r]).all(), (nl, b, r)
    fhe.fhe_device_status(ctx.handle, 1)


def test_hrotate_hoisted_arguments(fhe, small):
    import torch
    logn, prm, s, ctx = small
    x = torch.zeros((2, 2, 1, prm.N), dtype=torch.int32, device="cuda")
    y = torch.zeros((2, 2, 2, 1, prm.N), dtype=torch.int32, device="cuda")
    key = torch.zeros(16, dtype=torch.int32, device="cuda")
    p = x.data_ptr()
    # no rotations: nothing to do, no scratch needed
    fhe.fhe_hrotate_hoisted(ctx.handle, logn, 2, 1, [], p, [], y.data_ptr(), 0, 0)
    for g in ([5, 4], [5, 2 * prm.N + 1]):            # an even or out-of-range element
        with pytest.raises(fhe.FheError) as e:
            fhe.fhe_hrotate_hoisted(ctx.handle, logn, 2, 1, g, p, [key.data_ptr()] * 2, y.data_ptr(), p, 16)
        assert e.value.code == fhe.FHE_EINVAL
    with pytest.raises(fhe.FheError) as e:            # output overlapping the input
        fhe.fhe_hrotate_hoisted(ctx.handle, logn, 2, 1, [5, 25], y.data_ptr(), [key.data_ptr()] * 2,
                                y.data_ptr(), p, 16)
    assert e.value.code == fhe.FHE_EINVAL
    with pytest.raises(fhe.FheError) as e:            # scratch too small
        fhe.fhe_hrotate_hoisted(ctx.handle, logn, 2, 1, [5, 25], p, [key.data_ptr()] * 2, y.data_ptr(), p, 16)
    assert e.value.code == fhe.FHE_ENOMEM
    fhe.fhe_device_status(ctx.handle, 1)


def test_hrotate_decrypts_to_rotated_slots(fhe, small):
    import torch
    logn, prm, s, ctx = small
    nl, r = 6, 5
    k = C.galois_rotation(r, prm.N)
    ksk = rot_key(prm, s, k, 120)
    z = I.uniform_reals(121, prm.N // 2)
    delta = 2.0 ** 30
    a = I.uniform_residues(122, prm.qs[:nl], 1, prm.N, dtype=np.uint64)[:, 0]
    ct = C.encrypt(prm, nl, C.encode(z, prm.N, delta), s, a, I.gaussian_error(123, prm.N))
    out = ctx.hrotate(fhe.to_device(ct.astype(np.uint32)[:, :, None]), fhe.to_device(ksk.astype(np.uint32)), logn, k)
    torch.cuda.synchronize()
    dec = C.decrypt_coeffs(prm, fhe.to_host(out)[:, :, 0].astype(U64), s)
    # key-switching noise with P ~ Q_j here: about N (alpha + 1) 19 / delta ~ 2e-4 per slot
    assert np.abs(C.decode(np.array(dec, dtype=float), delta) - np.roll(z, -r)).max() < 2e-3


@pytest.mark.parametrize("nl", [1, 5, 12])
def test_cmult_hadd_bitexact(fhe, small, nl):
    import torch
    logn, prm, s, ctx = small
    mods = prm.qs[:nl]
    a, b = batch_cts(prm, nl, 5, 130 + nl), batch_cts(prm, nl, 5, 140 + nl)
    pt = I.uniform_residues(150 + nl, mods, 5, prm.N)
    da, db, dp = fhe.to_device(a), fhe.to_device(b), fhe.to_device(pt)
    cm = fhe.to_host(ctx.cmult(da, dp, logn))
    ha = fhe.to_host(ctx.hadd(da, db, logn))
    ctx.hadd(da, db, logn, out=da)                      # in place
    torch.cuda.synchronize()
    for k in range(5):
        assert (cm[:, :, k] == C.cmult(prm, nl, a[:, :, k].astype(U64), pt[:, k].astype(U64))).all(), k
        assert (ha[:, :, k] == C.hadd(prm, nl, a[:, :, k].astype(U64), b[:, :, k].astype(U64))).all(), k
    assert (fhe.to_host(da) == ha).all()


def test_ops_bad_arguments(fhe, small):
    logn, prm, s, ctx = small
    import torch
    x = torch.zeros((2, 2, 1, prm.N), dtype=torch.int32, device="cuda")
    y = torch.zeros_like(x)
    for k in (0, 4, 2 * prm.N + 1):                    # even or out of range
        with pytest.raises(fhe.FheError) as e:
            ctx.automorph(x, logn, k, out=y)
        assert e.value.code == fhe.FHE_EINVAL
    with pytest.raises(fhe.FheError):
        ctx.automorph(x, logn, 5, out=x)                # in place
    with pytest.raises(fhe.FheError) as e:
        fhe.fhe_hrotate(ctx.handle, logn, 2, 1, 5, x.data_ptr(), x.data_ptr(), y.data_ptr(), y.data_ptr(), 16)
    assert e.value.code == fhe.FHE_ENOMEM
    fhe.fhe_device_status(ctx.handle, 1)


def test_hrotate_full_size_config(fhe):
    """The benchmarked configuration of the other operations: N = 2^16, 24 ciphertext limbs +
    8 special primes, dnum = 3, 128 ciphertexts in one call, where the ModDown combine's cross
    passes run inside the forward NTT's local-pass launch. The first, middle and last
    ciphertexts of HROTATE, CMULT and HADD against the oracle, bit for bit."""
    import torch
    logn, n, nl, K, batch = 16, 1 << 16, 24, 8, 128
    qs, ps = P.default_moduli(nl, K)
    prm = C.Params(n, qs, ps, alpha=8)
    s = I.ternary_secret(160, n, hamming_weight=64)
    k = C.galois_rotation(1, n)
    ksk = rot_key(prm, s, k, 161)
    ct, ct2 = batch_cts(prm, nl, batch, 162), batch_cts(prm, nl, batch, 163)
    pt = I.uniform_residues(164, qs[:nl], batch, n)
    ctx = fhe.Context(logn, qs, ps, alpha=8)
    da, db, dp = fhe.to_device(ct), fhe.to_device(ct2), fhe.to_device(pt)
    got = fhe.to_host(ctx.hrotate(da, fhe.to_device(ksk.astype(np.uint32)), logn, k))
    cm = fhe.to_host(ctx.cmult(da, dp, logn))
    ha = fhe.to_host(ctx.hadd(da, db, logn))
    torch.cuda.synchronize()
    for b in (0, batch // 2 - 1, batch - 1):
        a_b = ct[:, :, b].astype(U64)
        assert (got[:, :, b] == C.hrotate(prm, nl, a_b, ksk, k)).all(), b
        assert (cm[:, :, b] == C.cmult(prm, nl, a_b, pt[:, b].astype(U64))).all(), b
        assert (ha[:, :, b] == C.hadd(prm, nl, a_b, ct2[:, :, b].astype(U64))).all(), b
    fhe.fhe_device_status(ctx.handle, 1)
    ctx.close()


def test_hrotate_hoisted_full_size_config(fhe):
    """N = 2^16, 24 ciphertext limbs + 8 special primes, dnum = 3, the benchmarked 128
    ciphertexts, a rotation and the conjugation sharing one ModUp: the first, middle and last
    ciphertexts of the GPU result against the oracle's hoisted rotation of that ciphertext,
    bit for bit."""
    import torch
    logn, n, nl, K, batch = 16, 1 << 16, 24, 8, 128
    qs, ps = P.default_moduli(nl, K)
    prm = C.Params(n, qs, ps, alpha=8)
    s = I.ternary_secret(160, n, hamming_weight=64)
    ks = [C.galois_rotation(2, n), C.galois_conjugation(n)]
    keys = [rot_key(prm, s, k, 170 + 2 * i) for i, k in enumerate(ks)]
    ct = batch_cts(prm, nl, batch, 180)
    ctx = fhe.Context(logn, qs, ps, alpha=8)
    out = ctx.hrotate_hoisted(fhe.to_device(ct), [fhe.to_device(k.astype(np.uint32)) for k in keys], logn, ks)
    torch.cuda.synchronize()
    got = fhe.to_host(out)
    for b in (0, batch // 2 - 1, batch - 1):
        want = C.hrotate_hoisted(prm, nl, ct[:, :, b].astype(U64), keys, ks)
        for r in range(len(ks)):
            assert (got[r, :, :, b] == want[r]).all(), (b, r)
    fhe.fhe_device_status(ctx.handle, 1)
    ctx.close()


def test_intt_out_of_place_and_copy_fallback(fhe):
    """N = 2^15, 6 + 2 limbs, 2 ciphertexts: key switching's INTT reads d2 (HMULT) and c1 (hoisted
    rotations) in place when the inverse runs the two-pass kernels (variant 6), and transforms a
    copy when it runs a cluster variant (0). Both give the same results, which also match the
    oracle (HMULT on one pair, the hoisted rotation on one ciphertext)."""
    import torch
    logn, nl, K, batch = 15, 6, 2, 2
    n = 1 << logn
    qs, ps = P.default_moduli(nl, K)
    prm = C.Params(n, qs, ps, alpha=2)
    s = I.ternary_secret(8, n, hamming_weight=64)
    ctx = fhe.Context(logn, qs, ps, alpha=2)
    A, B = batch_cts(prm, nl, batch, 720), batch_cts(prm, nl, batch, 721)
    evk = I.uniform_residues(722, qs + ps, prm.dnum(nl) * 2, n).reshape(
        len(qs) + len(ps), prm.dnum(nl), 2, n).transpose(1, 2, 0, 3).copy()
    ks = [C.galois_rotation(3, n)]
    keys = [rot_key(prm, s, k, 730) for k in ks]
    da, db, de = fhe.to_device(A), fhe.to_device(B), fhe.to_device(evk)
    dk = [fhe.to_device(k.astype(np.uint32)) for k in keys]
    res = {}
    for inv in (6, 0):
        fhe.fhe_ntt_set_variant(ctx.handle, logn, 6, inv)
        res[inv] = (ctx.hmult(da, db, de, logn).clone(), ctx.hrotate_hoisted(da, dk, logn, ks).clone())
    torch.cuda.synchronize()
    assert torch.equal(res[6][0], res[0][0]) and torch.equal(res[6][1], res[0][1])
    got_h, got_r = fhe.to_host(res[6][0]), fhe.to_host(res[6][1])
    want_h = C.hmult(prm, nl, A[:, :, 1].astype(U64), B[:, :, 1].astype(U64), evk.astype(U64))
    assert (got_h[:, :, 1] == want_h).all()
    want_r = C.hrotate_hoisted(prm, nl, A[:, :, 0].astype(U64), keys, ks)
    assert (got_r[0, :, :, 0] == want_r[0]).all()
    fhe.fhe_device_status(ctx.handle, 1)
    ctx.close()


@pytest.mark.parametrize("logn", [14, 15])
def test_moddown_combine_fused_matches_separate(fhe, logn):
    """6 + 2 limbs, 2 ciphertexts: with the plain forward NTT in its fused form (the two-pass
    kernels at 2^15, the one-CTA-per-row shape at 2^14) the ModDown combine of key switching,
    out += (ks - NTT(y)) P^-1, rides on the forward NTT of y (ks and y pre-scaled by P^-1), and
    the HMULT's RESCALE tail likewise; in the other form (a cluster forward variant at 2^15, the
    tensor-core path at 2^14) they run as separate passes. HMULT with and without rescale,
    HROTATE and hoisted rotations give identical results both ways, and match the oracle on one
    ciphertext; key switching alone (no accumulation) keeps the separate form."""
    import torch
    nl, K, batch = 6, 2, 2
    n = 1 << logn
    qs, ps = P.default_moduli(nl, K)
    prm = C.Params(n, qs, ps, alpha=2)
    s = I.ternary_secret(9, n, hamming_weight=64)
    ctx = fhe.Context(logn, qs, ps, alpha=2)
    A, B = batch_cts(prm, nl, batch, 740), batch_cts(prm, nl, batch, 741)
    evk = I.uniform_residues(742, qs + ps, prm.dnum(nl) * 2, n).reshape(
        len(qs) + len(ps), prm.dnum(nl), 2, n).transpose(1, 2, 0, 3).copy()
    ks = [C.galois_rotation(5, n), C.galois_conjugation(n)]
    keys = [rot_key(prm, s, k, 750 + i) for i, k in enumerate(ks)]
    da, db, de = fhe.to_device(A), fhe.to_device(B), fhe.to_device(evk)
    dk = [fhe.to_device(k.astype(np.uint32)) for k in keys]
    fused, separate = ((6, 6), (0, 6)) if logn == 15 else ((0, 0), (fhe.FHE_NTT_VARIANT_TC64,) * 2)
    res = {}
    for name, (fwd, inv) in (("fused", fused), ("separate", separate)):
        fhe.fhe_ntt_set_variant(ctx.handle, logn, fwd, inv)
        res[name] = [ctx.hmult_relin(da, db, de, logn).clone(), ctx.hrotate(da, dk[0], logn, ks[0]).clone(),
                     ctx.hrotate_hoisted(da, dk, logn, ks).clone(), ctx.hmult(da, db, de, logn).clone()]
    torch.cuda.synchronize()
    for x, y in zip(res["fused"], res["separate"]):
        assert torch.equal(x, y)
    relin, rot, hm = fhe.to_host(res["fused"][0]), fhe.to_host(res["fused"][1]), fhe.to_host(res["fused"][3])
    want = C.hmult_relin(prm, nl, A[:, :, 1].astype(U64), B[:, :, 1].astype(U64), evk.astype(U64))
    assert (relin[:, :, 1] == want).all()
    assert (rot[:, :, 0] == C.hrotate(prm, nl, A[:, :, 0].astype(U64), keys[0], ks[0])).all()
    assert (hm[:, :, 0] == C.hmult(prm, nl, A[:, :, 0].astype(U64), B[:, :, 0].astype(U64), evk.astype(U64))).all()
    fhe.fhe_device_status(ctx.handle, 1)
    ctx.close()

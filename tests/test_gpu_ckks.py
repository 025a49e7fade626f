"""GPU parity of the HMULT pipeline (tensor product, key switching, rescale) against
the CPU oracle: bit-exact on seeded inputs, plus CKKS decryption of the GPU result."""
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


def make_key(prm, seed, h=64):
    s = I.ternary_secret(seed, prm.N, hamming_weight=h)
    L = len(prm.qs)
    arand = I.uniform_residues(seed + 1, prm.qs + prm.ps, prm.dnum(L), prm.N, dtype=np.uint64).transpose(1, 0, 2)
    evk = C.keygen_evk(prm, s, arand, I.gaussian_error(seed + 2, (prm.dnum(L), prm.N)))
    return s, evk


def encrypt_pair(prm, nl, s, seed, delta=2.0 ** 30):
    N = prm.N
    z = I.uniform_reals(seed, N // 2)
    m = C.encode(z, N, delta)
    a = I.uniform_residues(seed + 1, prm.qs[:nl], 1, N, dtype=np.uint64)[:, 0]
    return z, C.encrypt(prm, nl, m, s, a, I.gaussian_error(seed + 2, N))


@pytest.fixture(scope="module")
def small(fhe):
    logn = 11
    qs, ps = P.default_moduli(12, 4)
    prm = C.Params(1 << logn, qs, ps, alpha=4)
    s, evk = make_key(prm, 5)
    ctx = fhe.Context(logn, qs, ps, alpha=4)
    yield logn, prm, s, evk, ctx
    ctx.close()


def batch_cts(prm, nl, batch, seed):
    """(2, nl, batch, N) uniform ciphertext residues (uint32)."""
    x = I.uniform_residues(seed, prm.qs[:nl], 2 * batch, prm.N)
    return x.reshape(nl, 2, batch, prm.N).transpose(1, 0, 2, 3).copy()


@pytest.mark.parametrize("nl", [1, 2, 4, 5, 12])
def test_keyswitch_bitexact(fhe, small, nl):
    import torch
    logn, prm, s, evk, ctx = small
    d2 = I.uniform_residues(20 + nl, prm.qs[:nl], 3, prm.N)
    out = ctx.keyswitch(fhe.to_device(d2), fhe.to_device(evk.astype(np.uint32)), logn)
    torch.cuda.synchronize()
    got = fhe.to_host(out)
    for b in range(3):
        k0, k1 = C.keyswitch(prm, nl, d2[:, b].astype(U64), evk)
        assert (got[0, :, b] == k0).all() and (got[1, :, b] == k1).all(), b


@pytest.mark.parametrize("nl,alpha", [(3, 3), (4, 2), (8, 2), (5, 1)])
def test_keyswitch_slice_counts(fhe, nl, alpha):
    """Key switching with dnum = 1, 2, 4 and 5 slices at N = 2^12, 3 ciphertexts: the inner
    product's unrolled kernels (1 to 4 slices) and its generic loop (5) bit-exact against the
    oracle, in HMULT + relinearisation as well."""
    import torch
    logn = 12
    n = 1 << logn
    qs, ps = P.default_moduli(nl, alpha)
    prm = C.Params(n, qs, ps, alpha=alpha)
    dn = prm.dnum(nl)
    evk = I.uniform_residues(60 + nl, qs + ps, 2 * dn, n).reshape(nl + alpha, dn, 2, n).transpose(1, 2, 0, 3).copy()
    d2 = I.uniform_residues(70 + nl, qs, 3, n)
    a, b = batch_cts(prm, nl, 3, 80 + nl), batch_cts(prm, nl, 3, 90 + nl)
    ctx = fhe.Context(logn, qs, ps, alpha=alpha)
    de = fhe.to_device(evk)
    ks = fhe.to_host(ctx.keyswitch(fhe.to_device(d2), de, logn))
    rel = fhe.to_host(ctx.hmult_relin(fhe.to_device(a), fhe.to_device(b), de, logn))
    torch.cuda.synchronize()
    e64 = evk.astype(U64)
    for j in range(3):
        k0, k1 = C.keyswitch(prm, nl, d2[:, j].astype(U64), e64)
        assert (ks[0, :, j] == k0).all() and (ks[1, :, j] == k1).all(), j
        want = C.hmult_relin(prm, nl, a[:, :, j].astype(U64), b[:, :, j].astype(U64), e64)
        assert (rel[:, :, j] == want).all(), j
    fhe.fhe_device_status(ctx.handle, 1)
    ctx.close()


@pytest.mark.parametrize("nl", [2, 3, 7, 12])
def test_rescale_bitexact(fhe, small, nl):
    import torch
    logn, prm, s, evk, ctx = small
    ct = batch_cts(prm, nl, 3, 40 + nl)
    out = ctx.rescale(fhe.to_device(ct), logn)
    torch.cuda.synchronize()
    got = fhe.to_host(out)
    for b in range(3):
        assert (got[:, :, b] == C.rescale(prm, ct[:, :, b].astype(U64))).all(), b


@pytest.mark.parametrize("nl", [2, 5, 9, 12])
def test_hmult_bitexact(fhe, small, nl):
    import torch
    logn, prm, s, evk, ctx = small
    a, b = batch_cts(prm, nl, 3, 60 + nl), batch_cts(prm, nl, 3, 70 + nl)
    dev_evk = fhe.to_device(evk.astype(np.uint32))
    da, db = fhe.to_device(a), fhe.to_device(b)
    relin = ctx.hmult_relin(da, db, dev_evk, logn)
    out = ctx.hmult(da, db, dev_evk, logn)
    torch.cuda.synchronize()
    got_r, got = fhe.to_host(relin), fhe.to_host(out)
    for k in range(3):
        r = C.hmult_relin(prm, nl, a[:, :, k].astype(U64), b[:, :, k].astype(U64), evk)
        assert (got_r[:, :, k] == r).all(), k
        assert (got[:, :, k] == C.rescale(prm, r)).all(), k


def test_hmult_decrypts(fhe, small):
    import torch
    logn, prm, s, evk, ctx = small
    nl = 9
    za, ca = encrypt_pair(prm, nl, s, 200)
    zb, cb = encrypt_pair(prm, nl, s, 300)
    out = ctx.hmult(fhe.to_device(ca[:, :, None, :].astype(np.uint32)),
                    fhe.to_device(cb[:, :, None, :].astype(np.uint32)),
                    fhe.to_device(evk.astype(np.uint32)), logn)
    torch.cuda.synchronize()
    res = fhe.to_host(out)[:, :, 0, :].astype(U64)
    scale = 2.0 ** 60 / prm.qs[nl - 1]
    dec = C.decode(np.array(C.decrypt_coeffs(prm, res, s), dtype=float), scale)
    ref = za * zb
    assert np.abs(dec - ref).max() / np.abs(ref).max() < 1e-5


def _full_size_hmult(fhe, path, genuine, secret_weight=64, seed=1000):
    """N = 2^16, 24 ciphertext limbs + 8 special primes, dnum = 3 (alpha = 8), 128 pairs
    through one fhe_hmult call on a context whose default NTT path is `path`. The pairs at
    `genuine` are encryptions of uniform reals in [-1, 1] at Delta = 2^30 under a ternary
    secret of Hamming weight `secret_weight` (None: dense); the rest are uniform residues.
    Returns (secret, key, inputs A and B, GPU output, slot products of the genuine pairs)."""
    import torch
    logn, N, nl, batch = 16, 1 << 16, 24, 128
    qs, ps = P.default_moduli(24, 8)
    prm = C.Params(N, qs, ps, alpha=8)
    s, evk = make_key(prm, seed, h=secret_weight)
    A = batch_cts(prm, nl, batch, 11)
    B = batch_cts(prm, nl, batch, 12)
    zs = {}
    for k, b in enumerate(genuine):
        za, ca = encrypt_pair(prm, nl, s, 400 + 10 * k)
        zb, cb = encrypt_pair(prm, nl, s, 500 + 10 * k)
        A[:, :, b] = ca
        B[:, :, b] = cb
        zs[b] = za * zb
    ctx = fhe.Context(16, qs, ps, alpha=8, default_path=path)
    out = ctx.hmult(fhe.to_device(A), fhe.to_device(B), fhe.to_device(evk.astype(np.uint32)), logn)
    torch.cuda.synchronize()
    fhe.fhe_device_status(ctx.handle, 1)
    got = fhe.to_host(out)
    ctx.close()
    return prm, s, evk, A, B, got, zs


def _decode_error(prm, nl, ct, s, z):
    """max_j |dec_j - z_j| / max_j |z_j| of the rescaled product (scale Delta^2 / q_(nl-1))."""
    scale = 2.0 ** 60 / prm.qs[nl - 1]
    dec = C.decode(np.array(C.decrypt_coeffs(prm, ct.astype(U64), s), dtype=float), scale)
    return np.abs(dec - z).max() / np.abs(z).max()


@pytest.mark.parametrize("path", ["u32", "tc"])
def test_hmult_full_size_config(fhe, path):
    """The benchmarked HMULT configuration on both NTT paths: N = 2^16, 24 + 8 limbs, dnum = 3,
    128 pairs in one call. Pairs b = 0, 63 and 127 (first, middle and last of the batch, so
    the 128 x 72 extended limbs' chunking through the tensor-core plane buffer is crossed)
    are compared with the oracle bit for bit; the genuine pairs b = 0 and 127 (sparse ternary
    secret, h = 64) decrypt to the slot products within 1e-5."""
    nl = 24
    p = fhe.FHE_NTT_U32 if path == "u32" else fhe.FHE_NTT_TC
    prm, s, evk, A, B, got, zs = _full_size_hmult(fhe, p, genuine=(0, 127))
    for b in (0, 63, 127):
        want = C.hmult(prm, nl, A[:, :, b].astype(U64), B[:, :, b].astype(U64), evk)
        assert (got[:, :, b] == want).all(), b
    for b, z in zs.items():
        assert _decode_error(prm, nl, got[:, :, b], s, z) < 1e-5, b


def test_hmult_dense_ternary_error(fhe):
    """Precision with a dense ternary secret (each coefficient uniform in {-1, 0, 1}) at the
    benchmarked shape (N = 2^16, 24 + 8 limbs, dnum = 3, 128 pairs; four genuine pairs). The
    1e-5 target is stated for the sparse secret (h = 64): with a dense one the rescale's
    rounding error r0 + r1 s grows with the secret's weight (about 2N/3 nonzero coefficients), so
    1e-5 is not claimed here. The test checks bit-exactness on one pair, prints the measured
    maximum relative error per genuine pair and bounds it loosely by 5e-4 (the oracle's own
    HMULT of the same pairs gives about 1e-4)."""
    nl = 24
    genuine = (0, 42, 85, 127)
    prm, s, evk, A, B, got, zs = _full_size_hmult(fhe, fhe.FHE_NTT_U32, genuine=genuine, secret_weight=None,
                                                  seed=1500)
    assert np.count_nonzero(s) > prm.N // 2          # dense: about 2N/3 nonzero coefficients
    want = C.hmult(prm, nl, A[:, :, 0].astype(U64), B[:, :, 0].astype(U64), evk)
    assert (got[:, :, 0] == want).all()
    errs = [_decode_error(prm, nl, got[:, :, b], s, zs[b]) for b in genuine]
    print("dense ternary HMULT max relative error per pair:", ["%.3e" % e for e in errs])
    assert max(errs) < 5e-4


def test_hmult_tensor_core_path(fhe):
    """The whole HMULT with the tensor-core NTT as the context's default path."""
    import torch
    logn, nl = 12, 6
    qs, ps = P.default_moduli(8, 4)
    prm = C.Params(1 << logn, qs, ps, alpha=4)
    s, evk = make_key(prm, 77)
    ctx = fhe.Context(logn, qs, ps, alpha=4, default_path=fhe.FHE_NTT_TC)
    a, b = batch_cts(prm, nl, 2, 81), batch_cts(prm, nl, 2, 82)
    out = ctx.hmult(fhe.to_device(a), fhe.to_device(b), fhe.to_device(evk.astype(np.uint32)), logn)
    torch.cuda.synchronize()
    fhe.fhe_device_status(ctx.handle, 1)
    got = fhe.to_host(out)
    for k in range(2):
        want = C.hmult(prm, nl, a[:, :, k].astype(U64), b[:, :, k].astype(U64), evk)
        assert (got[:, :, k] == want).all(), k
    ctx.close()


@pytest.mark.parametrize("logn,L,K", [(12, 2, 2), (13, 4, 4), (14, 7, 8)])
def test_hmult_heax_sets_bitexact(fhe, logn, L, K):
    """The paper's HEAX comparison sets in 30-bit primes (L ciphertext limbs + K special
    primes, one key-switching slice): HMULT + relinearisation + rescale bit-exact, plus the
    relinearised product decrypting to a*b."""
    import torch
    n = 1 << logn
    allp = P.ntt_primes(L + K)
    ps, qs = allp[:K], allp[K:]
    prm = C.Params(n, qs, ps, alpha=L)
    s, evk = make_key(prm, 300 + logn)
    a, b = batch_cts(prm, L, 2, 310 + logn), batch_cts(prm, L, 2, 320 + logn)
    ctx = fhe.Context(logn, qs, ps, alpha=L)
    out = ctx.hmult(fhe.to_device(a), fhe.to_device(b), fhe.to_device(evk.astype(np.uint32)), logn)
    torch.cuda.synchronize()
    got = fhe.to_host(out)
    for k in range(2):
        want = C.hmult(prm, L, a[:, :, k].astype(U64), b[:, :, k].astype(U64), evk)
        assert (got[:, :, k] == want).all(), k
    za, ca = encrypt_pair(prm, L, s, 330 + logn, delta=2.0 ** 25)
    zb, cb = encrypt_pair(prm, L, s, 340 + logn, delta=2.0 ** 25)
    rel = ctx.hmult_relin(fhe.to_device(ca.astype(np.uint32)[:, :, None]),
                          fhe.to_device(cb.astype(np.uint32)[:, :, None]), fhe.to_device(evk.astype(np.uint32)), logn)
    torch.cuda.synchronize()
    dec = C.decrypt_coeffs(prm, fhe.to_host(rel)[:, :, 0].astype(U64), s, n_crt=L)
    zz = C.decode(np.array(dec, dtype=float), 2.0 ** 50)
    assert np.abs(zz - za * zb).max() < 1e-3
    fhe.fhe_device_status(ctx.handle, 1)
    ctx.close()


@pytest.mark.parametrize("logn,L,K", [(12, 2, 2), (13, 4, 4), (14, 7, 8)])
def test_hmult_heax_sets_benchmarked_batch(fhe, logn, L, K):
    """The HEAX sets at the benchmark's 1024 ciphertexts per call: every stage on its full grid,
    and at N = 2^13 and 2^14 the fused RESCALE tail's cross pass inside the local-pass launch (a
    separate launch at batch 2, and at 2^12 with 1024 too): HMULT + relinearisation + rescale
    bit-exact against the oracle on sampled pairs."""
    import torch
    from paper_2212_14191_gb300 import configs as CFG
    n, batch = 1 << logn, CFG.HEAX_BATCH
    allp = P.ntt_primes(L + K)
    ps, qs = allp[:K], allp[K:]
    prm = C.Params(n, qs, ps, alpha=L)
    _, evk = make_key(prm, 350 + logn)
    a, b = batch_cts(prm, L, batch, 360 + logn), batch_cts(prm, L, batch, 370 + logn)
    ctx = fhe.Context(logn, qs, ps, alpha=L)
    out = ctx.hmult(fhe.to_device(a), fhe.to_device(b), fhe.to_device(evk.astype(np.uint32)), logn)
    torch.cuda.synchronize()
    got = fhe.to_host(out)
    for k in (0, batch // 2 - 1, batch - 1):
        want = C.hmult(prm, L, a[:, :, k].astype(U64), b[:, :, k].astype(U64), evk)
        assert (got[:, :, k] == want).all(), k
    fhe.fhe_device_status(ctx.handle, 1)
    ctx.close()


def _extreme(mods, count, n, kind):
    """(len(mods), count, n) uint32 residues at the ends of each range: all q - 1 ("max") or
    q - 1 at even and 0 at odd coefficients ("alt")."""
    q = np.array(mods, dtype=np.uint64)[:, None, None]
    x = np.broadcast_to(q - 1, (len(mods), count, n)).copy()
    if kind == "alt":
        x[:, :, 1::2] = 0
    return x.astype(np.uint32)


@pytest.mark.parametrize("logn,batch", [(12, 2), (15, 2), (16, 32)])
def test_ckks_ops_extreme_residues(fhe, logn, batch):
    """Ciphertexts, d2 and keys at the ends of every residue range (all q - 1, or q - 1 and 0
    alternating), 6 + 2 limbs, dnum = 3: HMULT, HMULT + relinearisation, key switching, RESCALE,
    HROTATE and hoisted rotations (a rotation and the conjugation) bit-exact against the oracle
    for every ciphertext of the batch. These are the inputs that push the lazy reductions
    (Shoup, Montgomery, the fused tails' loads) to the top of their ranges; at N = 2^16 with 32
    ciphertexts the fused tails' cross passes run inside the local-pass launch, at 2^15 in a
    separate one, at 2^12 on the one-CTA-per-row shape."""
    import torch
    nl, K, alpha = 6, 2, 2
    n = 1 << logn
    qs, ps = P.default_moduli(nl, K)
    prm = C.Params(n, qs, ps, alpha=alpha)
    dn = prm.dnum(nl)
    a = np.stack([_extreme(qs, batch, n, "max"), _extreme(qs, batch, n, "alt")])
    b = np.stack([_extreme(qs, batch, n, "alt"), _extreme(qs, batch, n, "max")])
    evk = _extreme(qs + ps, 2 * dn, n, "max").reshape(nl + K, dn, 2, n).transpose(1, 2, 0, 3).copy()
    k = C.galois_rotation(1, n)
    ctx = fhe.Context(logn, qs, ps, alpha=alpha)
    da, db, de = fhe.to_device(a), fhe.to_device(b), fhe.to_device(evk)
    got = {"hmult": ctx.hmult(da, db, de, logn), "relin": ctx.hmult_relin(da, db, de, logn),
           "ks": ctx.keyswitch(da[0].contiguous(), de, logn), "rescale": ctx.rescale(da, logn),
           "hrotate": ctx.hrotate(da, de, logn, k),
           "hoisted": ctx.hrotate_hoisted(da, [de, de], logn, [k, C.galois_conjugation(n)])}
    torch.cuda.synchronize()
    got = {name: fhe.to_host(v) for name, v in got.items()}
    a0, b0, e64 = a[:, :, 0].astype(U64), b[:, :, 0].astype(U64), evk.astype(U64)
    want = {"hmult": C.hmult(prm, nl, a0, b0, e64), "relin": C.hmult_relin(prm, nl, a0, b0, e64),
            "ks": np.stack(C.keyswitch(prm, nl, a0[0], e64)), "rescale": C.rescale(prm, a0),
            "hrotate": C.hrotate(prm, nl, a0, e64, k)}
    for name in want:
        for j in range(batch):
            assert (got[name][:, :, j] == want[name]).all(), (name, j)
    hw = C.hrotate_hoisted(prm, nl, a0, [e64, e64], [k, C.galois_conjugation(n)])
    for r in range(2):
        for j in range(batch):
            assert (got["hoisted"][r, :, :, j] == hw[r]).all(), (r, j)
    fhe.fhe_device_status(ctx.handle, 1)
    ctx.close()


def test_concurrent_streams_share_a_context(fhe):
    """HMULTs of one context on eight streams at once, with the two-pass NTT variants (whose
    chunk buffer each call takes from its own scratch): every result equals the result of the
    same inputs run alone."""
    import torch
    logn, nl, K, batch = 15, 6, 2, 4
    n = 1 << logn
    qs, ps = P.default_moduli(nl, K)
    prm = C.Params(n, qs, ps, alpha=2)
    s, evk = make_key(prm, 400)
    ctx = fhe.Context(logn, qs, ps, alpha=2)
    fhe.fhe_ntt_set_variant(ctx.handle, logn, 7, 7)            # two-pass both ways
    dev_evk = fhe.to_device(evk.astype(np.uint32))
    ins = [(fhe.to_device(batch_cts(prm, nl, batch, 410 + 2 * k)), fhe.to_device(batch_cts(prm, nl, batch, 411 + 2 * k)))
           for k in range(8)]
    alone = []
    for a, b in ins:                                          # one at a time, default stream
        alone.append(ctx.hmult(a, b, dev_evk, logn).clone())
    torch.cuda.synchronize()
    nbytes = fhe.fhe_scratch_bytes(ctx.handle, fhe.FHE_OP_HMULT, logn, nl, batch)
    streams = [torch.cuda.Stream() for _ in ins]
    scratch = [torch.empty(nbytes // 4 + 4, dtype=torch.int32, device="cuda") for _ in ins]
    outs = [torch.empty_like(x) for x in alone]
    for rep in range(3):
        for k, (a, b) in enumerate(ins):
            fhe.fhe_hmult(ctx.handle, logn, nl, batch, a.data_ptr(), b.data_ptr(), dev_evk.data_ptr(),
                          outs[k].data_ptr(), scratch[k].data_ptr(), nbytes, streams[k].cuda_stream)
        torch.cuda.synchronize()
        for k in range(len(ins)):
            assert torch.equal(outs[k], alone[k]), (rep, k)
    got = fhe.to_host(alone[0])
    a0, b0 = fhe.to_host(ins[0][0]), fhe.to_host(ins[0][1])
    assert (got[:, :, 0] == C.hmult(prm, nl, a0[:, :, 0].astype(U64), b0[:, :, 0].astype(U64), evk)).all()
    fhe.fhe_device_status(ctx.handle, 1)
    ctx.close()


@pytest.mark.parametrize("logn", [12, 15])
def test_concurrent_streams_tensor_core_context(fhe, logn):
    """HMULTs of one context whose default NTT path is the tensor-core one, on four streams at
    once: each call's digit planes live in its own scratch, so every result equals the same
    HMULT run alone; one pair is compared with the oracle."""
    import torch
    nl, K, batch = 6, 2, 3
    n = 1 << logn
    qs, ps = P.default_moduli(nl, K)
    prm = C.Params(n, qs, ps, alpha=2)
    s, evk = make_key(prm, 440 + logn)
    ctx = fhe.Context(logn, qs, ps, alpha=2, default_path=fhe.FHE_NTT_TC)
    dev_evk = fhe.to_device(evk.astype(np.uint32))
    ins = [(fhe.to_device(batch_cts(prm, nl, batch, 450 + 2 * k)), fhe.to_device(batch_cts(prm, nl, batch, 451 + 2 * k)))
           for k in range(4)]
    alone = []
    for a, b in ins:
        alone.append(ctx.hmult(a, b, dev_evk, logn).clone())
        torch.cuda.synchronize()
    nbytes = fhe.fhe_scratch_bytes(ctx.handle, fhe.FHE_OP_HMULT, logn, nl, batch)
    streams = [torch.cuda.Stream() for _ in ins]
    scratch = [torch.empty(nbytes // 4 + 4, dtype=torch.int32, device="cuda") for _ in ins]
    outs = [torch.empty_like(x) for x in alone]
    for rep in range(3):
        for k, (a, b) in enumerate(ins):
            fhe.fhe_hmult(ctx.handle, logn, nl, batch, a.data_ptr(), b.data_ptr(), dev_evk.data_ptr(),
                          outs[k].data_ptr(), scratch[k].data_ptr(), nbytes, streams[k].cuda_stream)
        torch.cuda.synchronize()
        for k in range(len(ins)):
            assert torch.equal(outs[k], alone[k]), (rep, k)
    got = fhe.to_host(alone[1])
    a1, b1 = fhe.to_host(ins[1][0]), fhe.to_host(ins[1][1])
    assert (got[:, :, 2] == C.hmult(prm, nl, a1[:, :, 2].astype(U64), b1[:, :, 2].astype(U64), evk)).all()
    fhe.fhe_device_status(ctx.handle, 1)
    ctx.close()


def test_hmult_fused_rescale_tail_wide_shapes(fhe):
    """N = 2^16: the fused tail in the default two-pass shape (512-thread CTAs, C = 4) and in the
    256-thread shape with C = 8 sub-transforms per row (whose cross pass loads ks and d at the
    store), both against the tail run as separate passes."""
    import torch
    logn, nl, K, batch = 16, 3, 2, 2
    n = 1 << logn
    qs, ps = P.default_moduli(nl, K)
    prm = C.Params(n, qs, ps, alpha=2)
    s, evk = make_key(prm, 650)
    A, B = batch_cts(prm, nl, batch, 651), batch_cts(prm, nl, batch, 652)
    ctx = fhe.Context(logn, qs, ps, alpha=2)
    da, db, de = fhe.to_device(A), fhe.to_device(B), fhe.to_device(evk.astype(np.uint32))
    fhe.fhe_ntt_set_variant(ctx.handle, logn, 0, 6)             # cluster forward: separate passes
    sep = ctx.hmult(da, db, de, logn).clone()
    for fwd in (6, 7):
        fhe.fhe_ntt_set_variant(ctx.handle, logn, fwd, 6)
        fused = ctx.hmult(da, db, de, logn).clone()
        torch.cuda.synchronize()
        assert torch.equal(fused, sep), fwd
    fhe.fhe_device_status(ctx.handle, 1)
    ctx.close()


@pytest.mark.parametrize("fwd_variant", [7, 6])
def test_hmult_fused_rescale_tail(fhe, fwd_variant):
    """The RESCALE tail fused into the two-pass forward NTT (z built on load, the output combined
    on store) against the same HMULT with a forward variant that runs the tail as separate
    passes: identical outputs for every pair, and the oracle on two of them. N = 2^15, 6 + 2
    limbs, 5 pairs (a batch that is not a multiple of the row chunking)."""
    import torch
    logn, nl, K, batch = 15, 6, 2, 5
    n = 1 << logn
    qs, ps = P.default_moduli(nl, K)
    prm = C.Params(n, qs, ps, alpha=2)
    s, evk = make_key(prm, 600)
    A, B = batch_cts(prm, nl, batch, 610), batch_cts(prm, nl, batch, 611)
    za, ca = encrypt_pair(prm, nl, s, 620)
    zb, cb = encrypt_pair(prm, nl, s, 630)
    A[:, :, 2], B[:, :, 2] = ca, cb
    ctx = fhe.Context(logn, qs, ps, alpha=2)
    da, db, de = fhe.to_device(A), fhe.to_device(B), fhe.to_device(evk.astype(np.uint32))
    fhe.fhe_ntt_set_variant(ctx.handle, logn, fwd_variant, 7)   # two-pass forward: fused tail
    fused = ctx.hmult(da, db, de, logn).clone()
    fhe.fhe_ntt_set_variant(ctx.handle, logn, 0, 7)             # cluster forward: separate passes
    sep = ctx.hmult(da, db, de, logn).clone()
    torch.cuda.synchronize()
    assert torch.equal(fused, sep)
    got = fhe.to_host(fused)
    for b in (0, 2):
        want = C.hmult(prm, nl, A[:, :, b].astype(U64), B[:, :, b].astype(U64), evk)
        assert (got[:, :, b] == want).all(), b
    dec = C.decode(np.array(C.decrypt_coeffs(prm, got[:, :, 2].astype(U64), s), dtype=float),
                   2.0 ** 60 / qs[nl - 1])
    assert np.abs(dec - za * zb).max() / np.abs(za * zb).max() < 1e-5
    fhe.fhe_device_status(ctx.handle, 1)
    ctx.close()


@pytest.mark.parametrize("logn,nl,K,alpha,batch", [(12, 6, 2, 2, 3), (11, 12, 5, 5, 2), (13, 9, 4, 3, 1)])
def test_tensor_core_conv_matches_cuda_core(fhe, logn, nl, K, alpha, batch):
    """Key switching and HMULT with the basis conversion on the tensor cores and on the CUDA
    cores (the default): identical results (both are the exact sum of Sec. IV-A's Conv), and
    the oracle on one ciphertext. Source counts 2..5, short last slices, ragged batches."""
    import torch
    n = 1 << logn
    qs, ps = P.default_moduli(nl, K)
    prm = C.Params(n, qs, ps, alpha=alpha)
    s, evk = make_key(prm, 700 + logn)
    A, B = batch_cts(prm, nl, batch, 710), batch_cts(prm, nl, batch, 711)
    ctx = fhe.Context(logn, qs, ps, alpha=alpha)
    assert fhe.fhe_conv_get_path(ctx.handle) == fhe.FHE_CONV_CUDA
    da, db, de = fhe.to_device(A), fhe.to_device(B), fhe.to_device(evk.astype(np.uint32))
    d2 = fhe.to_device(I.uniform_residues(712, qs[:nl], batch, n))
    res = {}
    for path in (fhe.FHE_CONV_TC, fhe.FHE_CONV_CUDA):
        fhe.fhe_conv_set_path(ctx.handle, path)
        res[path] = (ctx.hmult(da, db, de, logn).clone(), ctx.keyswitch(d2, de, logn).clone())
    torch.cuda.synchronize()
    for x, y in zip(res[fhe.FHE_CONV_TC], res[fhe.FHE_CONV_CUDA]):
        assert torch.equal(x, y)
    got = fhe.to_host(res[fhe.FHE_CONV_TC][0])
    want = C.hmult(prm, nl, A[:, :, 0].astype(U64), B[:, :, 0].astype(U64), evk)
    assert (got[:, :, 0] == want).all()
    with pytest.raises(fhe.FheError):
        fhe.fhe_conv_set_path(ctx.handle, 7)
    fhe.fhe_device_status(ctx.handle, 1)
    ctx.close()

"""Pins for the CKKS oracle (oracle/ckks.py) against exact big-integer
mathematics, not against itself:

* Conv returns x + u*B with 0 <= u < |B| (CRT lift, python big ints);
* ModDown returns floor(X / P) - u with 0 <= u < K (CRT lift);
* RESCALE returns round(X / q_l) exactly (CRT lift; q_l odd, so no ties);
* the tensor product decrypts as (c0 + c1 s)(c0' + c1' s) under (1, s, s^2);
* KeySwitch(d2) decrypts to d2 s^2 plus an error within the analytic bound;
* the canonical embedding agrees with direct complex evaluation and is a ring
  homomorphism for the product in R[X]/(X^N+1);
* decrypt(HMULT(enc a, enc b)) = a*b within 1e-5 (sparse ternary secret);
* the automorphism X -> X^k agrees with term-by-term evaluation at the roots
  through the brute-force Eq. (4) transform, obeys the group law, permutes
  NTT slots, and rotates / conjugates the canonical-embedding slots;
* decrypt(HROTATE(enc m)) = m(X^k) within the key-switching bound, and
  CMULT / HADD decrypt exactly to the schoolbook product / the sum;
* hoisted rotations: the permuted ModUp digits differ from ModUp of the permuted
  c1 by exactly -B_j times the count of nonzero y_i at negated coefficients (big
  ints), k = 1 reproduces HROTATE, and every rotation decrypts within the bound;
* the inverse Galois element by Newton's iteration equals the modular inverse, and
  permuting the key by sigma_{k^-1} and the inner product by sigma_k reproduces the
  hoisted rotation bit for bit.
"""
import math

import numpy as np
import pytest

from oracle import ckks as C
from oracle import params as P
from paper_2212_14191_gb300 import inputs as I

U64 = np.uint64


def lift(res, mods):
    """(k, N) residues -> list of python ints in [0, prod)."""
    M = math.prod(mods)
    out = []
    for n in range(res.shape[1]):
        x = 0
        for i, m in enumerate(mods):
            Mi = M // m
            x += int(res[i, n]) * Mi * pow(Mi % m, -1, m)
        out.append(x % M)
    return out


@pytest.fixture(scope="module")
def small():
    qs, ps = P.default_moduli(12, 4)
    prm = C.Params(256, qs, ps, alpha=4)
    s = I.ternary_secret(11, prm.N, hamming_weight=64)
    L = len(qs)
    arand = I.uniform_residues(12, qs + ps, prm.dnum(L), prm.N, dtype=np.uint64).transpose(1, 0, 2)
    erand = I.gaussian_error(13, (prm.dnum(L), prm.N))
    evk = C.keygen_evk(prm, s, arand, erand)
    return prm, s, evk


@pytest.mark.parametrize("nsrc,ndst", [(1, 3), (4, 6), (3, 2)])
def test_conv_is_x_plus_uB(nsrc, ndst):
    qs = P.ntt_primes(nsrc + ndst)
    src, dst = qs[:nsrc], qs[nsrc:]
    N = 64
    x = I.uniform_residues(nsrc, src, 1, N, dtype=np.uint64)[:, 0]
    y = C.conv(x, src, dst)
    X = lift(x, src)
    B = math.prod(src)
    ybig = [0] * N
    for i, b in enumerate(src):
        bh = B // b
        for n in range(N):
            ybig[n] += (int(x[i, n]) * pow(bh % b, -1, b) % b) * bh
    for n in range(N):
        u, r = divmod(ybig[n] - X[n], B)
        assert r == 0 and 0 <= u < nsrc
        for t_i, t in enumerate(dst):
            assert int(y[t_i, n]) == ybig[n] % t


def test_moddown_is_floor_div_P(small):
    prm, _, _ = small
    nl = 5
    mods = prm.qs[:nl] + prm.ps
    psis = prm.psi_q[:nl] + prm.psi_p
    ks_c = I.uniform_residues(21, mods, 1, prm.N, dtype=np.uint64)[:, 0]
    out = C.moddown(prm, nl, C.ntt(ks_c, mods, psis))
    out_c = C.intt(out, prm.qs[:nl], prm.psi_q[:nl])
    X = lift(ks_c, mods)
    Q = math.prod(prm.qs[:nl])
    got = lift(out_c, prm.qs[:nl])
    for n in range(prm.N):
        u = (X[n] // prm.P - got[n]) % Q
        assert 0 <= u < prm.K


@pytest.mark.parametrize("nl", [2, 3, 7])
def test_rescale_is_round_div_ql(small, nl):
    prm, _, _ = small
    mods, psis = prm.qs[:nl], prm.psi_q[:nl]
    c = I.uniform_residues(30 + nl, mods, 2, prm.N, dtype=np.uint64).transpose(1, 0, 2)
    out = C.rescale(prm, np.stack([C.ntt(c[k], mods, psis) for k in range(2)]))
    ql = mods[-1]
    for k in range(2):
        X = lift(c[k], mods)
        got = C.intt(out[k], mods[:-1], psis[:-1])
        for n in range(prm.N):
            want = (2 * X[n] + ql) // (2 * ql)      # round to nearest, ql odd
            for i, q in enumerate(mods[:-1]):
                assert int(got[i, n]) == want % q


def test_tensor_decrypts_under_1_s_s2(small):
    prm, s, _ = small
    nl = 4
    mods, psis = prm.qs[:nl], prm.psi_q[:nl]
    ca = I.uniform_residues(40, mods, 2, prm.N, dtype=np.uint64).transpose(1, 0, 2)
    cb = I.uniform_residues(41, mods, 2, prm.N, dtype=np.uint64).transpose(1, 0, 2)
    d0, d1, d2 = C.tensor(ca, cb, mods)
    sn = C.ntt(C.small_to_residues(s, mods), mods, psis)
    lhs = C.add(C.add(d0, C.hada(d1, sn, mods), mods), C.hada(d2, C.hada(sn, sn, mods), mods), mods)
    rhs = C.hada(C.add(ca[0], C.hada(ca[1], sn, mods), mods),
                 C.add(cb[0], C.hada(cb[1], sn, mods), mods), mods)
    assert (lhs == rhs).all()


@pytest.mark.parametrize("nl", [1, 4, 6, 9, 12])
def test_keyswitch_error_bound(small, nl):
    """ks0 + ks1 s - d2 s^2 is small in the coefficient domain.

    Bound: sum over slices of N * (alpha + 1) * (Q_j / P) * max|e|, plus the
    ModDown rounding (1 + ||s||_1)(K + 1).
    """
    prm, s, evk = small
    mods, psis = prm.qs[:nl], prm.psi_q[:nl]
    d2 = I.uniform_residues(50 + nl, mods, 1, prm.N, dtype=np.uint64)[:, 0]
    k0, k1 = C.keyswitch(prm, nl, d2, evk)
    sn = C.ntt(C.small_to_residues(s, mods), mods, psis)
    diff = C.sub(C.add(k0, C.hada(k1, sn, mods), mods), C.hada(d2, C.hada(sn, sn, mods), mods), mods)
    err = C.crt_centered(C.intt(diff, mods, psis), mods)
    bound = 0.0
    for j in range(prm.dnum(nl)):
        Qj = math.prod(prm.qs[i] for i in prm.slice_limbs(j, nl))
        bound += prm.N * (prm.alpha + 1) * Qj / prm.P * 19
    bound += (1 + int(np.abs(s).sum())) * (prm.K + 1)
    assert max(abs(e) for e in err) <= bound
    assert math.prod(mods) > 1e6 * bound   # the check is meaningful


def test_embedding_matches_direct_evaluation():
    N = 32
    m = np.random.default_rng(3).normal(size=N)
    zeta = np.exp(1j * np.pi / N)
    direct = np.array([sum(m[n] * zeta ** ((2 * k + 1) * n) for n in range(N)) for k in range(N)])
    assert np.allclose(C.embed(m), direct, atol=1e-9)
    z = np.random.default_rng(4).uniform(-1, 1, N // 2) + 1j * np.random.default_rng(5).uniform(-1, 1, N // 2)
    mm = C.encode(z, N, 2.0 ** 40)
    assert np.abs(C.decode(np.array(mm, dtype=float), 2.0 ** 40) - z).max() < N * 2.0 ** -40
    for j, k in enumerate(C.slot_index(N)):
        assert np.isclose(zeta ** (2 * k + 1), zeta ** pow(5, j, 2 * N))


def test_embedding_is_multiplicative():
    N = 64
    za, zb = I.uniform_reals(1, N // 2), I.uniform_reals(2, N // 2)
    ma, mb = C.encode(za, N, 2.0 ** 20), C.encode(zb, N, 2.0 ** 20)
    full = [0] * (2 * N)
    for i in range(N):
        for j in range(N):
            full[i + j] += ma[i] * mb[j]
    prod = np.array([full[k] - full[k + N] for k in range(N)], dtype=float)
    assert np.abs(C.decode(prod, 2.0 ** 40) - za * zb).max() < 1e-4


def _hmult_case(N, nq, nl, h, seed):
    qs, ps = P.default_moduli(nq, 8)
    prm = C.Params(N, qs, ps, alpha=8)
    s = I.ternary_secret(seed, N, hamming_weight=h)
    L = len(qs)
    arand = I.uniform_residues(seed + 1, qs + ps, prm.dnum(L), N, dtype=np.uint64).transpose(1, 0, 2)
    evk = C.keygen_evk(prm, s, arand, I.gaussian_error(seed + 2, (prm.dnum(L), N)))
    delta = 2.0 ** 30
    za, zb = I.uniform_reals(seed + 3, N // 2), I.uniform_reals(seed + 4, N // 2)
    cts = []
    for k, z in enumerate((za, zb)):
        m = C.encode(z, N, delta)
        a = I.uniform_residues(seed + 5 + k, qs[:nl], 1, N, dtype=np.uint64)[:, 0]
        cts.append(C.encrypt(prm, nl, m, s, a, I.gaussian_error(seed + 7 + k, N)))
    out = C.hmult(prm, nl, cts[0], cts[1], evk)
    scale = delta * delta / qs[nl - 1]
    dec = C.decode(np.array(C.decrypt_coeffs(prm, out, s), dtype=float), scale)
    ref = za * zb
    return np.abs(dec - ref).max() / np.abs(ref).max()


@pytest.mark.parametrize("N,nq,nl", [(1024, 24, 24), (1024, 24, 9), (2048, 12, 3)])
def test_hmult_decrypts_to_product(N, nq, nl):
    assert _hmult_case(N, nq, nl, 64, 70 + nl) < 1e-5


def test_hmult_constant():
    """Encryptions of constants: every slot of the product equals the product constant."""
    N, nl = 512, 5
    qs, ps = P.default_moduli(8, 8)
    prm = C.Params(N, qs, ps, alpha=8)
    s = I.ternary_secret(90, N, hamming_weight=64)
    arand = I.uniform_residues(91, qs + ps, 1, N, dtype=np.uint64).transpose(1, 0, 2)
    evk = C.keygen_evk(prm, s, arand, I.gaussian_error(92, (1, N)))
    delta = 2.0 ** 30
    cts = []
    for k, v in enumerate((0.75, -0.5)):
        m = C.encode(np.full(N // 2, v), N, delta)
        assert m[0] == round(v * delta) and all(c == 0 for c in m[1:])
        a = I.uniform_residues(93 + k, qs[:nl], 1, N, dtype=np.uint64)[:, 0]
        cts.append(C.encrypt(prm, nl, m, s, a, I.gaussian_error(95 + k, N)))
    out = C.hmult(prm, nl, cts[0], cts[1], evk)
    dec = C.decode(np.array(C.decrypt_coeffs(prm, out, s), dtype=float), delta * delta / qs[nl - 1])
    assert np.abs(dec - (-0.375)).max() < 1e-6


# --------------------------------------------------------------------------
# FrobeniusMap / HROTATE, CMULT, HADD


def test_automorph_is_substitution_x_to_xk():
    """NTT(a(X^k))[j] equals sum_n a_n psi^((2j+1) n k), evaluated term by term with python
    ints through the brute-force Eq. (4) transform (not through automorph_coeff's index map)."""
    from oracle import ntt as ON
    N = 32
    q = P.ntt_primes(1, logn_max=5, bits=12)[0]
    psi = P.psi(q, N)
    a = I.uniform_residues(3, [q], 1, N, dtype=np.uint64)[:, 0]
    for k in (3, 5, 25, 2 * N - 1, 2 * N - 3):
        b = C.automorph_coeff(a, [q], k)[0]
        got = ON.ntt_brute(b.astype(np.uint32), q, psi)
        for j in range(N):
            x = pow(psi, 2 * j + 1, q)
            want = sum(int(a[0, n]) * pow(x, n * k, q) for n in range(N)) % q
            assert int(got[j]) == want, (k, j)


def test_automorph_group_law_and_ntt_permutation():
    N = 64
    qs = P.ntt_primes(2, logn_max=6, bits=20)
    psis = [P.psi(q, N) for q in qs]
    a = I.uniform_residues(4, qs, 1, N, dtype=np.uint64)[:, 0]
    assert (C.automorph_coeff(a, qs, 1) == a).all()
    for k, l in ((3, 5), (5, 2 * N - 1), (7, 77)):
        lhs = C.automorph_coeff(C.automorph_coeff(a, qs, l), qs, k)
        assert (lhs == C.automorph_coeff(a, qs, (k * l) % (2 * N))).all()
    # in the NTT domain the map only permutes: output j takes input j' with
    # 2j' + 1 = (2j + 1) k mod 2N
    A = C.ntt(a, qs, psis)
    for k in (3, 5, 2 * N - 1):
        B = C.automorph(A, qs, psis, k)
        perm = [(((2 * j + 1) * k) % (2 * N) - 1) // 2 for j in range(N)]
        assert (B == A[:, perm]).all()


def _int_automorph(coeffs, k, mods):
    """Integer polynomial through automorph_coeff on residues and a CRT lift (centred)."""
    res = C.small_to_residues(np.asarray(coeffs, dtype=np.int64), mods)
    return C.crt_centered(C.automorph_coeff(res, mods, k), mods)


@pytest.mark.parametrize("r", [1, 3, -2])
def test_rotation_rotates_slots(r):
    N = 128
    mods = P.ntt_primes(3, logn_max=7, bits=30)
    z = I.uniform_reals(5 + r % 7, N // 2) + 1j * I.uniform_reals(9 + r % 5, N // 2)
    m = C.encode(z, N, 2.0 ** 30)
    k = C.galois_rotation(r, N)
    out = C.decode(np.array(_int_automorph(m, k, mods), dtype=float), 2.0 ** 30)
    assert np.abs(out - np.roll(z, -r)).max() < 1e-6


def test_conjugation_conjugates_slots():
    N = 128
    mods = P.ntt_primes(3, logn_max=7, bits=30)
    z = I.uniform_reals(6, N // 2) + 1j * I.uniform_reals(7, N // 2)
    m = C.encode(z, N, 2.0 ** 30)
    out = C.decode(np.array(_int_automorph(m, C.galois_conjugation(N), mods), dtype=float), 2.0 ** 30)
    assert np.abs(out - np.conj(z)).max() < 1e-6


@pytest.mark.parametrize("nl,r", [(4, 1), (9, -3), (12, 5)])
def test_hrotate_decrypts_to_rotation(small, nl, r):
    """decrypt(HROTATE(enc m)) = m(X^k) + e(X^k) + key-switching error (same bound as the
    key-switching test plus the fresh error), and its slots are the rotated slots."""
    prm, s, _ = small
    k = C.galois_rotation(r, prm.N)
    L = len(prm.qs)
    arand = I.uniform_residues(60 + nl, prm.qs + prm.ps, prm.dnum(L), prm.N, dtype=np.uint64).transpose(1, 0, 2)
    ksk = C.keygen_rot(prm, s, k, arand, I.gaussian_error(61 + nl, (prm.dnum(L), prm.N)))
    z = I.uniform_reals(62 + nl, prm.N // 2)
    delta = 2.0 ** 25
    m = C.encode(z, prm.N, delta)
    a = I.uniform_residues(63 + nl, prm.qs[:nl], 1, prm.N, dtype=np.uint64)[:, 0]
    ct = C.encrypt(prm, nl, m, s, a, I.gaussian_error(64 + nl, prm.N))
    out = C.hrotate(prm, nl, ct, ksk, k)
    dec = C.decrypt_coeffs(prm, out, s, n_crt=min(nl, 3))
    want = _int_automorph(m, k, prm.qs[:3])
    bound = 19.0
    for j in range(prm.dnum(nl)):
        Qj = math.prod(prm.qs[i] for i in prm.slice_limbs(j, nl))
        bound += prm.N * (prm.alpha + 1) * Qj / prm.P * 19
    bound += (1 + int(np.abs(s).sum())) * (prm.K + 1)
    assert max(abs(x - y) for x, y in zip(dec, want)) <= bound
    slots = C.decode(np.array(dec, dtype=float), delta)
    assert np.abs(slots - np.roll(z, -r)).max() < 1e-2


def test_cmult_and_hadd_decrypt_exactly(small):
    """decrypt(CMULT(enc m, p)) = (m + e) p and decrypt(HADD(enc m1, enc m2)) = m1 + e1 + m2 + e2
    exactly, with the negacyclic product from the schoolbook oracle."""
    from oracle import ntt as ON
    prm, s, _ = small
    nl = 3
    mods, psis = prm.qs[:nl], prm.psi_q[:nl]
    g = np.random.default_rng(71)
    m1 = g.integers(-1000, 1000, prm.N)
    m2 = g.integers(-1000, 1000, prm.N)
    p = g.integers(-50, 50, prm.N)
    e1, e2 = I.gaussian_error(72, prm.N), I.gaussian_error(73, prm.N)
    a1 = I.uniform_residues(74, mods, 1, prm.N, dtype=np.uint64)[:, 0]
    a2 = I.uniform_residues(75, mods, 1, prm.N, dtype=np.uint64)[:, 0]
    ct1 = C.encrypt(prm, nl, m1, s, a1, e1)
    ct2 = C.encrypt(prm, nl, m2, s, a2, e2)
    q0 = prm.qs[0]
    pt = C.ntt(C.small_to_residues(p, mods), mods, psis)
    dec = C.decrypt_coeffs(prm, C.cmult(prm, nl, ct1, pt), s)
    want = ON.negacyclic_mul(np.mod(m1 + e1, q0).astype(np.uint32), np.mod(p, q0).astype(np.uint32), q0)
    want = [int(w) - q0 if int(w) > q0 // 2 else int(w) for w in want]
    assert dec == want
    dec = C.decrypt_coeffs(prm, C.hadd(prm, nl, ct1, ct2), s)
    assert dec == [int(v) for v in (m1 + e1 + m2 + e2)]


@pytest.mark.parametrize("nl", [2, 5, 12])
def test_fused_moddown_rescale_is_exact(small, nl):
    """Reading 20 on the CPU: the fused tail (one NTT of z_i = y_i P^-1 + [last]_i, output
    (ks_i P^-1 + d_i - z^_i) q_l^-1) and its scaled form (d'_i = d_i q_l^-1,
    ks'_i = ks_i P^-1 q_l^-1, y'_i = y_i P^-1 q_l^-1, output ks'_i + d'_i - NTT(y'_i +
    [last]_i q_l^-1)) both equal relinearisation followed by RESCALE bit for bit."""
    prm, s, evk = small
    N = prm.N
    qm, psi = prm.qs[:nl], prm.psi_q[:nl]
    ql, l = prm.qs[nl - 1], nl - 1
    ct_a = I.uniform_residues(70 + nl, qm, 2, N, dtype=np.uint64).transpose(1, 0, 2)
    ct_b = I.uniform_residues(80 + nl, qm, 2, N, dtype=np.uint64).transpose(1, 0, 2)
    want = C.hmult(prm, nl, ct_a, ct_b, evk)
    d0, d1, d2 = C.tensor(ct_a, ct_b, qm)
    ks = C.inner_product(prm, nl, d2, evk)
    pinv = np.array([pow(prm.P % q, -1, q) for q in qm], dtype=U64)[:, None]
    qlinv = np.array([pow(ql, -1, q) if q != ql else 0 for q in qm], dtype=U64)[:, None]
    mods = np.array(qm, dtype=U64)[:, None]
    for c, d in enumerate((d0, d1)):
        k = ks[c]
        y = C.conv(C.intt(k[nl:], prm.ps, prm.psi_p), prm.ps, qm)            # coefficient domain
        # the last relinearised limb in the coefficient domain, centred
        rel_l = (C.sub(k[l:l + 1], C.ntt(y[l:l + 1], [ql], [psi[l]]), [ql]) * pinv[l]) % ql
        rel_l = (rel_l + d[l:l + 1]) % ql
        last = C.intt(rel_l, [ql], [psi[l]])[0].astype(np.int64)
        last = np.where(last > (ql - 1) // 2, last - ql, last)
        x = C.small_to_residues(last, qm[:l])                                # [last]_i, i < l
        m = mods[:l]
        # fused form of reading 20
        z = ((y[:l] * pinv[:l]) % m + x) % m
        out = (((k[:l] * pinv[:l]) % m + d[:l]) % m + m - C.ntt(z, qm[:l], psi[:l])) % m
        out = (out * qlinv[:l]) % m
        assert (out == want[c]).all(), (nl, c)
        # scaled form (the GPU's fused tail)
        sc = (pinv[:l] * qlinv[:l]) % m
        ks_s, d_s, y_s = (k[:l] * sc) % m, (d[:l] * qlinv[:l]) % m, (y[:l] * sc) % m
        z_s = (y_s + (x * qlinv[:l]) % m) % m
        out_s = ((ks_s + d_s) % m + m - C.ntt(z_s, qm[:l], psi[:l])) % m
        assert (out_s == want[c]).all(), (nl, c)


def _rot_key(prm, s, k, seed):
    L = len(prm.qs)
    arand = I.uniform_residues(seed, prm.qs + prm.ps, prm.dnum(L), prm.N, dtype=np.uint64).transpose(1, 0, 2)
    return C.keygen_rot(prm, s, k, arand, I.gaussian_error(seed + 1, (prm.dnum(L), prm.N)))


@pytest.mark.parametrize("nl", [5, 12])
def test_hoisted_digits_differ_by_multiples_of_Qj(small, nl):
    """Hoisting's one departure from hrotate, exactly: in the coefficient domain the permuted
    digit automorph(ModUp_j(c1)) and ModUp_j(c1(X^k)) agree on slice j's own limbs, and on every
    other limb differ by -B_j #{i : y_i != 0} at each coefficient that X -> X^k negates and by 0
    at the others, with y_i = [c1_i (B_j/b_i)^-1]_{b_i} taken at the source coefficient."""
    prm, _, _ = small
    N, k = prm.N, C.galois_rotation(3, prm.N)
    mods, psis = prm.qs[:nl], prm.psi_q[:nl]
    emods, epsis = prm.qs[:nl] + prm.ps, prm.psi_q[:nl] + prm.psi_p
    c1 = I.uniform_residues(90 + nl, mods, 1, N, dtype=np.uint64)[:, 0]
    c1c = C.intt(c1, mods, psis)
    c1k = C.automorph(c1, mods, psis, k)
    c1kc = C.intt(c1k, mods, psis)
    nonzero_seen = 0
    for j in range(prm.dnum(nl)):
        own = prm.slice_limbs(j, nl)
        Bj = math.prod(prm.qs[i] for i in own)
        hoisted = C.intt(C.automorph(C.modup(prm, nl, c1, c1c, j), emods, epsis, k), emods, epsis)
        direct = C.intt(C.modup(prm, nl, c1k, c1kc, j), emods, epsis)
        cnt = np.zeros(N, dtype=np.int64)
        for i in own:
            b = prm.qs[i]
            y = (c1c[i] * U64(pow((Bj // b) % b, -1, b))) % U64(b)
            cnt += (y != 0)
        want = [0] * N
        for n in range(N):
            t = (n * k) % (2 * N)
            if t >= N:
                want[t - N] = -Bj * int(cnt[n])
        for r, m in enumerate(emods):
            diff = (hoisted[r].astype(np.int64) - direct[r].astype(np.int64)) % m
            expect = np.array([w % m for w in want], dtype=np.int64)
            np.testing.assert_array_equal(diff, expect, err_msg="slice %d limb %d" % (j, r))
            nonzero_seen += int((diff != 0).sum())
    assert nonzero_seen > 0   # the two forms really differ, so the parity definition matters


def test_hoisted_identity_rotation_equals_hrotate(small):
    """With k = 1 the automorphism is the identity and hoisting changes nothing: bit-exact."""
    prm, s, evk = small
    nl = 7
    ct = I.uniform_residues(95, prm.qs[:nl], 2, prm.N, dtype=np.uint64).transpose(1, 0, 2)
    out = C.hrotate_hoisted(prm, nl, ct, [evk], [1])
    assert out.shape == (1, 2, nl, prm.N)
    assert (out[0] == C.hrotate(prm, nl, ct, evk, 1)).all()


def test_hoisted_rotations_decrypt_to_rotations(small):
    """decrypt(hoisted HROTATE_k(enc m)) = m(X^k) within the key-switching bound (the hoisted
    digits are lifts in (-alpha B_j, alpha B_j) instead of [0, alpha B_j), the same magnitude),
    for three rotations and the conjugation of one ciphertext, and the slots are rotated /
    conjugated; each agrees with the unhoisted HROTATE to within twice that bound."""
    prm, s, _ = small
    nl, N = 9, prm.N
    rs = [1, -3, 5]
    ks = [C.galois_rotation(r, N) for r in rs] + [C.galois_conjugation(N)]
    keys = [_rot_key(prm, s, k, 300 + 2 * i) for i, k in enumerate(ks)]
    z = I.uniform_reals(310, N // 2)
    delta = 2.0 ** 25
    m = C.encode(z, N, delta)
    a = I.uniform_residues(311, prm.qs[:nl], 1, N, dtype=np.uint64)[:, 0]
    ct = C.encrypt(prm, nl, m, s, a, I.gaussian_error(312, N))
    outs = C.hrotate_hoisted(prm, nl, ct, keys, ks)
    bound = 19.0
    for j in range(prm.dnum(nl)):
        Qj = math.prod(prm.qs[i] for i in prm.slice_limbs(j, nl))
        bound += N * (prm.alpha + 1) * Qj / prm.P * 19
    bound += (1 + int(np.abs(s).sum())) * (prm.K + 1)
    for i, k in enumerate(ks):
        dec = C.decrypt_coeffs(prm, outs[i], s, n_crt=3)
        want = _int_automorph(m, k, prm.qs[:3])
        assert max(abs(x - y) for x, y in zip(dec, want)) <= bound
        ref = C.decrypt_coeffs(prm, C.hrotate(prm, nl, ct, keys[i], k), s, n_crt=3)
        assert max(abs(x - y) for x, y in zip(dec, ref)) <= 2 * bound
        slots = C.decode(np.array(dec, dtype=float), delta)
        target = np.roll(z, -rs[i]) if i < len(rs) else np.conj(z)
        assert np.abs(slots - target).max() < 1e-2


def _newton_inv_pow2(k, bits):
    """Inverse of an odd k modulo 2^bits (bits <= 32) by Newton's iteration x <- x (2 - k x)
    in 32-bit wrap-around arithmetic: x = k is right to 3 bits (k^2 = 1 mod 8) and each step
    doubles that, so five steps give 96 >= 32 bits."""
    x = k
    for _ in range(5):
        x = (x * ((2 - k * x) % 2 ** 32)) % 2 ** 32
    return x % (2 ** bits)


def test_newton_inverse_of_galois_elements():
    """The inverse Galois element k^-1 mod 2N for every odd k at N = 2^10 and a sample at
    2^16: k k^-1 = 1 mod 2N and it equals Python's modular inverse."""
    for logn in (10, 16):
        two_n = 2 ** (logn + 1)
        ks = range(1, two_n, 2) if logn == 10 else [1, 3, 5, 25, 5 ** 7 % two_n, two_n - 1, 2 ** logn + 1]
        for k in ks:
            kinv = _newton_inv_pow2(k, logn + 1)
            assert (k * kinv) % two_n == 1
            assert kinv == pow(k, -1, two_n)


def test_hoisted_key_permutation_order(small):
    """The hoisted rotation can permute each key by sigma_{k^-1} once, take the inner product
    with the unpermuted ModUp digits and permute that sum by sigma_k: since sigma_k only
    permutes NTT slots it commutes with the slot-wise product, so
    sum_j sigma_k(d_j) (.) e_j = sigma_k(sum_j d_j (.) sigma_{k^-1}(e_j)) exactly. With ModDown
    and c0(X^k) added, this order reproduces hrotate_hoisted bit for bit (k a rotation and
    the conjugation); sigma_{k^-1} sigma_k is the identity on the extended limbs."""
    prm, s, _ = small
    nl, N = 7, prm.N
    mods, psis = prm.qs[:nl], prm.psi_q[:nl]
    emods = prm.qs[:nl] + prm.ps
    epsis = prm.psi_q[:nl] + prm.psi_p
    ct = I.uniform_residues(320, mods, 2, N, dtype=np.uint64).transpose(1, 0, 2)
    c1_coeff = C.intt(ct[1], mods, psis)
    digits = [C.modup(prm, nl, ct[1], c1_coeff, j) for j in range(prm.dnum(nl))]
    for i, k in enumerate((C.galois_rotation(3, N), C.galois_conjugation(N))):
        key = _rot_key(prm, s, k, 330 + 2 * i)
        kinv = _newton_inv_pow2(k, int(math.log2(N)) + 1)
        assert (C.automorph(C.automorph(digits[0], emods, epsis, k), emods, epsis, kinv) == digits[0]).all()
        ks = []
        for c in range(2):
            acc = np.zeros((nl + prm.K, N), dtype=U64)
            for j, dt in enumerate(digits):
                ek = C.evk_at_level(prm, key, j, nl)[c]
                acc = C.add(acc, C.hada(dt, C.automorph(ek, emods, epsis, kinv), emods), emods)
            ks.append(C.automorph(acc, emods, epsis, k))
        c0 = C.automorph(ct[0], mods, psis, k)
        got = np.stack([C.add(c0, C.moddown(prm, nl, ks[0]), mods),
                        C.moddown(prm, nl, ks[1]) % np.array(mods, dtype=U64)[:, None]])
        assert (got == C.hrotate_hoisted(prm, nl, ct, [key], [k])[0]).all()


def test_conv_hand_worked_example():
    """The oracle's Conv against the hand-worked example in tests/golden/conv_b5_7_t11_13.txt
    (Sec. IV-A): x = 1 and x = 23 come back as x + 35, the approximate conversion's u = 1."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "conv_b5_7_t11_13.txt")
    rows = {}
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            k, *vals = line.split()
            rows[k] = [int(v) for v in vals]
    src, dst, x = rows["src"], rows["dst"], np.array(rows["x"], dtype=U64)
    res = np.stack([x % U64(b) for b in src])
    out = C.conv(res, src, dst)
    assert out[0].tolist() == rows["out11"] and out[1].tolist() == rows["out13"]
    assert [v % 11 for v in rows["lift"]] == rows["out11"]
    assert all((l - v) % 35 == 0 and 0 <= (l - v) // 35 < len(src) for l, v in zip(rows["lift"], rows["x"]))

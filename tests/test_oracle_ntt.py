"""Pins for the NTT oracle (oracle/ntt_oracle.c, oracle/params.py).

Every check here ties the oracle to something other than itself: a worked
example computed by hand from Eq. (4), polynomial evaluation at the roots of
X^N + 1 (Horner), closed forms for monomials, the schoolbook product in
Z_q[X]/(X^N+1) (convolution theorem, Sec. II-A Eq. (3)), INTT(NTT(x)) = x (the
correctness check of Sec. VI-A), linearity, and library primality.
"""
import math

import numpy as np
import pytest

from oracle import ntt as O
from oracle import params as P
from tests.conftest import golden

Q30 = P.ntt_primes(4)


def horner_at_odd_roots(a, q, psi):
    """a(psi^(2k+1)) for k < N: Eq. (4) read as evaluation at the roots of X^N+1."""
    N = len(a)
    out = []
    for k in range(N):
        x = pow(psi, 2 * k + 1, q)
        acc = 0
        for c in reversed([int(v) for v in a]):
            acc = (acc * x + c) % q
        out.append(acc)
    return np.array(out, dtype=np.uint32)


def test_hand_worked_example():
    g = golden("ntt_q17_n4.txt")
    q, n, psi = g["q"][0], g["n"][0], g["psi"][0]
    assert P.psi(q, n) == psi
    assert [pow(psi, e, q) for e in range(8)] == g["powers"]
    a = np.array(g["a"], dtype=np.uint32)
    assert O.ntt_brute(a, q, psi).tolist() == g["A"]
    assert O.ntt(a, q, psi).tolist() == g["A"]
    assert O.intt(np.array(g["A"], dtype=np.uint32), q, psi).tolist() == g["a"]
    assert O.intt_brute(np.array(g["A"], dtype=np.uint32), q, psi).tolist() == g["a"]


def test_primes_and_roots():
    qs, ps = P.default_moduli(44, 8)
    allp = ps + qs
    assert len(set(allp)) == 52
    assert allp == sorted(allp, reverse=True)
    sympy = pytest.importorskip("sympy")
    for q in allp:
        assert sympy.isprime(q)
        assert (q - 1) % (1 << 17) == 0 and (1 << 29) < q < (1 << 30)
    # nothing skipped between consecutive candidates
    step = 1 << 17
    for hi, lo in zip(allp, allp[1:]):
        for c in range(lo + step, hi, step):
            assert not sympy.isprime(c)
    # P exceeds every slice product Q_j of alpha = 8 primes (Sec. II-B, GKS)
    Pp = math.prod(ps)
    for j in range(0, 44, 8):
        assert Pp > math.prod(qs[j:j + 8])
    for q in allp[:6]:
        for logn in (4, 10, 12, 16):
            n = 1 << logn
            r = P.psi(q, n)
            assert pow(r, n, q) == q - 1 and pow(r, 2 * n, q) == 1
            if logn > 4:
                assert P.psi(q, n // 2) == r * r % q


@pytest.mark.parametrize("q,n", [(17, 8), (97, 16), (Q30[0], 8), (Q30[1], 32), (Q30[2], 64)])
def test_brute_equals_evaluation_at_roots(q, n):
    psi = P.psi(q, n)
    a = np.random.default_rng(n).integers(0, q, n, dtype=np.uint64).astype(np.uint32)
    A = O.ntt_brute(a, q, psi)
    assert (A == horner_at_odd_roots(a, q, psi)).all()
    # the evaluation points are the N distinct roots of X^N + 1
    pts = {pow(psi, 2 * k + 1, q) for k in range(n)}
    assert len(pts) == n and all(pow(x, n, q) == q - 1 for x in pts)


def test_monomials_exhaustive_tiny_prime():
    """Every c * X^j over Z_17, N = 8: NTT is c * psi^((2k+1) j) (closed form)."""
    q, n = 17, 8
    psi = P.psi(q, n)
    for j in range(n):
        for c in range(q):
            a = np.zeros(n, dtype=np.uint32)
            a[j] = c
            want = [c * pow(psi, (2 * k + 1) * j, q) % q for k in range(n)]
            assert O.ntt(a, q, psi).tolist() == want
            assert O.ntt_brute(a, q, psi).tolist() == want
            assert O.intt(np.array(want, dtype=np.uint32), q, psi).tolist() == a.tolist()


@pytest.mark.parametrize("logn", [3, 5, 8, 10])
def test_fast_equals_brute(logn):
    n = 1 << logn
    for q in Q30[:2]:
        psi = P.psi(q, n)
        a = np.random.default_rng(logn).integers(0, q, n, dtype=np.uint64).astype(np.uint32)
        assert (O.ntt(a, q, psi) == O.ntt_brute(a, q, psi)).all()
        A = O.ntt(a, q, psi)
        assert (O.intt(A, q, psi) == O.intt_brute(A, q, psi)).all()


@pytest.mark.parametrize("logn", [4, 8, 10])
def test_convolution_theorem(logn):
    """Schoolbook product in Z_q[X]/(X^N+1) == INTT(NTT(a) . NTT(b)) (Sec. II-A)."""
    n = 1 << logn
    q = Q30[0]
    psi = P.psi(q, n)
    g = np.random.default_rng(100 + logn)
    a = g.integers(0, q, n, dtype=np.uint64).astype(np.uint32)
    b = g.integers(0, q, n, dtype=np.uint64).astype(np.uint32)
    prod = (O.ntt(a, q, psi).astype(np.uint64) * O.ntt(b, q, psi).astype(np.uint64)) % q
    assert (O.intt(prod.astype(np.uint32), q, psi) == O.negacyclic_mul(a, b, q)).all()
    # and the schoolbook routine against python big-int negacyclic reduction
    if logn <= 4:
        full = [0] * (2 * n)
        for i in range(n):
            for j in range(n):
                full[i + j] += int(a[i]) * int(b[j])
        want = [(full[k] - full[k + n]) % q for k in range(n)]
        assert O.negacyclic_mul(a, b, q).tolist() == want


@pytest.mark.parametrize("logn", [12, 16])
def test_roundtrip_and_linearity(logn):
    n = 1 << logn
    q = Q30[1]
    psi = P.psi(q, n)
    g = np.random.default_rng(logn)
    a = g.integers(0, q, n, dtype=np.uint64).astype(np.uint32)
    b = g.integers(0, q, n, dtype=np.uint64).astype(np.uint32)
    A, B = O.ntt(a, q, psi), O.ntt(b, q, psi)
    assert (O.intt(A, q, psi) == a).all()
    s = ((a.astype(np.uint64) + b) % q).astype(np.uint32)
    assert (O.ntt(s, q, psi) == ((A.astype(np.uint64) + B) % q)).all()
    # X^1 closed form at full size
    x = np.zeros(n, dtype=np.uint32)
    x[1] = 1
    k = np.arange(n, dtype=object)
    assert O.ntt(x, q, psi).tolist() == [pow(psi, 2 * int(kk) + 1, q) for kk in k]


def test_batch_matches_single():
    qs = Q30[:3]
    n = 256
    psis = [P.psi(q, n) for q in qs]
    x = np.stack([np.random.default_rng(i).integers(0, q, (5, n), dtype=np.uint64)
                  for i, q in enumerate(qs)]).astype(np.uint32)
    y, used = O.ntt_batch(x, qs, psis)
    assert used >= 1
    for l in range(3):
        for b in range(5):
            assert (y[l, b] == O.ntt(x[l, b], qs[l], psis[l])).all()
    z, _ = O.ntt_batch(y, qs, psis, inverse=True)
    assert (z == x).all()


# ---- the readings of Sec. IV-B Eq. (9) and the Sec. IV-C segmentation ---------


def _matmul_mod(A, B, q):
    return np.array(np.dot(A.astype(object), B.astype(object)) % q, dtype=np.uint64)


@pytest.mark.parametrize("n1,n2", [(8, 8), (16, 16), (32, 8), (4, 64)])
def test_four_step_identity(n1, n2):
    """A[k1 + N1 k2] = sum_n2 w^(n2 k2) psi^((2k1+1) n2) sum_n1 psi^(N2(2k1+1)n1) a[N2 n1 + n2].

    W1 = psi_2N1^(2ij+j), W2 = psi_2N^(2ij+j), W3 = psi_2N2^(2ij) as printed in
    Sec. IV-B; the output of the last product is k1-major and lands in natural
    order through a transposed store.
    """
    n = n1 * n2
    q = Q30[0]
    psi = P.psi(q, n)
    a = np.random.default_rng(n1 * 7 + n2).integers(0, q, n, dtype=np.uint64)
    amat = a.reshape(n1, n2)
    psi1 = pow(psi, n2, q)            # primitive 2N1-th root
    W1 = np.array([[pow(psi1, 2 * i * j + j, q) for j in range(n1)] for i in range(n1)], dtype=object)
    W2 = np.array([[pow(psi, 2 * i * j + j, q) for j in range(n2)] for i in range(n1)], dtype=object)
    w_n2 = pow(psi, 2 * n1, q)        # psi_(2N2)^2 : primitive N2-th root
    W3 = np.array([[pow(w_n2, i * j, q) for j in range(n2)] for i in range(n2)], dtype=object)
    assert pow(pow(psi, n1, q), 2, q) == w_n2
    Bm = _matmul_mod(W1, amat, q)
    Cm = np.array((Bm.astype(object) * W2) % q, dtype=np.uint64)
    Dm = _matmul_mod(Cm, W3, q)       # [k1][k2]
    out = Dm.T.reshape(-1)            # out[k1 + N1 k2] = Dm[k1][k2]
    assert (out.astype(np.uint32) == O.ntt_brute(a.astype(np.uint32), q, psi)).all()


def test_segment_fusion_identities():
    """u32 -> four 8-bit planes (Sec. IV-C, Stage 1) and their fusion (Stages 3/5).

    Unsigned planes: sum_{i,j} 2^(8(i+j)) W_i T_j = W a exactly; balanced planes
    d in [-128, 127] reconstruct a exactly; the concatenated-K form
    sum_i 2^(8i) sum_j [W 2^(8j) mod q]_i T_j = W a (mod q).
    """
    q = Q30[0]
    g = np.random.default_rng(5)
    K = 64
    W = g.integers(0, q, (8, K), dtype=np.uint64).astype(object)
    a = g.integers(0, q, (K, 4), dtype=np.uint64).astype(object)
    exact = W.dot(a)

    def planes(x):
        return [(x >> (8 * j)) & 255 for j in range(4)]

    Wp, Tp = planes(W), planes(a)
    fused = sum((Wp[i].dot(Tp[j])) << (8 * (i + j)) for i in range(4) for j in range(4))
    assert (fused == exact).all()
    assert max(int(v) for i in range(4) for j in range(4) for v in Wp[i].dot(Tp[j]).ravel()) \
        <= K * 255 * 255

    def balanced(x):
        ds, r = [], x
        for _ in range(4):
            d = ((r + 128) & 255) - 128
            ds.append(d)
            r = (r - d) >> 8
        assert (r == 0).all()
        return ds

    edge = np.array([0, 1, 127, 128, 255, 256, q - 1, (1 << 30) - 1, 0x7F7F7F7F & ((1 << 30) - 1),
                     0x3F808080], dtype=object)
    for x in (edge, a.ravel()):
        ds = balanced(x)
        assert all(((d >= -128) & (d <= 127)).all() for d in ds)
        assert (sum(ds[j] * (1 << (8 * j)) for j in range(4)) == x).all()
    Wj = [(W * (1 << (8 * j))) % q for j in range(4)]
    acc = [sum(planes(Wj[j])[i].dot(Tp[j]) for j in range(4)) for i in range(4)]
    assert (sum(acc[i] << (8 * i) for i in range(4)) % q == exact % q).all()


@pytest.mark.parametrize("n,c", [(64, 2), (64, 4), (128, 8), (256, 4)])
def test_two_pass_dit_identity(n, c):
    """Reading 21, the plain path's two-pass forward: with N = NC C,
    B_j = NTT_NC(a[j + C m]) under the root psi^C, and A[k' + NC t] =
    sum_j w^(t j) psi^((2k'+1) j) B_j[k'] with w = psi^(2 NC) (a C-th root of unity).
    psi^C is the library's own NC-point root (psi_{N/2} = psi_N^2), so the local pass is the
    plain NC-point transform with its own tables."""
    q = Q30[1]
    psi = P.psi(q, n)
    nc = n // c
    psi_c = pow(psi, c, q)
    assert psi_c == P.psi(q, nc)
    w = pow(psi, 2 * nc, q)
    assert pow(w, c, q) == 1 and (c == 1 or pow(w, c // 2, q) == q - 1)
    a = np.random.default_rng(n + c).integers(0, q, n, dtype=np.uint64).astype(np.uint32)
    B = [O.ntt_brute(a[j::c].copy(), q, psi_c) for j in range(c)]
    out = np.zeros(n, dtype=np.uint64)
    for t in range(c):
        for k in range(nc):
            acc = 0
            for j in range(c):
                acc += pow(w, t * j, q) * pow(psi, (2 * k + 1) * j, q) * int(B[j][k])
            out[k + nc * t] = acc % q
    assert (out.astype(np.uint32) == O.ntt_brute(a, q, psi)).all()


@pytest.mark.parametrize("n1,n2", [(4, 4), (8, 4), (16, 8), (32, 32)])
def test_inverse_four_step_identity(n1, n2):
    """The inverse in four-step form (Eq. (2)-(3) with the index maps of Eq. (9)):
    a[N2 n1 + n2] = N^-1 sum_k1 psi^(-N2 (2k1+1) n1) psi^(-(2k1+1) n2)
                    sum_k2 psi^(-2 N1 n2 k2) A[k1 + N1 k2],
    a GEMM over k2, a Hadamard twiddle carrying N^-1, a GEMM over k1, against brute force."""
    n = n1 * n2
    q = Q30[2]
    psi = P.psi(q, n)
    pinv = pow(psi, -1, q)
    ninv = pow(n, -1, q)
    A = np.random.default_rng(n1 * 11 + n2).integers(0, q, n, dtype=np.uint64)
    Am = A.reshape(n2, n1).T                        # Am[k1][k2] = A[k1 + N1 k2]
    W3i = np.array([[pow(pinv, 2 * n1 * i * j, q) for j in range(n2)] for i in range(n2)], dtype=object)
    Bm = _matmul_mod(Am, W3i, q)                    # [k1][n2]
    T = np.array([[pow(pinv, (2 * k1 + 1) * j, q) * ninv % q for j in range(n2)] for k1 in range(n1)],
                 dtype=object)
    Cm = np.array((Bm.astype(object) * T) % q, dtype=np.uint64)
    W1i = np.array([[pow(pinv, n2 * (2 * k1 + 1) * i, q) for k1 in range(n1)] for i in range(n1)], dtype=object)
    Dm = _matmul_mod(W1i, Cm, q)                    # [n1][n2]
    out = Dm.reshape(-1)                            # a[N2 n1 + n2]
    assert (out.astype(np.uint32) == O.intt_brute(A.astype(np.uint32), q, psi)).all()


@pytest.mark.parametrize("n,c", [(64, 2), (64, 4), (128, 8), (256, 4)])
def test_two_pass_dif_inverse_identity(n, c):
    """The plain path's two-pass inverse splits the inputs by residue class of k mod C (each
    local pass takes the class r, k = C k' + r, at stride C), then the cross pass combines
    the C partial results: with N = NC C and n = n' + NC s,
    a[n] = N^-1 sum_r psi^(-(2r+1) n) G_r[n'],   G_r[n'] = sum_k' A[C k' + r] psi^(-2 C k' n'),
    G_r being a length-NC transform of the class (psi^(2C) is an NC-th root of unity)."""
    q = Q30[3]
    psi = P.psi(q, n)
    pinv = pow(psi, -1, q)
    nc = n // c
    assert pow(psi, 2 * c * nc, q) == 1 and pow(psi, 2 * c * (nc // 2), q) == q - 1
    A = np.random.default_rng(3 * n + c).integers(0, q, n, dtype=np.uint64).astype(np.uint32)
    G = [[sum(int(A[c * kk + r]) * pow(pinv, 2 * c * kk * m, q) for kk in range(nc)) % q
          for m in range(nc)] for r in range(c)]
    ninv = pow(n, -1, q)
    out = np.zeros(n, dtype=np.uint64)
    for nn in range(n):
        acc = sum(pow(pinv, (2 * r + 1) * nn, q) * G[r][nn % nc] for r in range(c))
        out[nn] = acc * ninv % q
    assert (out.astype(np.uint32) == O.intt_brute(A, q, psi)).all()

"""Full-RNS CKKS oracle: basis conversion, key switching, HMULT, rescale
(test infrastructure only; see oracle/__init__.py).

Everything here follows Sec. II-B and Sec. IV-A of TensorFHE (arXiv
2212.14191). The paper's Algorithms 1-6 are not legible in the available text,
so the key-switching steps follow the hybrid ("generalized") key switching of
Han and Ki that Sec. II-B and Sec. IV-A name, in this reading:

* ciphertexts ct = (c0, c1) decrypt as c0 + c1*s (the paper writes the pair as
  (b*s + m + e, b); this is the same scheme with the sign of the random part
  absorbed), and are stored limb-major, every limb in the NTT domain of Eq. (4);
* Q = q_0 ... q_l is split into slices Q_j of alpha consecutive primes
  (Sec. II-B, GKS; the last slice may be short), P = p_0 ... p_{K-1} > max Q_j;
* Conv is the approximate fast basis conversion (Sec. IV-A, "Conv"):
      Conv_{B->C}(x)_t = ( sum_i [x_i * (B/b_i)^-1]_{b_i} * [B/b_i]_t ) mod t
  which returns x + u*B for an integer 0 <= u < |B| (no correction term);
* KeySwitch(d2) = ModDown( sum_j ModUp_j(d2) (.) evk_j ), with ModUp_j the
  Conv from Q_j to the other limbs of Q_l and to P, and ModDown the
  floor-type Conv from P back to Q_l followed by the multiplication by P^-1;
* HMULT (Sec. II-B) = (d0 + ks0, d1 + ks1) with (d0, d1, d2) the tensor product
  and (ks0, ks1) = KeySwitch(d2);
* RESCALE (Sec. II-B) divides by the last prime q_l with rounding to nearest:
  the last limb is centred to (-q_l/2, q_l/2] before it is subtracted;
* HROTATE / conjugation (Sec. II-B's operation table, FrobeniusMap) applies the
  automorphism X -> X^k to both components and key-switches c1(X^k) from
  s(X^k) back to s; CMULT and HADD are limbwise Hada-Mult and Ele-Add;
* hoisted HROTATE (several rotations of one ciphertext) forms ModUp(c1) once and
  applies each automorphism to the extended digits (hrotate_hoisted says how
  that differs from hrotate).

Arrays are numpy uint64 holding canonical residues; products of two residues
below 2^30 fit in 64 bits, and every step reduces with '%'. The NTTs run in the
C oracle (oracle/ntt_oracle.c).
"""
import math

import numpy as np

from . import ntt as _ntt
from . import params as _params

U64 = np.uint64


# --------------------------------------------------------------------------
# parameters


class Params:
    """Ring degree N, ciphertext primes q_0.., special primes p_0.., slice width alpha."""

    def __init__(self, N, qs, ps, alpha):
        self.N = int(N)
        self.qs = [int(x) for x in qs]
        self.ps = [int(x) for x in ps]
        self.alpha = int(alpha)
        self.psi_q = [_params.psi(q, self.N) for q in self.qs]
        self.psi_p = [_params.psi(p, self.N) for p in self.ps]
        self.P = math.prod(self.ps)

    @property
    def K(self):
        return len(self.ps)

    def dnum(self, nl):
        """Number of slices used at nl ciphertext limbs (the last may be short)."""
        return -(-nl // self.alpha)

    def slice_limbs(self, j, nl):
        return list(range(j * self.alpha, min((j + 1) * self.alpha, nl)))


# --------------------------------------------------------------------------
# elementwise kernels of Sec. IV-A (Hada-Mult, Ele-Add, Ele-Sub), per limb


def _mods_col(mods):
    return np.asarray(mods, dtype=U64)[:, None]


def hada(a, b, mods):
    return (a.astype(U64) * b.astype(U64)) % _mods_col(mods)


def add(a, b, mods):
    return (a.astype(U64) + b.astype(U64)) % _mods_col(mods)


def sub(a, b, mods):
    m = _mods_col(mods)
    return (a.astype(U64) + m - b.astype(U64)) % m


def ntt(x, mods, psis):
    out, _ = _ntt.ntt_batch(np.asarray(x, dtype=np.uint32), mods, psis, inverse=False)
    return out.astype(U64)


def intt(x, mods, psis):
    out, _ = _ntt.ntt_batch(np.asarray(x, dtype=np.uint32), mods, psis, inverse=True)
    return out.astype(U64)


def to_residues(coeffs, mods):
    """Signed integer coefficients (python ints or int64) -> (len(mods), N) residues."""
    c = np.asarray(coeffs, dtype=object)
    return np.stack([np.array([int(v) % m for v in c], dtype=U64) for m in mods])


def small_to_residues(coeffs, mods):
    """Same as to_residues for |coeff| < 2^62 given as int64 (vectorised)."""
    c = np.asarray(coeffs, dtype=np.int64)
    return np.stack([np.mod(c, np.int64(m)).astype(U64) for m in mods])


# --------------------------------------------------------------------------
# Conv: approximate fast basis conversion (Sec. IV-A)


def conv(x, src, dst):
    """Conv_{B->C}: x is (|B|, N) coefficient residues mod src; returns (|C|, N) mod dst."""
    B = math.prod(src)
    y = []
    for i, b in enumerate(src):
        bhat_inv = pow((B // b) % b, -1, b)
        y.append((x[i].astype(U64) * U64(bhat_inv)) % U64(b))
    out = np.zeros((len(dst), x.shape[1]), dtype=U64)
    for t_i, t in enumerate(dst):
        acc = np.zeros(x.shape[1], dtype=U64)
        for i, b in enumerate(src):
            acc = (acc + (y[i] * U64((B // b) % t)) % U64(t)) % U64(t)
        out[t_i] = acc
    return out


# --------------------------------------------------------------------------
# key generation and encryption (host test harness; random draws are inputs)


def keygen_ksk(prm, s_coeff, target_ntt, a_rand, e_rand):
    """Key-switching key from `target` to s (Han-Ki hybrid form), one pair per slice.

    s_coeff    : (N,) small signed ints (the secret key).
    target_ntt : (L+K, N) NTT-domain residues of the key being switched away from, over
                 q_0..q_{L-1}, p_0..p_{K-1} (s^2 for relinearisation, s(X^k) for a
                 rotation or conjugation).
    a_rand     : (dnum, L+K, N) uniform residues, limb t uniform in [0, mod_t); used
                 directly as NTT-domain values (a uniform polynomial is uniform in
                 either domain).
    e_rand     : (dnum, N) small signed ints (coefficient domain).
    Returns (dnum, 2, L+K, N) uint64, NTT domain, limbs q_0..q_{L-1}, p_0..p_{K-1}.

    Slice j encrypts P * (Q/Q_j) * [(Q/Q_j)^-1]_{Q_j} * target, whose residue is
    [P]_{q_i} * target for q_i in slice j and 0 for every other limb.
    """
    mods = prm.qs + prm.ps
    psis = prm.psi_q + prm.psi_p
    L = len(prm.qs)
    dnum = prm.dnum(L)
    s = ntt(small_to_residues(s_coeff, mods), mods, psis)
    ksk = np.zeros((dnum, 2, len(mods), prm.N), dtype=U64)
    for j in range(dnum):
        a = np.asarray(a_rand[j], dtype=U64) % _mods_col(mods)
        e = ntt(small_to_residues(e_rand[j], mods), mods, psis)
        b = add(sub(np.zeros_like(a), hada(a, s, mods), mods), e, mods)
        for i in prm.slice_limbs(j, L):
            q = prm.qs[i]
            b[i] = (b[i] + (target_ntt[i] * U64(prm.P % q)) % U64(q)) % U64(q)
        ksk[j, 0] = b
        ksk[j, 1] = a
    return ksk


def keygen_evk(prm, s_coeff, a_rand, e_rand):
    """Relinearisation key: keygen_ksk for the target s^2."""
    mods = prm.qs + prm.ps
    s = ntt(small_to_residues(s_coeff, mods), mods, prm.psi_q + prm.psi_p)
    return keygen_ksk(prm, s_coeff, hada(s, s, mods), a_rand, e_rand)


def keygen_rot(prm, s_coeff, k, a_rand, e_rand):
    """Rotation / conjugation key for the Galois element k: keygen_ksk for s(X^k)."""
    mods = prm.qs + prm.ps
    sk = automorph_coeff(small_to_residues(s_coeff, mods), mods, k)
    return keygen_ksk(prm, s_coeff, ntt(sk, mods, prm.psi_q + prm.psi_p), a_rand, e_rand)


def encrypt(prm, nl, m_coeff, s_coeff, a_rand, e_coeff):
    """Symmetric encryption at nl limbs: c1 = a, c0 = -a*s + m + e (NTT domain)."""
    mods, psis = prm.qs[:nl], prm.psi_q[:nl]
    s = ntt(small_to_residues(s_coeff, mods), mods, psis)
    m = ntt(small_to_residues(m_coeff, mods), mods, psis)
    e = ntt(small_to_residues(e_coeff, mods), mods, psis)
    a = np.asarray(a_rand, dtype=U64)[:nl] % _mods_col(mods)
    c0 = add(add(sub(np.zeros_like(a), hada(a, s, mods), mods), m, mods), e, mods)
    return np.stack([c0, a])


def decrypt_coeffs(prm, ct, s_coeff, n_crt=2):
    """c0 + c1*s, back to centred integer coefficients via CRT over the first n_crt limbs."""
    nl = ct.shape[1]
    mods, psis = prm.qs[:nl], prm.psi_q[:nl]
    s = ntt(small_to_residues(s_coeff, mods), mods, psis)
    m = intt(add(ct[0], hada(ct[1], s, mods), mods), mods, psis)
    return crt_centered(m[:n_crt], mods[:n_crt])


def crt_centered(res, mods):
    """(k, N) residues -> python ints in (-M/2, M/2], M = prod(mods)."""
    M = math.prod(mods)
    out = []
    for n in range(res.shape[1]):
        x = 0
        for i, m in enumerate(mods):
            Mi = M // m
            x += int(res[i, n]) * Mi * pow(Mi % m, -1, m)
        x %= M
        if x > M // 2:
            x -= M
        out.append(x)
    return out


# --------------------------------------------------------------------------
# HMULT pieces (Sec. II-B operations, Sec. IV-A kernel composition)


def tensor(ct_a, ct_b, mods):
    """(d0, d1, d2) = (c0 c0', c0 c1' + c1 c0', c1 c1'), NTT domain."""
    d0 = hada(ct_a[0], ct_b[0], mods)
    d1 = add(hada(ct_a[0], ct_b[1], mods), hada(ct_a[1], ct_b[0], mods), mods)
    d2 = hada(ct_a[1], ct_b[1], mods)
    return d0, d1, d2


def modup(prm, nl, d2_ntt, d2_coeff, j):
    """ModUp of slice j: (nl + K, N) NTT-domain residues over q_0..q_{nl-1}, p_0..

    The limbs of slice j keep d2's own NTT-domain values; every other limb gets
    the NTT of Conv_{Q_j -> t} of slice j's coefficient residues.
    """
    own = prm.slice_limbs(j, nl)
    src = [prm.qs[i] for i in own]
    others = [i for i in range(nl) if i not in own]
    dst_mods = [prm.qs[i] for i in others] + prm.ps
    dst_psis = [prm.psi_q[i] for i in others] + prm.psi_p
    conv_c = conv(d2_coeff[own], src, dst_mods)
    conv_n = ntt(conv_c, dst_mods, dst_psis)
    out = np.zeros((nl + prm.K, prm.N), dtype=U64)
    out[own] = d2_ntt[own]
    for k, i in enumerate(others):
        out[i] = conv_n[k]
    out[nl:] = conv_n[len(others):]
    return out


def evk_at_level(prm, evk, j, nl):
    """Key j restricted to limbs q_0..q_{nl-1}, p_0..p_{K-1}: (2, nl + K, N)."""
    L = len(prm.qs)
    idx = list(range(nl)) + list(range(L, L + prm.K))
    return evk[j][:, idx]


def inner_product(prm, nl, d2_ntt, evk):
    """(ks0, ks1) over nl + K limbs before ModDown: sum_j ModUp_j(d2) (.) evk_j."""
    mods = prm.qs[:nl] + prm.ps
    d2_coeff = intt(d2_ntt, prm.qs[:nl], prm.psi_q[:nl])
    ks0 = np.zeros((nl + prm.K, prm.N), dtype=U64)
    ks1 = np.zeros_like(ks0)
    for j in range(prm.dnum(nl)):
        dt = modup(prm, nl, d2_ntt, d2_coeff, j)
        ek = evk_at_level(prm, evk, j, nl)
        ks0 = add(ks0, hada(dt, ek[0], mods), mods)
        ks1 = add(ks1, hada(dt, ek[1], mods), mods)
    return ks0, ks1


def moddown(prm, nl, ks):
    """(ks|_Q - NTT(Conv_{P->Q}(INTT(ks|_P)))) * P^-1 mod q_i, for i < nl."""
    qm, qpsi = prm.qs[:nl], prm.psi_q[:nl]
    y_coeff = intt(ks[nl:], prm.ps, prm.psi_p)
    y = ntt(conv(y_coeff, prm.ps, qm), qm, qpsi)
    pinv = np.array([pow(prm.P % q, -1, q) for q in qm], dtype=U64)[:, None]
    return (sub(ks[:nl], y, qm) * pinv) % _mods_col(qm)


def keyswitch(prm, nl, d2_ntt, evk):
    ks0, ks1 = inner_product(prm, nl, d2_ntt, evk)
    return moddown(prm, nl, ks0), moddown(prm, nl, ks1)


def hmult_relin(prm, nl, ct_a, ct_b, evk):
    """HMULT of Sec. II-B without rescale: (d0 + ks0, d1 + ks1), nl limbs."""
    mods = prm.qs[:nl]
    d0, d1, d2 = tensor(ct_a, ct_b, mods)
    k0, k1 = keyswitch(prm, nl, d2, evk)
    return np.stack([add(d0, k0, mods), add(d1, k1, mods)])


def rescale(prm, ct):
    """RESCALE of Sec. II-B, rounding to nearest: nl limbs -> nl - 1 limbs."""
    nl = ct.shape[1]
    ql = prm.qs[nl - 1]
    mods, psis = prm.qs[:nl - 1], prm.psi_q[:nl - 1]
    out = np.zeros((2, nl - 1, prm.N), dtype=U64)
    for c in range(2):
        x = intt(ct[c][nl - 1:nl], [ql], [prm.psi_q[nl - 1]])[0].astype(np.int64)
        x = np.where(x > (ql - 1) // 2, x - ql, x)
        xr = ntt(small_to_residues(x, mods), mods, psis)
        qinv = np.array([pow(ql, -1, q) for q in mods], dtype=U64)[:, None]
        out[c] = (sub(ct[c][:nl - 1], xr, mods) * qinv) % _mods_col(mods)
    return out


def hmult(prm, nl, ct_a, ct_b, evk):
    """HMULT followed by RESCALE: (2, nl, N) x2 -> (2, nl - 1, N)."""
    return rescale(prm, hmult_relin(prm, nl, ct_a, ct_b, evk))


# --------------------------------------------------------------------------
# FrobeniusMap / HROTATE, CMULT, HADD (the other operations of Sec. II-B's table)


def galois_rotation(r, N):
    """Galois element 5^r mod 2N of a rotation of the N/2 slots by r (left for r > 0)."""
    return pow(5, r % (N // 2), 2 * N)


def galois_conjugation(N):
    """Galois element 2N - 1 (X -> X^-1): complex conjugation of every slot."""
    return 2 * N - 1


def automorph_coeff(a, mods, k):
    """a(X) -> a(X^k) in Z_q[X]/(X^N + 1), k odd: coefficient n moves to n k mod 2N and is
    negated when that index lies in [N, 2N) (X^N = -1). a is (len(mods), N) residues."""
    a = np.asarray(a, dtype=U64)
    N = a.shape[1]
    assert k % 2 == 1 and 0 < k < 2 * N
    out = np.zeros_like(a)
    m = _mods_col(mods)
    for n in range(N):
        t = (n * k) % (2 * N)
        if t < N:
            out[:, t] = a[:, n]
        else:
            out[:, t - N] = (m[:, 0] - a[:, n]) % m[:, 0]
    return out


def automorph(x_ntt, mods, psis, k):
    """The same map on NTT-domain limbs, by its definition: INTT, automorph_coeff, NTT."""
    return ntt(automorph_coeff(intt(x_ntt, mods, psis), mods, k), mods, psis)


def hrotate(prm, nl, ct, ksk, k):
    """HROTATE (FrobeniusMap + key switching): (c0(X^k) + ks0, ks1) with
    (ks0, ks1) = KeySwitch(c1(X^k)) under the key from s(X^k) to s; nl limbs, NTT domain."""
    mods, psis = prm.qs[:nl], prm.psi_q[:nl]
    c0 = automorph(ct[0], mods, psis, k)
    c1 = automorph(ct[1], mods, psis, k)
    k0, k1 = keyswitch(prm, nl, c1, ksk)
    return np.stack([add(c0, k0, mods), k1 % _mods_col(mods)])


def hrotate_hoisted(prm, nl, ct, ksks, ks):
    """Several HROTATEs of one ciphertext sharing one ModUp (hoisted rotations): the digits
    ModUp_j(c1) over q_0..q_{nl-1}, p_0.. are formed once in the NTT domain; for each Galois
    element k they go through the automorphism, are multiplied by that rotation's key and
    summed, and ModDown plus c0(X^k) finish as in hrotate. Returns (len(ks), 2, nl, N).

    The automorphism commutes with the NTT and with products, but not exactly with the
    approximate Conv: where X -> X^k negates a coefficient, the permuted digit holds the
    negated lift -(sum_i y_i [B_j/b_i]) and ModUp of the permuted c1 the lift
    sum_i [-y_i]_{b_i} [B_j/b_i]; they differ by B_j times the number of nonzero y_i. Both
    are lifts of the same residues mod Q_j, so both key switches are valid, but they are
    different results: this is a parity definition of its own, not hrotate's."""
    mods, psis = prm.qs[:nl], prm.psi_q[:nl]
    emods = prm.qs[:nl] + prm.ps
    epsis = prm.psi_q[:nl] + prm.psi_p
    c1_coeff = intt(ct[1], mods, psis)
    digits = [modup(prm, nl, ct[1], c1_coeff, j) for j in range(prm.dnum(nl))]
    outs = []
    for ksk, k in zip(ksks, ks):
        ks0 = np.zeros((nl + prm.K, prm.N), dtype=U64)
        ks1 = np.zeros_like(ks0)
        for j, dt in enumerate(digits):
            dk = automorph(dt, emods, epsis, k)
            ek = evk_at_level(prm, ksk, j, nl)
            ks0 = add(ks0, hada(dk, ek[0], emods), emods)
            ks1 = add(ks1, hada(dk, ek[1], emods), emods)
        c0 = automorph(ct[0], mods, psis, k)
        outs.append(np.stack([add(c0, moddown(prm, nl, ks0), mods), moddown(prm, nl, ks1) % _mods_col(mods)]))
    return np.stack(outs)


def cmult(prm, nl, ct, pt_ntt):
    """CMULT: both components times a plaintext, limbwise in the NTT domain (no rescale)."""
    mods = prm.qs[:nl]
    return np.stack([hada(ct[0], pt_ntt, mods), hada(ct[1], pt_ntt, mods)])


def hadd(prm, nl, ct_a, ct_b):
    """HADD: componentwise sum mod q_i."""
    mods = prm.qs[:nl]
    return np.stack([add(ct_a[0], ct_b[0], mods), add(ct_a[1], ct_b[1], mods)])


# --------------------------------------------------------------------------
# CKKS encoding through the canonical embedding (Sec. II-B, host FP64)


def slot_index(N):
    """Position k of root zeta^(2k+1) holding slot j (zeta^(5^j)), j < N/2."""
    two_n = 2 * N
    g = 1
    idx = []
    for _ in range(N // 2):
        idx.append((g - 1) // 2)
        g = (g * 5) % two_n
    return np.array(idx, dtype=np.int64)


def conj_index(N):
    """Position k' with 2k'+1 = -(5^j) mod 2N."""
    two_n = 2 * N
    g = 1
    idx = []
    for _ in range(N // 2):
        idx.append(((two_n - g) - 1) // 2)
        g = (g * 5) % two_n
    return np.array(idx, dtype=np.int64)


def embed(m_real):
    """Evaluate a real polynomial of R[X]/(X^N+1) at zeta^(2k+1), k < N; zeta = e^(i pi/N)."""
    m = np.asarray(m_real, dtype=np.float64)
    N = m.shape[0]
    tw = np.exp(1j * np.pi * np.arange(N) / N)
    return N * np.fft.ifft(m * tw)


def decode(m_real, scale):
    """Slots z_j = m(zeta^(5^j)) / scale."""
    N = len(m_real)
    return embed(m_real)[slot_index(N)] / scale


def encode(z, N, scale):
    """Integer coefficients round(scale * sigma^-1(z)) for z in C^(N/2)."""
    z = np.asarray(z, dtype=np.complex128)
    ev = np.zeros(N, dtype=np.complex128)
    ev[slot_index(N)] = z
    ev[conj_index(N)] = np.conj(z)
    tw = np.exp(-1j * np.pi * np.arange(N) / N)
    m = np.fft.fft(ev) / N * tw
    return [int(v) for v in np.rint(scale * m.real)]

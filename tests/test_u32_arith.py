"""Host-side checks of the arithmetic the plain 32-bit NTT kernels rely on (Sec. II-A, Eq. (4);
the comparison path of Sec. IV-B): Harvey's lazy butterflies with Shoup's precomputed-quotient
products, in 32-bit words. A complete textbook negacyclic transform is run with those
butterflies at the largest prime the library accepts (q < 2^30, so 4q < 2^32): the forward
Cooley-Tukey butterflies keep every value in [0, 4q), the inverse Gentleman-Sande ones in
[0, 2q), no word wraps, and after the final conditional subtractions the result equals the
oracle's transform. Also the 64-bit reduction of the CKKS kernels (Conv, inner product,
Hada-Mult) and the accumulation bound it relies on. These run on the CPU and use no GPU code."""
import numpy as np
import pytest

from oracle import ntt as O
from oracle import params as P

U64 = np.uint64
M32 = U64(0xFFFFFFFF)


def shoup_quotient(w, q):
    return (w.astype(object) * (1 << 32) // q).astype(U64) if isinstance(w, np.ndarray) else U64((w << 32) // q)


def mul_shoup_lazy(x, w, wq, q):
    """x w mod q in [0, 2q) for any 32-bit x: x w - floor(x wq / 2^32) q, taken mod 2^32."""
    qt = (x * wq) >> U64(32)
    return (x * w - qt * U64(q)) & M32


def csub(x, m):
    """[0, 2m) -> [0, m) as the kernels do it: min(x, x - m) on unsigned 32-bit words."""
    return np.minimum(x, (x - U64(m)) & M32)


def bitrev(k, bits):
    return int(format(k, "0%db" % bits)[::-1], 2)


def forward_lazy(a, q, psi):
    n = a.size
    bits = n.bit_length() - 1
    psi_rev = np.array([pow(psi, bitrev(k, bits), q) for k in range(n)], dtype=U64)
    psi_rev_q = shoup_quotient(psi_rev, q)
    a = a.astype(U64).copy()
    m, t = 1, n
    while m < n:
        t //= 2
        v = a.reshape(m, 2, t)
        w, wq = psi_rev[m:2 * m, None], psi_rev_q[m:2 * m, None]
        # the kernels' first stage takes canonical inputs and skips this reduction
        x2 = v[:, 0, :].copy() if m == 1 else csub(v[:, 0, :], 2 * q)
        tt = mul_shoup_lazy(v[:, 1, :], w, wq, q)
        assert x2.max() < 2 * q and tt.max() < 2 * q
        x, y = x2 + tt, x2 - tt + U64(2 * q)
        assert x.max() < 4 * q and y.max() < 4 * q and y.min() > 0
        v[:, 0, :], v[:, 1, :] = x, y
        m *= 2
    out = csub(csub(a, 2 * q), q)                   # [0, 4q) -> [0, q)
    return out[[bitrev(k, bits) for k in range(n)]]  # bit-reversed -> natural order


def inverse_lazy(A, q, psi):
    n = A.size
    bits = n.bit_length() - 1
    pinv = pow(psi, -1, q)
    pinv_rev = np.array([pow(pinv, bitrev(k, bits), q) for k in range(n)], dtype=U64)
    pinv_rev_q = shoup_quotient(pinv_rev, q)
    a = A.astype(U64)[[bitrev(k, bits) for k in range(n)]].copy()   # natural -> bit-reversed
    m, t = n, 1
    while m > 1:
        h = m // 2
        v = a.reshape(h, 2, t)
        w, wq = pinv_rev[h:2 * h, None], pinv_rev_q[h:2 * h, None]
        x, y = v[:, 0, :], v[:, 1, :]
        s = x + y if m == n else csub(x + y, 2 * q)   # first stage: canonical inputs, x + y < 2q
        d = x - y + U64(2 * q)
        assert s.max() < 2 * q and d.max() < 4 * q and d.min() > 0
        v[:, 0, :], v[:, 1, :] = s, mul_shoup_lazy(d, w, wq, q)
        assert v[:, 1, :].max() < 2 * q
        t *= 2
        m = h
    ninv = pow(n, -1, q)
    return csub(mul_shoup_lazy(a, U64(ninv), shoup_quotient(ninv, q), q), q)


@pytest.mark.parametrize("logn", [4, 10, 12])
def test_lazy_butterflies_at_the_largest_prime(logn):
    n = 1 << logn
    q = P.ntt_primes(1, logn_max=16)[0]
    assert q < (1 << 30) and 4 * q < (1 << 32)
    psi = P.psi(q, n)
    rng = np.random.default_rng(logn)
    for a in (rng.integers(0, q, n, dtype=np.int64).astype(U64),
              np.full(n, q - 1, dtype=U64),                      # every input at its maximum
              np.zeros(n, dtype=U64)):
        A = forward_lazy(a, q, psi)
        np.testing.assert_array_equal(A, O.ntt(a.astype(np.uint32), q, psi).astype(U64))
        np.testing.assert_array_equal(inverse_lazy(A, q, psi), a)


def test_shoup_product_bound_on_extreme_words():
    """x w - floor(x wq / 2^32) q lies in [0, 2q) for every 32-bit x (the quotient estimate is
    short by at most one), which is what lets the butterflies feed it values up to 4q."""
    q = P.ntt_primes(1, logn_max=16)[0]
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.integers(0, 1 << 32, 100000, dtype=np.int64).astype(U64),
                        np.array([0, 1, q - 1, q, 2 * q - 1, 4 * q - 1, (1 << 32) - 1], dtype=U64)])
    for w in (0, 1, 2, q // 2, q - 2, q - 1, int(rng.integers(0, q))):
        r = mul_shoup_lazy(x, U64(w), shoup_quotient(w, q), q)
        assert r.max() < 2 * q
        np.testing.assert_array_equal(r % U64(q), (x.astype(object) * w % q).astype(U64))


def reduce_red(x, q):
    """x mod q for a 64-bit x as the CKKS kernels do it: the high word times [2^32]_q by
    Shoup's method and the low word by one 32-bit Barrett step with floor(2^32 / q), each in
    [0, 2q), summed below 4q and corrected twice."""
    r32 = (1 << 32) % q
    hi, lo = x >> U64(32), x & M32
    t = mul_shoup_lazy(hi, U64(r32), shoup_quotient(r32, q), q)
    u = (lo - (((lo * U64((1 << 32) // q)) >> U64(32)) * U64(q))) & M32
    assert t.max() < 2 * q and u.max() < 2 * q
    return csub(csub(t + u, 2 * q), q)


def test_64bit_reduction_and_accumulation_bounds():
    """Conv and the inner product add up to 15 products of residues below 2^30 in 64 bits
    before one reduction (the inner product reduces after every 15 slices and continues from
    a value below q): 15 (q - 1)^2 + q < 2^64, and reduce_red is exact on every 64-bit word,
    including those extremes."""
    rng = np.random.default_rng(9)
    for q in (P.ntt_primes(1, logn_max=16)[0], P.ntt_primes(40, logn_max=16)[-1]):
        assert 15 * (q - 1) ** 2 + q < (1 << 64)
        x = np.concatenate([
            rng.integers(0, 1 << 63, 200000, dtype=np.int64).astype(U64) * U64(2) + U64(1),
            np.array([0, 1, q - 1, q, (1 << 32) - 1, 1 << 32, (1 << 64) - 1,
                      15 * (q - 1) ** 2, 15 * (q - 1) ** 2 + q - 1], dtype=U64)])
        got = reduce_red(x, q)
        np.testing.assert_array_equal(got, np.array([int(v) % q for v in x], dtype=U64))


def _bitrev_small(x, bits):
    return int(format(x, "0%db" % bits)[::-1], 2) if bits else 0


@pytest.mark.parametrize("log_c", [1, 2, 3])
def test_two_pass_forward_cross_pass_ranges(log_c):
    """The forward two-pass cross pass at the largest accepted prime with every input of the C
    streams anywhere in [0, 4q) (the local pass stores its Cooley-Tukey outputs unreduced): stream
    0 gets one conditional subtraction of 2q, the twists of the other streams are lazy Shoup
    products in [0, 2q), the C-point cyclic DFT's butterflies (trivial ones at omega^0,
    Gentleman-Sande ones otherwise) keep [0, 2q), and after one final conditional subtraction
    output t equals sum_j omega^(t j) twist_j y_j mod q, canonical."""
    C = 1 << log_c
    q = P.ntt_primes(1, logn_max=16)[0]
    rng = np.random.default_rng(40 + log_c)
    omega = pow(P.psi(q, 1 << 16), (1 << 16) * 2 // C, q)          # a primitive C-th root of unity
    om = [pow(omega, m, q) for m in range(C // 2)]
    om_q = [shoup_quotient(w, q) for w in om]
    for trial in range(4):
        y0 = rng.integers(0, 4 * q, (C, 256), dtype=np.int64).astype(U64)
        if trial == 1:
            y0[:] = 4 * q - 1
        if trial == 2:
            y0[:] = 0
        tw = rng.integers(1, q, C, dtype=np.int64)
        y = y0.copy()
        y[0] = csub(y[0], 2 * q)
        for j in range(1, C):
            y[j] = mul_shoup_lazy(y[j], U64(tw[j]), shoup_quotient(int(tw[j]), q), q)
        assert y.max() < 2 * q
        for s in range(log_c):
            h = C >> (s + 1)
            for b in range(0, C, 2 * h):
                for jj in range(h):
                    m = jj << s
                    x, z = y[b + jj].copy(), y[b + jj + h].copy()
                    if m == 0:
                        y[b + jj] = csub((x + z) & M32, 2 * q)
                        y[b + jj + h] = csub((x - z + U64(2 * q)) & M32, 2 * q)
                    else:
                        y[b + jj] = csub(x + z, 2 * q)
                        y[b + jj + h] = mul_shoup_lazy((x - z + U64(2 * q)) & M32, U64(om[m]), om_q[m], q)
            assert y.max() < 2 * q
        out = csub(y, q)
        tw_all = [1] + [int(t) for t in tw[1:]]
        for t in range(C):
            want = sum(pow(omega, t * j, q) * tw_all[j] * y0[j].astype(object) for j in range(C)) % q
            got = out[_bitrev_small(t, log_c)]
            assert (got.astype(object) == want).all(), (t, trial)


def test_two_pass_inverse_last_stage_with_scaling():
    """The inverse two-pass cross pass's last Gentleman-Sande stage with N^-1 folded in, at the
    largest accepted prime and inputs anywhere in [0, 2q): (u + w) N^-1 and (u - w + 2q) (tw N^-1)
    as single Shoup products are canonical and equal to the stage followed by the scaling."""
    q = P.ntt_primes(1, logn_max=16)[0]
    n = 1 << 16
    rng = np.random.default_rng(7)
    ninv = pow(n, -1, q)
    tw = int(rng.integers(1, q))
    niw = ninv * tw % q
    u = rng.integers(0, 2 * q, 4096, dtype=np.int64).astype(U64)
    w = rng.integers(0, 2 * q, 4096, dtype=np.int64).astype(U64)
    u[:2], w[:2] = [2 * q - 1, 0], [0, 2 * q - 1]
    folded_x = csub(mul_shoup_lazy(u + w, U64(ninv), shoup_quotient(ninv, q), q), q)
    folded_y = csub(mul_shoup_lazy(u - w + U64(2 * q), U64(niw), shoup_quotient(niw, q), q), q)
    s = csub(u + w, 2 * q)
    d = mul_shoup_lazy(u - w + U64(2 * q), U64(tw), shoup_quotient(tw, q), q)
    sep_x = csub(mul_shoup_lazy(s, U64(ninv), shoup_quotient(ninv, q), q), q)
    sep_y = csub(mul_shoup_lazy(d, U64(ninv), shoup_quotient(ninv, q), q), q)
    assert folded_x.max() < q and folded_y.max() < q
    np.testing.assert_array_equal(folded_x, sep_x)
    np.testing.assert_array_equal(folded_y, sep_y)
    uo, wo = u.astype(object), w.astype(object)
    assert (folded_x.astype(object) == (uo + wo) * ninv % q).all()
    assert (folded_y.astype(object) == (uo - wo) * tw * ninv % q).all()


@pytest.mark.parametrize("ql_side", ["above", "below"])
def test_fused_tail_load_without_reductions(ql_side):
    """The fused RESCALE tail's load side (Sec. II-B: z_i = y_i + [last]_i q_l^-1 with the last
    limb centred) as the local pass computes it: x = last, plus q - (q_l mod q) where last stands
    for last - q_l, goes into a lazy Shoup product unreduced (x < 2^31), z = y + that product
    lies in [0, 3q), and only the first half of the sub-transform (the x side of the first
    butterfly stage) gets one conditional subtraction to [0, 2q). Checked with q_l above and
    below q (the largest accepted prime as one of them) against exact integers, then as the input of a whole lazy forward transform
    (its first stage asserts x < 2q), whose output must equal the oracle's transform of z."""
    primes = sorted(P.ntt_primes(3, logn_max=16))        # primes[2] is the largest accepted
    q, ql = (primes[1], primes[2]) if ql_side == "above" else (primes[2], primes[0])
    assert (ql > q) == (ql_side == "above")
    n = 1 << 10
    rng = np.random.default_rng(11 if ql_side == "above" else 12)
    last = rng.integers(0, ql, n, dtype=np.int64).astype(U64)
    last[:4] = [0, (ql - 1) // 2, (ql - 1) // 2 + 1, ql - 1]       # both sides of the centring
    y = rng.integers(0, q, n, dtype=np.int64).astype(U64)
    y[4:6] = q - 1
    qlinv = pow(ql, -1, q)
    half, lift = (ql - 1) // 2, q - ql % q
    x = np.where(last > U64(half), last + U64(lift), last)
    assert x.max() < (1 << 31)
    z = y + mul_shoup_lazy(x, U64(qlinv), shoup_quotient(qlinv, q), q)
    assert z.max() < 3 * q
    v = z.copy()
    v[:n // 2] = csub(v[:n // 2], q)
    assert v[:n // 2].max() < 2 * q
    centred = [int(l) - ql if int(l) > half else int(l) for l in last]
    want = np.array([(int(yy) + c * qlinv) % q for yy, c in zip(y, centred)], dtype=U64)
    np.testing.assert_array_equal(v % U64(q), want)
    psi = P.psi(q, n)
    np.testing.assert_array_equal(forward_lazy(v, q, psi), O.ntt(want.astype(np.uint32), q, psi).astype(U64))


def redc_lazy(t, q, qinv, guarded=False):
    """Montgomery reduction as Conv does it: m = t_lo q^-1 mod 2^32, then t_hi - floor(m q / 2^32)
    (m q has the same low word as t, so the subtraction is exact), congruent to t 2^-32 mod q and
    above -q; q is added always, or (guarded) only where t_hi < floor(m q / 2^32)."""
    m = ((t & M32) * U64(qinv)) & M32
    hi, u = t >> U64(32), (m * U64(q)) >> U64(32)
    if guarded:
        return (hi - u + np.where(hi < u, U64(q), U64(0))) & M32
    return (hi - u + U64(q)) & M32


@pytest.mark.parametrize("ns", [1, 8, 12, 15])
def test_conv_montgomery_reduction(ns):
    """Conv's sum over NS source limbs, out_t = sum_i y_i [B/b_i]_t mod p (Sec. IV-A), with the
    constants taken in Montgomery form ([B/b_i]_t 2^32 mod p, folded in once per CTA) and the
    64-bit sum reduced by one Montgomery step: every y_i < 2^30 and constant < p keep the sum
    below NS 2^30 p, so its high word is below NS p / 4. For NS <= 12 the step adds p always
    and stays below 4p < 2^32; above 12 that could pass 2^32, so p is added only where the
    subtraction went below zero, leaving [0, NS p / 4) below 4p. Two conditional subtractions
    (2p, p) then give the canonical residue. Checked at the largest and a small accepted prime,
    with every source and constant at its maximum among the cases."""
    rng = np.random.default_rng(50 + ns)
    for p in (P.ntt_primes(1, logn_max=16)[0], P.ntt_primes(40, logn_max=16)[-1]):
        qinv = pow(p, -1, 1 << 32)
        srcq = P.ntt_primes(ns + 1, logn_max=16)[1:]
        for trial in range(3):
            y = np.stack([rng.integers(0, q, 4096, dtype=np.int64) for q in srcq]).astype(U64)
            h = rng.integers(0, p, ns, dtype=np.int64)
            if trial == 1:
                y = np.stack([np.full(4096, q - 1, dtype=np.int64) for q in srcq]).astype(U64)
                h[:] = p - 1
            hm = [(int(v) << 32) % p for v in h]                # Montgomery form of the constants
            acc = np.zeros(4096, dtype=U64)
            for i in range(ns):
                acc += y[i] * U64(hm[i])                        # no wrap: < ns 2^30 p < 2^64
            assert int(acc.max()) < ns * (1 << 30) * p
            assert int(acc.max() >> U64(32)) < ns * p / 4
            r = redc_lazy(acc, p, qinv, guarded=ns > 12)
            assert int(r.max()) < 4 * p
            r = csub(csub(r, 2 * p), p)
            want = sum(y[i].astype(object) * int(h[i]) for i in range(ns)) % p
            assert (r.astype(object) == want).all(), (p, trial)


@pytest.mark.parametrize("dnum", [1, 3, 12, 13, 15])
def test_inner_product_montgomery_with_post_factor(dnum):
    """The key-switching inner product's reduction (Sec. IV-A Hada-Mult + Ele-Add): each sum of
    dnum products of residues below q (at most 15 before a mid-way reduction) takes one guarded
    Montgomery step, then a lazy Shoup product by 2^32 s mod q (s = P^-1 q_l^-1 on the limbs the
    fused tail scales, else 1) and one conditional subtraction: the result must be the
    canonical sum times s. Checked at the largest and a small accepted prime, with every
    operand at its maximum among the cases."""
    rng = np.random.default_rng(70 + dnum)
    for q in (P.ntt_primes(1, logn_max=16)[0], P.ntt_primes(40, logn_max=16)[-1]):
        qinv = pow(q, -1, 1 << 32)
        for scale in (1, int(rng.integers(2, q))):
            post = ((1 << 32) * scale) % q
            post_q = shoup_quotient(post, q)
            for trial in range(2):
                x = rng.integers(0, q, (dnum, 4096), dtype=np.int64).astype(U64)
                w = rng.integers(0, q, (dnum, 4096), dtype=np.int64).astype(U64)
                if trial == 1:
                    x[:], w[:] = q - 1, q - 1
                acc = np.zeros(4096, dtype=U64)
                for j in range(dnum):
                    acc += x[j] * w[j]                          # < 15 q^2 < 2^64
                m = redc_lazy(acc, q, qinv, guarded=True)
                r = csub(mul_shoup_lazy(m, U64(post), post_q, q), q)
                want = sum(x[j].astype(object) * w[j].astype(object) for j in range(dnum)) * scale % q
                assert (r.astype(object) == want).all(), (q, scale, trial)

"""Host-side checks of the arithmetic the tensor-core NTT relies on (Sec. IV-B, segment fusion
of Eq. (9)): the balanced 8-bit digits the kernels produce, their exact fp16 encoding, and the
exactness of the digit GEMM under fp32 accumulation at the largest reduction size, the
epilogues' rebuild mod q from signed accumulators; and of the tensor-core form of Conv
(Sec. IV-A), its 32-bit reconstruction included.

These run on the CPU and use no GPU code: they pin the identities the kernel arithmetic is
built on, so that a plausible slip there (a wrong bias, an unbalanced digit, an accumulation
bound that overflows the fp32 significand) fails here before any parity test.
"""
import numpy as np
import pytest

from oracle import params as P


def _digits_from_bias(v):
    """The kernels' split: bytes of v + 0x80808080, each minus 128 (v < 2^30)."""
    y = (v.astype(np.uint64) + 0x80808080) & 0xFFFFFFFF
    return np.stack([((y >> (8 * j)) & 0xFF).astype(np.int64) - 128 for j in range(4)], axis=-1)


def _balanced_base(v, base, ndig):
    """Balanced digits by repeated centred remainder (the textbook definition)."""
    x = v.astype(np.int64).copy()
    out = []
    for _ in range(ndig - 1):
        d = ((x + base // 2) % base) - base // 2
        out.append(d)
        x = (x - d) // base
    out.append(x)
    return np.stack(out, axis=-1)


def test_bias_split_equals_balanced_digits():
    rng = np.random.default_rng(11)
    v = np.concatenate([rng.integers(0, 1 << 30, 200000, dtype=np.int64),
                        np.array([0, 1, 127, 128, 255, 256, (1 << 30) - 1, (1 << 29), 0x7F7F7F,
                                  0x808080, 0x3FFFFFFF], dtype=np.int64)])
    d = _digits_from_bias(v)
    assert d.min() >= -128 and d.max() <= 127
    w = np.array([1, 256, 65536, 1 << 24], dtype=np.int64)
    np.testing.assert_array_equal((d * w).sum(axis=-1), v)
    # the balanced representation is unique, so it equals the centred-remainder digits
    np.testing.assert_array_equal(d, _balanced_base(v, 256, 4))


def test_fp16_magic_encoding_is_exact():
    b = np.arange(256, dtype=np.uint16)
    h = (0x6400 | b).view(np.float16)
    np.testing.assert_array_equal(h.astype(np.float64), 1024.0 + b)
    # the f16x2 subtraction of 1152 (bits 0x6480) is exact for every byte
    k = np.array([0x6480], dtype=np.uint16).view(np.float16)[0]
    assert float(k) == 1152.0
    r = (h - k).astype(np.float64)
    np.testing.assert_array_equal(r, b.astype(np.float64) - 128.0)


def test_constant_digits_base255_bounds():
    rng = np.random.default_rng(12)
    w = rng.integers(0, 1 << 30, 100000, dtype=np.int64)
    e = _balanced_base(w, 255, 4)
    assert np.abs(e[..., :3]).max() <= 127
    assert np.abs(e[..., 3]).max() <= 127  # w < 2^30 < 127 * 255^3 + ...
    np.testing.assert_array_equal((e * np.array([1, 255, 255 ** 2, 255 ** 3])).sum(axis=-1), w)


@pytest.mark.parametrize("K", [32, 256])
def test_digit_gemm_exact_under_fp32(K):
    """One sub-transform GEMM in the kernels' form: y_c = sum_n W[c][n] x_n (mod q) as
    acc_i = sum_{n, j} d_j(x_n) e_i(W[c][n] 256^j mod q) with fp16 digits and fp32
    accumulation, y = sum_i 255^i acc_i. The exact integer sums are computed beside the fp32
    ones and must stay below 2^24, the bound 4 K x 128 x 127 < 2^24 guarantees."""
    q = P.ntt_primes(1)[0]
    rng = np.random.default_rng(K)
    C, M = 64, 48
    W = rng.integers(0, q, (C, K), dtype=np.int64)
    X = rng.integers(0, q, (M, K), dtype=np.int64)
    # a row whose three low digits are all -128 (the largest data-digit magnitude)
    X[0, :] = 63 * (1 << 24) - 0x808080
    assert X[0, 0] < q
    dx = _digits_from_bias(X)                                  # (M, K, 4) data digits
    pw = np.array([pow(256, j, q) for j in range(4)], dtype=np.int64)
    Wj = (W[:, :, None] * pw[None, None, :]) % q               # (C, K, 4): W 256^j mod q
    e = _balanced_base(Wj, 255, 4)                             # (C, K, 4 j, 4 i)
    A = dx.reshape(M, 4 * K).astype(np.float16)                # K' = 4 K, index 4 n + j
    # exact reference in int64: W = 2^15 Wh + Wl keeps every partial sum below 2^53
    Wh, Wl = W >> 15, W & 0x7FFF
    ref = (((X @ Wh.T) % q) * (1 << 15) + X @ Wl.T) % q
    y = np.zeros((M, C), dtype=np.int64)
    for i in range(4):
        B = e[..., i].reshape(C, 4 * K).astype(np.float16)
        assert np.array_equal(B.astype(np.int64), e[..., i].reshape(C, 4 * K))
        acc = A.astype(np.float32) @ B.astype(np.float32).T    # fp32 products and sums
        exact = dx.reshape(M, 4 * K) @ e[..., i].reshape(C, 4 * K).T
        assert np.abs(exact).max() < (1 << 24)
        np.testing.assert_array_equal(acc.astype(np.int64), exact)
        y += (255 ** i) * exact
    np.testing.assert_array_equal(y % q, ref)
    assert 4 * K * 128 * 127 < (1 << 24)


def _shoup(x, w, q):
    """Shoup's product x w mod q for x < 2^32, w < q, in 32-bit words: the quotient estimate
    floor(x floor(2^32 w / q) / 2^32) is short by at most one, then one conditional subtract."""
    x = x.astype(np.uint64)
    wq = np.uint64((int(w) << 32) // int(q))
    qt = (x * wq) >> np.uint64(32)
    r = (x * np.uint64(w) - qt * np.uint64(q)) & np.uint64(0xFFFFFFFF)
    assert (r < 2 * q).all()
    return np.where(r >= q, r - np.uint64(q), r)


@pytest.mark.parametrize("nsrc", [1, 8, 15])
def test_tensor_core_conv_reconstruction(nsrc):
    """The tensor-core form of Conv (Sec. IV-A) restated on the CPU: y_i = [x_i (B/b_i)^-1]_{b_i}
    and the constants [(B/b_i) 256^j]_{q_t} split into balanced base-256 digits, the digit GEMM
    acc_{t,k} = sum_{i,j} d_{ij} e_{ijk} in fp32, each acc read back exactly by adding 1.5 2^23,
    then lo = acc_0 + 256 acc_1 and hi = acc_2 + 256 acc_3 made positive by the multiple of q_t
    at or above 2^29, and out = [lo + [2^16 hi]_q]_q by two Shoup products, all in 32-bit words.
    It must equal the oracle's Conv for up to 15 sources (the largest the kernel takes)."""
    from oracle import ckks as OC
    qs = P.ntt_primes(nsrc + 6)
    src, dst = qs[:nsrc], qs[nsrc:]
    B = 1
    for b in src:
        B *= b
    n = 4096
    rng = np.random.default_rng(100 + nsrc)
    x = np.stack([rng.integers(0, b, n, dtype=np.int64) for b in src]).astype(np.uint64)
    # coefficient 0: every y_i has low digits -128 (largest data-digit magnitude)
    yext = 63 * (1 << 24) - 0x808080
    for i, b in enumerate(src):
        x[i, 0] = yext * ((B // b) % b) % b
    y = np.stack([(x[i] * np.uint64(pow((B // b) % b, -1, b))) % np.uint64(b)
                  for i, b in enumerate(src)]).astype(np.int64)
    assert (y[:, 0] == yext).all()
    d = _digits_from_bias(y.T)                                  # (n, nsrc, 4): digit j of y_i
    A = d.reshape(n, 4 * nsrc)                                  # K' = 4 i + j
    ref = OC.conv(x, src, dst)
    for ti, q in enumerate(dst):
        w = np.array([[(B // b) % q * pow(256, j, q) % q for j in range(4)] for b in src], dtype=np.int64)
        e = _digits_from_bias(w)                                # (nsrc, 4 j, 4 k)
        assert np.abs(e).max() <= 128
        E = e.reshape(4 * nsrc, 4)                              # row K' = 4 i + j, column k
        exact = A @ E
        assert np.abs(exact).max() <= 4 * nsrc * 128 * 128 < (1 << 20)
        acc32 = A.astype(np.float16).astype(np.float32) @ E.astype(np.float16).astype(np.float32)
        bits = (acc32 + np.float32(12582912.0)).astype(np.float32).view(np.int32).astype(np.int64)
        acc = bits - 0x4B400000
        np.testing.assert_array_equal(acc, exact)
        off = -(-(1 << 29) // q) * q
        lo = acc[:, 0] + 256 * acc[:, 1] + off
        hi = acc[:, 2] + 256 * acc[:, 3] + off
        assert lo.min() > 0 and hi.min() > 0 and lo.max() < (1 << 31) and hi.max() < (1 << 31)
        th = _shoup(hi.astype(np.uint64), (1 << 16) % q, q)
        s = lo.astype(np.uint64) + th
        assert s.max() < (1 << 32)
        out = _shoup(s, 1, q)
        np.testing.assert_array_equal(out, ref[ti])


def test_epilogue_reconstruction_bounds():
    """The GEMM epilogues' rebuild mod q: y = acc_0 + 255 acc_1 + 255^2 acc_2 + 255^3 acc_3 from
    accumulators |acc_i| <= 4K x 128 x 127 (K <= 256) stays within 2^49 in magnitude, so adding
    the least multiple of q at or above 2^49 makes it positive and below 2^51; the 64-bit
    Barrett step with mu = floor((2^64 - 1) / q) leaves a remainder below 3q, and two
    conditional subtractions give y mod q. Checked at random and at every sign corner."""
    amax = 4 * 256 * 128 * 127
    assert amax < (1 << 24)
    assert amax * (1 + 255 + 255 ** 2 + 255 ** 3) < (1 << 49)
    rng = np.random.default_rng(21)
    corners = [[s0 * amax, s1 * amax, s2 * amax, s3 * amax]
               for s0 in (-1, 1) for s1 in (-1, 1) for s2 in (-1, 1) for s3 in (-1, 1)]
    accs = corners + rng.integers(-amax, amax + 1, (20000, 4)).tolist() + [[0, 0, 0, 0]]
    for q in (P.ntt_primes(1)[0], P.ntt_primes(44)[-1]):
        mu = ((1 << 64) - 1) // q
        off = -(-(1 << 49) // q) * q
        for a in accs:
            y = a[0] + 255 * a[1] + 65025 * a[2] + 16581375 * a[3]
            x = y + off
            assert 0 < x < (1 << 51)
            r = x - ((x * mu) >> 64) * q
            assert 0 <= r < 3 * q
            r = r - 2 * q if r >= 2 * q else r
            r = r - q if r >= q else r
            assert r == y % q

"""Host-side checks of the arithmetic the tensor-core NTT relies on (Sec. IV-B, segment fusion
of Eq. (9)): the balanced 8-bit digits the kernels produce, their exact fp16 encoding, and the
exactness of the digit GEMM under fp32 accumulation at the largest reduction size.

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

"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle's
callers.

This module holds no arithmetic of the method: it only draws random numbers
(uniform residues, ternary secrets, rounded-Gaussian errors, uniform reals)
with numpy's PCG64 generator from a given seed. Both the GPU library's callers
and the CPU oracle's callers take their inputs from here, so the two sides see
identical bits.
"""
import numpy as np


def rng(seed):
    return np.random.default_rng(seed)


def uniform_residues(seed, mods, batch, n, dtype=np.uint32):
    """(len(mods), batch, n) array, limb l uniform in [0, mods[l])."""
    g = rng(seed)
    out = np.empty((len(mods), batch, n), dtype=dtype)
    for l, m in enumerate(mods):
        out[l] = g.integers(0, int(m), size=(batch, n), dtype=np.uint64).astype(dtype)
    return out


def ternary_secret(seed, n, hamming_weight=None):
    """Coefficients in {-1, 0, 1}. hamming_weight=None draws each uniformly (dense)."""
    g = rng(seed)
    if hamming_weight is None:
        return g.integers(-1, 2, size=n).astype(np.int64)
    s = np.zeros(n, dtype=np.int64)
    pos = g.choice(n, size=hamming_weight, replace=False)
    s[pos] = g.choice(np.array([-1, 1], dtype=np.int64), size=hamming_weight)
    return s


def gaussian_error(seed, shape, sigma=3.2, bound=19):
    """Rounded Gaussian, redrawn where |e| > bound (6 sigma)."""
    g = rng(seed)
    e = np.rint(g.normal(0.0, sigma, size=shape)).astype(np.int64)
    bad = np.abs(e) > bound
    while bad.any():
        e[bad] = np.rint(g.normal(0.0, sigma, size=int(bad.sum()))).astype(np.int64)
        bad = np.abs(e) > bound
    return e


def uniform_reals(seed, shape, lo=-1.0, hi=1.0):
    return rng(seed).uniform(lo, hi, size=shape)

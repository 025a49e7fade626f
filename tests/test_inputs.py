"""The seeded input generators (paper_2212_14191_gb300/inputs.py) on the CPU: the same seed
gives the same bits on every call, so the GPU and oracle sides see identical inputs; every
draw has the shape and range it documents (residues below their limb's modulus, ternary
secrets with the exact Hamming weight, rounded Gaussians within 6 sigma, reals in [lo, hi))."""
import numpy as np
import pytest

from oracle import params as P
from paper_2212_14191_gb300 import inputs as I


def test_uniform_residues_are_reproducible_and_in_range():
    mods = P.ntt_primes(5)
    a = I.uniform_residues(7, mods, 3, 1024)
    b = I.uniform_residues(7, mods, 3, 1024)
    assert a.shape == (5, 3, 1024) and a.dtype == np.uint32
    np.testing.assert_array_equal(a, b)
    assert not np.array_equal(a, I.uniform_residues(8, mods, 3, 1024))
    for l, m in enumerate(mods):
        assert a[l].max() < m
    c = I.uniform_residues(7, mods, 3, 1024, dtype=np.uint64)
    np.testing.assert_array_equal(c, a.astype(np.uint64))   # the dtype changes the carrier only


@pytest.mark.parametrize("h", [None, 64, 1])
def test_ternary_secret(h):
    s = I.ternary_secret(11, 4096, hamming_weight=h)
    np.testing.assert_array_equal(s, I.ternary_secret(11, 4096, hamming_weight=h))
    assert set(np.unique(s)) <= {-1, 0, 1}
    if h is not None:
        assert int(np.count_nonzero(s)) == h


def test_gaussian_error_bounded_and_reproducible():
    e = I.gaussian_error(13, (4, 65536))
    np.testing.assert_array_equal(e, I.gaussian_error(13, (4, 65536)))
    assert np.abs(e).max() <= 19 and abs(float(e.std()) - 3.2) < 0.05


def test_uniform_reals_range():
    z = I.uniform_reals(5, 10000)
    np.testing.assert_array_equal(z, I.uniform_reals(5, 10000))
    assert z.min() >= -1.0 and z.max() < 1.0

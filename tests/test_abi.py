"""CPU-side checks of the C-ABI library: it loads, exports every function that
include/fhe.h declares, validates arguments before touching the GPU, and its own
prime generator agrees with the oracle's (two independent implementations)."""
import ctypes

import pytest

from oracle import params as P


@pytest.fixture(scope="module")
def fhe():
    from paper_2212_14191_gb300 import build
    build.build()
    from paper_2212_14191_gb300 import fhe as f
    return f


def test_exports_every_declared_symbol(fhe):
    names = fhe.declared_functions()
    assert len(names) >= 11
    lib = ctypes.CDLL(fhe.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert set(fhe._SIGS) == set(names)


def test_gen_primes_matches_oracle(fhe):
    qs, ps = P.default_moduli(44, 8)
    assert fhe.fhe_gen_primes(16, 30, 52) == ps + qs
    for logn in (12, 14):
        assert fhe.fhe_gen_primes(logn, 30, 5) == P.ntt_primes(5, logn_max=logn)


def test_argument_validation_without_gpu(fhe):
    with pytest.raises(fhe.FheError) as e:
        fhe.fhe_gen_primes(9, 30, 1)
    assert e.value.code == fhe.FHE_EINVAL
    with pytest.raises(fhe.FheError):
        fhe.fhe_gen_primes(16, 19, 1)
    with pytest.raises(fhe.FheError) as e:
        fhe.fhe_ntt_fwd(None, 0, 12, 16, 0, 1, 1, 0)
    assert e.value.code == fhe.FHE_EINVAL and "ctx" in str(e.value)
    with pytest.raises(fhe.FheError):
        fhe.fhe_hmult(None, 12, 2, 1, 16, 16, 16, 16, 16, 0, 0)
    assert fhe.fhe_scratch_bytes(None, fhe.FHE_OP_HMULT, 12, 2, 1) == 0
    assert fhe.fhe_scratch_bytes(None, fhe.FHE_OP_HROTATE, 12, 2, 1) == 0
    assert fhe.fhe_scratch_bytes(None, fhe.FHE_OP_HROTATE_HOISTED, 12, 2, 1) == 0
    with pytest.raises(ValueError):
        fhe.fhe_hrotate_hoisted(None, 12, 2, 1, [5, 25], 16, [16], 32, 16, 0)
    for call in (lambda: fhe.fhe_automorph(None, 12, 1, 5, 16, 32),
                 lambda: fhe.fhe_hrotate(None, 12, 2, 1, 5, 16, 16, 32, 16, 0),
                 lambda: fhe.fhe_hrotate_hoisted(None, 12, 2, 1, [5, 25], 16, [16, 16], 32, 16, 0),
                 lambda: fhe.fhe_cmult(None, 12, 2, 1, 16, 16, 16),
                 lambda: fhe.fhe_hadd(None, 12, 2, 1, 16, 16, 16),
                 lambda: fhe.fhe_conv_set_path(None, fhe.FHE_CONV_TC),
                 lambda: fhe.fhe_selftest_wait_timeout(None, 1000)):
        with pytest.raises(fhe.FheError) as e:
            call()
        assert e.value.code == fhe.FHE_EINVAL and "ctx" in str(e.value)
    assert fhe.fhe_conv_get_path(None) == -1
    # bad moduli are rejected before any device allocation
    composite = ((1 << 30) - 1) // (1 << 17) * (1 << 17) + 1   # above the largest such prime
    assert composite > P.ntt_primes(1)[0]
    q0 = P.ntt_primes(1)[0]
    for q, p in (([17], []), ([(1 << 30) + 1], []), ([composite], []), ([q0, q0], [])):
        with pytest.raises(fhe.FheError) as e:
            fhe.fhe_ctx_create(16, q, p, 8)
        assert e.value.code == fhe.FHE_EINVAL
    qs, ps = P.default_moduli(16, 1)
    with pytest.raises(fhe.FheError) as e:   # P = p_0 alone is smaller than a slice of 8 primes
        fhe.fhe_ctx_create(16, qs, ps, 8)
    assert "P" in str(e.value)
    code, msg = fhe.last_error()
    assert code == fhe.FHE_EINVAL and msg


def test_binding_constants_match_the_header(fhe):
    """Every numeric #define of include/fhe.h that a caller passes or receives (status codes,
    paths, operations, batch kinds, sizes) has the same value in the binding."""
    import re
    text = open(fhe.HEADER).read()
    defs = {}
    for m in re.finditer(r"^#define (FHE_[A-Z0-9_]+) \(?(\d+)u?(?: << (\d+))?\)?", text, re.M):
        v = int(m.group(2)) << int(m.group(3) or 0)
        defs[m.group(1)] = v
    skip = {"FHE_LOGN_MIN", "FHE_LOGN_MAX", "FHE_MAX_MODULI"}   # limits checked by the library itself
    names = [n for n in defs if n not in skip]
    assert len(names) >= 20
    for n in names:
        assert hasattr(fhe, n), n
        assert getattr(fhe, n) == defs[n], (n, getattr(fhe, n), defs[n])

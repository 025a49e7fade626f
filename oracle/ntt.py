"""ctypes wrapper for oracle/ntt_oracle.c (test infrastructure only).

The C file holds the definitions: Eq. (4) of Sec. II-A evaluated term by term
(O(N^2)), the same transform via pre-twist + textbook radix-2 cyclic DFT
(O(N log N)), its inverse, and the schoolbook product in Z_q[X]/(X^N+1).
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ntt_oracle.c")
_LIB = os.path.join(_HERE, "libntt_oracle.so")
_lib = None

_u32p = ctypes.POINTER(ctypes.c_uint32)


def build(force: bool = False) -> str:
    """Compile the oracle C file with gcc -O3 (+OpenMP). Portable flags only: no -march=native, so
    the same source builds on the x86 and the Arm hosts."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O3", "-fopenmp", "-shared", "-fPIC", "-std=c99",
                               _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.oracle_powmod.restype = ctypes.c_uint32
        L.oracle_powmod.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32]
        for name in ("oracle_ntt_brute", "oracle_intt_brute", "oracle_ntt", "oracle_intt"):
            f = getattr(L, name)
            f.restype = None
            f.argtypes = [_u32p, _u32p, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint32]
        L.oracle_negacyclic_mul.restype = None
        L.oracle_negacyclic_mul.argtypes = [_u32p, _u32p, _u32p, ctypes.c_int, ctypes.c_uint32]
        L.oracle_ntt_batch.restype = ctypes.c_int
        L.oracle_ntt_batch.argtypes = [_u32p, _u32p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       _u32p, _u32p, ctypes.c_int, ctypes.c_int]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(_u32p)


def _vec(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint32))


def _one(fn, a, q, psi):
    a = _vec(a)
    out = np.empty_like(a)
    getattr(lib(), fn)(_p(a), _p(out), int(a.shape[-1]), int(q), int(psi))
    return out


def ntt_brute(a, q, psi):
    """Eq. (4), term by term."""
    return _one("oracle_ntt_brute", a, q, psi)


def intt_brute(A, q, psi):
    """Inverse of Eq. (4), term by term."""
    return _one("oracle_intt_brute", A, q, psi)


def ntt(a, q, psi):
    """Eq. (4) via pre-twist + cyclic DFT, one polynomial."""
    return _one("oracle_ntt", a, q, psi)


def intt(A, q, psi):
    return _one("oracle_intt", A, q, psi)


def negacyclic_mul(a, b, q):
    a, b = _vec(a), _vec(b)
    c = np.empty_like(a)
    lib().oracle_negacyclic_mul(_p(a), _p(b), _p(c), int(a.shape[-1]), int(q))
    return c


def ntt_batch(x, qs, psis, inverse=False, threads=0):
    """Transform every row of a (L, B, N) (or (L, N)) array; limb l uses qs[l], psis[l].

    Returns (out, threads_used).
    """
    x = _vec(x)
    squeeze = x.ndim == 2
    if squeeze:
        x = x[:, None, :]
    L, B, N = x.shape
    qa, pa = _vec(qs), _vec(psis)
    assert qa.shape == (L,) and pa.shape == (L,)
    out = np.empty_like(x)
    used = lib().oracle_ntt_batch(_p(x), _p(out), L, B, N, _p(qa), _p(pa), int(bool(inverse)),
                                  int(threads))
    return (out[:, 0, :] if squeeze else out), used


def powmod(b, e, q):
    return int(lib().oracle_powmod(int(b), int(e), int(q)))

"""Thin ctypes binding of libfhe.so (include/fhe.h).

The functions named fhe_* below have the C entry points' names and arguments and only
marshal them (ints, device pointers as ints, the CUDA stream handle). Every step of the
computation runs in the library's CUDA kernels; there is no Python or CPU fallback: if the
library is missing, importing this module raises.

`Context` is a convenience layer that takes torch tensors (int32 carriers of uint32 bits,
on the CUDA device) and passes their data pointers and the current torch stream.
"""
import ctypes
import os
import re

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfhe.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "fhe.h")

FHE_OK, FHE_EINVAL, FHE_ENOMEM, FHE_ECUDA, FHE_ETIMEOUT = 0, 1, 2, 3, 4
FHE_NTT_DEFAULT, FHE_NTT_U32, FHE_NTT_TC = 0, 1, 2
FHE_NTT_VARIANT_TC64, FHE_NTT_VARIANT_TC32 = 32, 33
FHE_CONV_CUDA, FHE_CONV_TC = 0, 1
FHE_OP_HMULT, FHE_OP_KEYSWITCH, FHE_OP_RESCALE, FHE_OP_HMULT_RELIN, FHE_OP_HROTATE = 1, 2, 3, 4, 5
FHE_OP_HROTATE_HOISTED = 6
FHE_RESCALE_NOALLOC_MAX_BYTES = 32 << 20

if not os.path.exists(LIB_PATH):
    raise ImportError("libfhe.so is not built (run `python -c 'import __graft_entry__ as g; g.build()'`)")

_lib = ctypes.CDLL(LIB_PATH)

_u32p = ctypes.POINTER(ctypes.c_uint32)
_vp = ctypes.c_void_p
_u32 = ctypes.c_uint32
_i = ctypes.c_int
_sz = ctypes.c_size_t

FHE_OPK_NTT_FWD, FHE_OPK_NTT_INV, FHE_OPK_HMULT = 1, 2, 3
FHE_BATCH_PERSISTENT, FHE_BATCH_GROUPED = 0, 1


class FheOp(ctypes.Structure):
    """struct fhe_op of include/fhe.h."""
    _fields_ = [("kind", ctypes.c_int), ("logN", ctypes.c_uint32), ("first_limb", ctypes.c_int),
                ("n_limbs", ctypes.c_int), ("batch", ctypes.c_int), ("data", ctypes.c_void_p),
                ("a", ctypes.c_void_p), ("b", ctypes.c_void_p), ("evk", ctypes.c_void_p),
                ("out", ctypes.c_void_p)]


_SIGS = {
    "fhe_gen_primes": (_i, [_u32, _i, _i, _u32p]),
    "fhe_ctx_create": (_i, [_u32, _u32p, _i, _u32p, _i, _i, _i, ctypes.POINTER(_vp)]),
    "fhe_ctx_destroy": (_i, [_vp]),
    "fhe_ntt_fwd": (_i, [_vp, _i, _u32, _vp, _i, _i, _i, _vp]),
    "fhe_ntt_inv": (_i, [_vp, _i, _u32, _vp, _i, _i, _i, _vp]),
    "fhe_scratch_bytes": (_sz, [_vp, _i, _u32, _i, _i]),
    "fhe_keyswitch": (_i, [_vp, _u32, _i, _i, _vp, _vp, _vp, _vp, _sz, _vp]),
    "fhe_hmult_relin": (_i, [_vp, _u32, _i, _i, _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "fhe_rescale": (_i, [_vp, _u32, _i, _i, _vp, _vp, _vp, _sz, _vp]),
    "fhe_hmult": (_i, [_vp, _u32, _i, _i, _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "fhe_rescale_noalloc": (_i, [_vp, _u32, _i, _i, _vp, _vp, _vp]),
    "fhe_automorph": (_i, [_vp, _u32, ctypes.c_longlong, _u32, _vp, _vp, _vp]),
    "fhe_hrotate": (_i, [_vp, _u32, _i, _i, _u32, _vp, _vp, _vp, _vp, _sz, _vp]),
    "fhe_hrotate_hoisted": (_i, [_vp, _u32, _i, _i, _i, _u32p, _vp, ctypes.POINTER(_vp), _vp, _vp, _sz, _vp]),
    "fhe_cmult": (_i, [_vp, _u32, _i, _i, _vp, _vp, _vp, _vp]),
    "fhe_hadd": (_i, [_vp, _u32, _i, _i, _vp, _vp, _vp, _vp]),
    "fhe_device_status": (_i, [_vp, _i]),
    "fhe_ntt_variant_count": (_i, [_vp, _u32]),
    "fhe_ntt_get_variant": (_i, [_vp, _u32, _i]),
    "fhe_ntt_set_variant": (_i, [_vp, _u32, _i, _i]),
    "fhe_conv_set_path": (_i, [_vp, _i]),
    "fhe_selftest_wait_timeout": (_i, [_vp, ctypes.c_longlong, _vp]),
    "fhe_conv_get_path": (_i, [_vp]),
    "fhe_autotune_ntt": (_i, [_vp, _u32, _vp, _i, _i, _i, ctypes.POINTER(ctypes.c_float), _vp]),
    "fhe_last_error": (_i, [ctypes.c_char_p, _sz]),
    "fhe_batch_create": (_i, [_vp, ctypes.POINTER(FheOp), _i, ctypes.POINTER(_vp)]),
    "fhe_batch_create_ex": (_i, [_vp, ctypes.POINTER(FheOp), _i, _i, _sz, ctypes.POINTER(_vp)]),
    "fhe_selftest_queue_timeout": (_i, [_vp, ctypes.c_longlong, _vp]),
    "fhe_batch_scratch_bytes": (_sz, [_vp]),
    "fhe_batch_run": (_i, [_vp, _vp, _sz, _vp]),
    "fhe_batch_capture": (_i, [_vp, _vp, _sz]),
    "fhe_batch_launch": (_i, [_vp, _vp]),
    "fhe_batch_destroy": (_i, [_vp]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class FheError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("libfhe error %d: %s" % (code, msg))
        self.code = code


def last_error():
    buf = ctypes.create_string_buffer(512)
    code = _lib.fhe_last_error(buf, 512)
    return code, buf.value.decode(errors="replace")


def _check(rc):
    if rc != FHE_OK:
        raise FheError(rc, last_error()[1])
    return rc


def declared_functions():
    """Names of the functions declared in include/fhe.h."""
    with open(HEADER) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|size_t)\s+(fhe_\w+)\s*\(", text, flags=re.M)))


# ---------------------------------------------------------------- C entry points


def fhe_gen_primes(logN_max, bits, count):
    out = (ctypes.c_uint32 * count)()
    _check(_lib.fhe_gen_primes(logN_max, bits, count, out))
    return [int(x) for x in out]


def fhe_ctx_create(logN_max, q, p, alpha, default_path=FHE_NTT_U32):
    qa = (ctypes.c_uint32 * max(1, len(q)))(*q)
    pa = (ctypes.c_uint32 * max(1, len(p)))(*p)
    h = _vp()
    _check(_lib.fhe_ctx_create(logN_max, qa, len(q), pa, len(p), alpha, default_path, ctypes.byref(h)))
    return h.value


def fhe_ctx_destroy(ctx):
    return _check(_lib.fhe_ctx_destroy(ctx))


def fhe_ntt_fwd(ctx, path, logN, d_ptr, first_limb, n_limbs, batch, stream=0):
    return _check(_lib.fhe_ntt_fwd(ctx, path, logN, d_ptr, first_limb, n_limbs, batch, stream))


def fhe_ntt_inv(ctx, path, logN, d_ptr, first_limb, n_limbs, batch, stream=0):
    return _check(_lib.fhe_ntt_inv(ctx, path, logN, d_ptr, first_limb, n_limbs, batch, stream))


def fhe_scratch_bytes(ctx, op, logN, n_limbs, batch):
    return int(_lib.fhe_scratch_bytes(ctx, op, logN, n_limbs, batch))


def fhe_keyswitch(ctx, logN, n_limbs, batch, d2, evk, ks_out, scratch, scratch_bytes, stream=0):
    return _check(_lib.fhe_keyswitch(ctx, logN, n_limbs, batch, d2, evk, ks_out, scratch, scratch_bytes, stream))


def fhe_hmult_relin(ctx, logN, n_limbs, batch, a, b, evk, out, scratch, scratch_bytes, stream=0):
    return _check(_lib.fhe_hmult_relin(ctx, logN, n_limbs, batch, a, b, evk, out, scratch, scratch_bytes, stream))


def fhe_rescale(ctx, logN, n_limbs, batch, ct_in, ct_out, scratch, scratch_bytes, stream=0):
    return _check(_lib.fhe_rescale(ctx, logN, n_limbs, batch, ct_in, ct_out, scratch, scratch_bytes, stream))


def fhe_rescale_noalloc(ctx, logN, n_limbs, batch, ct_in, ct_out, stream=0):
    return _check(_lib.fhe_rescale_noalloc(ctx, logN, n_limbs, batch, ct_in, ct_out, stream))


def fhe_hmult(ctx, logN, n_limbs, batch, a, b, evk, out, scratch, scratch_bytes, stream=0):
    return _check(_lib.fhe_hmult(ctx, logN, n_limbs, batch, a, b, evk, out, scratch, scratch_bytes, stream))


def fhe_automorph(ctx, logN, rows, galois, d_in, d_out, stream=0):
    return _check(_lib.fhe_automorph(ctx, logN, rows, galois, d_in, d_out, stream))


def fhe_hrotate(ctx, logN, n_limbs, batch, galois, ct_in, ksk, ct_out, scratch, scratch_bytes, stream=0):
    return _check(_lib.fhe_hrotate(ctx, logN, n_limbs, batch, galois, ct_in, ksk, ct_out, scratch, scratch_bytes,
                                   stream))


def fhe_hrotate_hoisted(ctx, logN, n_limbs, batch, galois, ct_in, ksks, ct_out, scratch, scratch_bytes, stream=0):
    """galois: list of Galois elements; ksks: list of device pointers (one key per element)."""
    n = len(galois)
    if len(ksks) != n:
        raise ValueError("one key per Galois element")
    g = (ctypes.c_uint32 * max(1, n))(*galois)
    k = (_vp * max(1, n))(*ksks)
    return _check(_lib.fhe_hrotate_hoisted(ctx, logN, n_limbs, batch, n, g, ct_in, k, ct_out, scratch,
                                           scratch_bytes, stream))


def fhe_cmult(ctx, logN, n_limbs, batch, ct, pt, ct_out, stream=0):
    return _check(_lib.fhe_cmult(ctx, logN, n_limbs, batch, ct, pt, ct_out, stream))


def fhe_hadd(ctx, logN, n_limbs, batch, ct_a, ct_b, ct_out, stream=0):
    return _check(_lib.fhe_hadd(ctx, logN, n_limbs, batch, ct_a, ct_b, ct_out, stream))


def fhe_device_status(ctx, clear=1):
    return _check(_lib.fhe_device_status(ctx, clear))


def fhe_ntt_variant_count(ctx, logN):
    return int(_lib.fhe_ntt_variant_count(ctx, logN))


def fhe_ntt_get_variant(ctx, logN, inverse=0):
    return int(_lib.fhe_ntt_get_variant(ctx, logN, 1 if inverse else 0))


def fhe_ntt_set_variant(ctx, logN, variant, inv_variant=None):
    """Select the forward variant and the inverse one (the same unless given)."""
    inv = variant if inv_variant is None else inv_variant
    return _check(_lib.fhe_ntt_set_variant(ctx, logN, variant, inv))


def fhe_conv_set_path(ctx, path):
    return _check(_lib.fhe_conv_set_path(ctx, path))


def fhe_conv_get_path(ctx):
    return int(_lib.fhe_conv_get_path(ctx))


def fhe_selftest_wait_timeout(ctx, limit_cycles, stream=0):
    return _check(_lib.fhe_selftest_wait_timeout(ctx, limit_cycles, stream))


def fhe_autotune_ntt(ctx, logN, d_ptr, n_limbs, batch, reps=3, stream=0):
    """Returns (forward_ms, inverse_ms): per-variant milliseconds per call measured by the
    library (-1 where a variant does not apply); the fastest of each is kept."""
    n = max(1, fhe_ntt_variant_count(ctx, logN))
    ms = (ctypes.c_float * (2 * n))()
    _check(_lib.fhe_autotune_ntt(ctx, logN, d_ptr, n_limbs, batch, reps, ms, stream))
    return [float(x) for x in ms[:n]], [float(x) for x in ms[n:]]


def fhe_batch_create(ctx, ops):
    arr = (FheOp * max(1, len(ops)))(*ops)
    h = _vp()
    _check(_lib.fhe_batch_create(ctx, arr, len(ops), ctypes.byref(h)))
    return h.value


def fhe_batch_create_ex(ctx, ops, mode=FHE_BATCH_PERSISTENT, slot_bytes=0):
    arr = (FheOp * max(1, len(ops)))(*ops)
    h = _vp()
    _check(_lib.fhe_batch_create_ex(ctx, arr, len(ops), mode, slot_bytes, ctypes.byref(h)))
    return h.value


def fhe_selftest_queue_timeout(ctx, limit_cycles, stream=0):
    return _check(_lib.fhe_selftest_queue_timeout(ctx, limit_cycles, stream))


def fhe_batch_scratch_bytes(batch):
    return int(_lib.fhe_batch_scratch_bytes(batch))


def fhe_batch_run(batch, scratch, scratch_bytes, stream=0):
    return _check(_lib.fhe_batch_run(batch, scratch, scratch_bytes, stream))


def fhe_batch_capture(batch, scratch, scratch_bytes):
    return _check(_lib.fhe_batch_capture(batch, scratch, scratch_bytes))


def fhe_batch_launch(batch, stream=0):
    return _check(_lib.fhe_batch_launch(batch, stream))


def fhe_batch_destroy(batch):
    return _check(_lib.fhe_batch_destroy(batch))


# ---------------------------------------------------------------- torch convenience layer


def _ptr(t):
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "expected a contiguous CUDA tensor"
    return t.data_ptr()


def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


class Context:
    """Owns an fhe_ctx; tensors are int32 CUDA tensors carrying uint32 residues."""

    def __init__(self, logN_max, q, p=(), alpha=8, default_path=FHE_NTT_U32):
        self.logN_max = logN_max
        self.q = list(q)
        self.p = list(p)
        self.alpha = alpha
        self.handle = fhe_ctx_create(logN_max, self.q, self.p, alpha, default_path)
        self._scratch = None

    def close(self):
        if self.handle:
            fhe_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def moduli(self):
        return self.q + self.p

    def ntt_fwd(self, x, logN, first_limb=0, path=FHE_NTT_DEFAULT):
        n_limbs, batch = x.shape[0], x.shape[1]
        fhe_ntt_fwd(self.handle, path, logN, _ptr(x), first_limb, n_limbs, batch, _stream())
        return x

    def ntt_inv(self, x, logN, first_limb=0, path=FHE_NTT_DEFAULT):
        n_limbs, batch = x.shape[0], x.shape[1]
        fhe_ntt_inv(self.handle, path, logN, _ptr(x), first_limb, n_limbs, batch, _stream())
        return x

    def scratch(self, op, logN, n_limbs, batch):
        import torch
        nbytes = fhe_scratch_bytes(self.handle, op, logN, n_limbs, batch)
        if self._scratch is None or self._scratch.numel() * 4 < nbytes:
            self._scratch = torch.empty(max(4, nbytes // 4), dtype=torch.int32, device="cuda")
        return self._scratch, nbytes

    def hmult(self, a, b, evk, logN, out=None):
        import torch
        nl, batch = a.shape[1], a.shape[2]
        if out is None:
            out = torch.empty((2, nl - 1, batch, 1 << logN), dtype=torch.int32, device=a.device)
        s, n = self.scratch(FHE_OP_HMULT, logN, nl, batch)
        fhe_hmult(self.handle, logN, nl, batch, _ptr(a), _ptr(b), _ptr(evk), _ptr(out), _ptr(s), n, _stream())
        return out

    def hmult_relin(self, a, b, evk, logN, out=None):
        import torch
        nl, batch = a.shape[1], a.shape[2]
        if out is None:
            out = torch.empty((2, nl, batch, 1 << logN), dtype=torch.int32, device=a.device)
        s, n = self.scratch(FHE_OP_HMULT_RELIN, logN, nl, batch)
        fhe_hmult_relin(self.handle, logN, nl, batch, _ptr(a), _ptr(b), _ptr(evk), _ptr(out), _ptr(s), n, _stream())
        return out

    def keyswitch(self, d2, evk, logN, out=None):
        import torch
        nl, batch = d2.shape[0], d2.shape[1]
        if out is None:
            out = torch.empty((2, nl, batch, 1 << logN), dtype=torch.int32, device=d2.device)
        s, n = self.scratch(FHE_OP_KEYSWITCH, logN, nl, batch)
        fhe_keyswitch(self.handle, logN, nl, batch, _ptr(d2), _ptr(evk), _ptr(out), _ptr(s), n, _stream())
        return out

    def rescale(self, ct, logN, out=None):
        import torch
        nl, batch = ct.shape[1], ct.shape[2]
        if out is None:
            out = torch.empty((2, nl - 1, batch, 1 << logN), dtype=torch.int32, device=ct.device)
        s, n = self.scratch(FHE_OP_RESCALE, logN, nl, batch)
        fhe_rescale(self.handle, logN, nl, batch, _ptr(ct), _ptr(out), _ptr(s), n, _stream())
        return out

    def automorph(self, x, logN, galois, out=None):
        """FrobeniusMap of every row of x (..., N), NTT domain."""
        import torch
        if out is None:
            out = torch.empty_like(x)
        fhe_automorph(self.handle, logN, x.numel() >> logN, galois, _ptr(x), _ptr(out), _stream())
        return out

    def hrotate(self, ct, ksk, logN, galois, out=None):
        import torch
        nl, batch = ct.shape[1], ct.shape[2]
        if out is None:
            out = torch.empty_like(ct)
        s, n = self.scratch(FHE_OP_HROTATE, logN, nl, batch)
        fhe_hrotate(self.handle, logN, nl, batch, galois, _ptr(ct), _ptr(ksk), _ptr(out), _ptr(s), n, _stream())
        return out

    def hrotate_hoisted(self, ct, ksks, logN, galois, out=None):
        """Hoisted rotations of ct by every element of `galois` (one key each, same order):
        returns (len(galois), 2, nl, batch, N)."""
        import torch
        nl, batch = ct.shape[1], ct.shape[2]
        if out is None:
            out = torch.empty((len(galois),) + tuple(ct.shape), dtype=ct.dtype, device=ct.device)
        s, n = self.scratch(FHE_OP_HROTATE_HOISTED, logN, nl, batch)
        fhe_hrotate_hoisted(self.handle, logN, nl, batch, list(galois), _ptr(ct), [_ptr(k) for k in ksks],
                            _ptr(out), _ptr(s), n, _stream())
        return out

    def cmult(self, ct, pt, logN, out=None):
        import torch
        nl, batch = ct.shape[1], ct.shape[2]
        if out is None:
            out = torch.empty_like(ct)
        fhe_cmult(self.handle, logN, nl, batch, _ptr(ct), _ptr(pt), _ptr(out), _stream())
        return out

    def hadd(self, a, b, logN, out=None):
        import torch
        nl, batch = a.shape[1], a.shape[2]
        if out is None:
            out = torch.empty_like(a)
        fhe_hadd(self.handle, logN, nl, batch, _ptr(a), _ptr(b), _ptr(out), _stream())
        return out


def to_device(arr_u32):
    """numpy uint32 array -> int32 CUDA tensor with the same bits."""
    import numpy as np
    import torch
    a = np.ascontiguousarray(arr_u32, dtype=np.uint32).view(np.int32)
    return torch.from_numpy(a).cuda()


def to_host(t):
    """int32 tensor -> numpy uint32 array with the same bits."""
    import numpy as np
    return t.detach().cpu().numpy().view(np.uint32)

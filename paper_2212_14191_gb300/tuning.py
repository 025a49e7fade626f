"""Autotune cache for the NTT variants (the autotuned kernel shapes of Sec. IV-E).

fhe_autotune_ntt times every applicable variant of a ring degree on the caller's data (the
plain-path kernel shapes and the tensor-core path's two output tile widths) and keeps the
fastest forward and inverse choices in the context. This module stores those choices in a
JSON file keyed by (GPU name, ring degree, limbs, batch), so that a later process on the same
kind of GPU and workload sets them directly instead of timing every variant again. A stored
id that the library no longer offers is ignored and the autotuner runs again.
"""
import json
import os
import tempfile


def cache_key(device_name, logN, n_limbs, batch):
    return "%s|N=2^%d|limbs=%d|batch=%d" % (device_name, logN, n_limbs, batch)


class TuneCache:
    """Variant choices by key, read from and written to one JSON file (written atomically)."""

    def __init__(self, path):
        self.path = path
        self.entries = {}
        try:
            with open(path) as f:
                data = json.load(f)
            if isinstance(data, dict):
                self.entries = {k: v for k, v in data.items()
                                if isinstance(v, dict) and isinstance(v.get("fwd"), int)
                                and isinstance(v.get("inv"), int)}
        except (OSError, ValueError):
            self.entries = {}

    def get(self, key):
        e = self.entries.get(key)
        return None if e is None else (e["fwd"], e["inv"])

    def put(self, key, fwd, inv, ms=None):
        self.entries[key] = {"fwd": int(fwd), "inv": int(inv)}
        if ms is not None:
            self.entries[key]["ms"] = ms

    def save(self):
        d = os.path.dirname(os.path.abspath(self.path))
        os.makedirs(d, exist_ok=True)
        fd, tmp = tempfile.mkstemp(dir=d, prefix=".tune-", suffix=".json")
        with os.fdopen(fd, "w") as f:
            json.dump(self.entries, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)


def tuned_variants(fhe, ctx, logN, d_ptr, n_limbs, batch, device_name, cache, reps=2, stream=0):
    """Set the context's forward and inverse variants for logN from the cache, or autotune on
    `d_ptr` ((n_limbs, batch, N) on the device, restored by the autotuner) and record the
    result. Returns ((fwd, inv), hit). `fhe` is the binding module (or a stand-in)."""
    key = cache_key(device_name, logN, n_limbs, batch)
    hit = cache.get(key)
    count = fhe.fhe_ntt_variant_count(ctx, logN)
    if hit is not None and all(0 <= v < count for v in hit):
        try:
            fhe.fhe_ntt_set_variant(ctx, logN, hit[0], hit[1])
            return hit, True
        except fhe.FheError:
            pass                                   # not applicable any more: tune again
    fwd_ms, inv_ms = fhe.fhe_autotune_ntt(ctx, logN, d_ptr, n_limbs, batch, reps=reps, stream=stream)
    chosen = (fhe.fhe_ntt_get_variant(ctx, logN, 0), fhe.fhe_ntt_get_variant(ctx, logN, 1))
    ms = None
    if fwd_ms is not None:
        ms = {"fwd": fwd_ms[chosen[0]], "inv": inv_ms[chosen[1]]}
    cache.put(key, chosen[0], chosen[1], ms)
    cache.save()
    return chosen, False

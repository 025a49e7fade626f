"""The padded shared-memory layout of the plain NTT kernels (PadLayout in csrc/common.cuh:
position p at p + p/32 + p/T for T > 32 threads), checked on the CPU for every CTA shape and
row split the kernels are built with: the map is one-to-one and fits its allocation, every
access the rounds make is a per-thread base plus a compile-time offset (the forms the
kernels precompute), and every warp-wide access of a round and of the bit-reversal store
touches 32 distinct banks. The formulas are restated here and matched against the source."""
import os
import re

import pytest

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_2212_14191_gb300", "csrc", "common.cuh")

# (log2 threads per CTA, log2 parts per row) of the kernel instantiations
SHAPES = [(5, 0), (6, 0), (7, 0), (8, 0), (9, 0), (9, 1), (9, 2), (6, 1), (7, 1), (8, 1), (8, 2), (8, 3)]


def rev(x, b):
    r = 0
    for i in range(b):
        r |= ((x >> i) & 1) << (b - 1 - i)
    return r


def layout(lt):
    t = 1 << lt
    hi = 1 if lt > 5 else 0
    return t, hi, t + t // 32 + hi, 33 * t + 32, (lambda p: p + (p >> 5) + hi * (p >> lt))


def test_restated_formulas_match_the_source():
    src = re.sub(r"\s+", " ", open(SRC).read())
    for piece in ("kHi = LOG_T > 5 ? 1 : 0;", "kSA = T + T / 32 + kHi;", "kWords = 33 * T + 32;",
                  "return p + (p >> 5) + (kHi ? (p >> LOG_T) : 0);",
                  "return u * ((T >> LOG_C) + (T >> (LOG_C + 5))) + kHi * (u >> LOG_C);"):
        assert piece in src, piece


@pytest.mark.parametrize("lt,lc", SHAPES)
def test_layout_is_a_bijection_with_fixed_offsets(lt, lc):
    t, hi, sa, words, pad = layout(lt)
    c_parts, nc = 1 << lc, 32 * t
    vals = [pad(p) for p in range(nc)]
    assert len(set(vals)) == nc and max(vals) < words

    def off_k(u):
        return u * ((t >> lc) + (t >> (lc + 5))) + hi * (u >> lc)

    for c in range(c_parts):
        for tid in range(t):
            base = pad(tid)
            assert all(pad(tid + t * e) == base + sa * e for e in range(32))          # round A
            g = rev(tid, lt)
            assert all(pad(32 * g + e) == pad(32 * g) + e for e in range(32))         # round C
            if c_parts > 1:
                per = nc // c_parts
                px = pad(c * per + tid)
                assert all(pad(c * per + u * t + tid) == px + u * sa for u in range(32 // c_parts))
                pk = pad((c * nc + tid) >> lc)
                for u in range(32):
                    k = c * nc + u * t + tid
                    assert pad(k >> lc) == pk + off_k(u)
    rb = lt - 5
    if rb > 0:                                                                        # round B
        for g in range(32):
            for lane in range(32):
                for e in range(1 << rb):
                    assert pad(t * g + lane + 32 * e) == g * sa + lane + 33 * e


@pytest.mark.parametrize("lt", sorted({s[0] for s in SHAPES}))
def test_warp_accesses_are_conflict_free(lt):
    t, hi, sa, _, pad = layout(lt)

    def distinct_banks(addrs):
        return len({a % 32 for a in addrs}) == len(addrs)

    for w in range(t // 32):
        tids = [32 * w + lane for lane in range(32)]
        for e in range(32):
            assert distinct_banks([pad(x + t * e) for x in tids])                     # round A
            assert distinct_banks([pad(32 * rev(x, lt) + e) for x in tids])           # round C
            assert distinct_banks([pad(rev(e, 5) * t + x) for x in tids])             # natural-order store
        rb = lt - 5
        if rb > 0:
            per_warp = 32 >> rb
            for gi in range(per_warp):
                g = w * per_warp + gi
                for e in range(1 << rb):
                    assert distinct_banks([g * sa + lane + 33 * e for lane in range(32)])  # round B

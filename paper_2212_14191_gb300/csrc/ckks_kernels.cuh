// Device code of the CKKS HMULT stages (Sec. IV-A: Hada-Mult, Ele-Add, Conv) as range functions:
// each processes the 16-byte words [i, end) of one limb with stride `step`, so that the
// stand-alone launches of ckks.cu (grid-stride loops) and the tiles of the persistent batch
// kernel (persist.cu, one chunk of a limb per tile) run the same arithmetic.
//
// COH selects how data written earlier in the same kernel is read: through L2 (ld.global.cg,
// coherent across CTAs) instead of the read-only path. The stand-alone kernels read only what
// earlier launches wrote and use the read-only path.
#pragma once
#include "common.cuh"

namespace fhe {
namespace {

// Per-limb moduli with the constants of reduce_red: r32 = 2^32 mod q with its Shoup quotient,
// m32 = floor(2^32 / q); and qinv = q^-1 mod 2^32 for the Montgomery step of Conv.
struct ModVec {
    uint32_t q[kMaxLimbs];
    uint32_t r32[kMaxLimbs], r32s[kMaxLimbs], m32[kMaxLimbs], qinv[kMaxLimbs];
};

inline ModVec modvec(const fhe_ctx* ctx, const int* mod_idx, int n) {
    ModVec m;
    memset(&m, 0, sizeof(m));
    for (int l = 0; l < n; ++l) {
        const uint32_t q = ctx->mods[mod_idx[l]];
        m.q[l] = q;
        m.r32[l] = (uint32_t)((1ull << 32) % q);
        m.r32s[l] = shoup_h(m.r32[l], q);
        m.m32[l] = (uint32_t)((1ull << 32) / q);
        uint32_t x = q;  // q^-1 mod 2^32 by Newton's iteration (q odd; each step doubles the bits)
        for (int k = 0; k < 5; ++k) x *= 2u - q * x;
        m.qinv[l] = x;
    }
    return m;
}

struct Red {
    uint32_t q, r32, r32s, m32;
};
__device__ __forceinline__ Red red_of(const ModVec& m, int l) { return Red{m.q[l], m.r32[l], m.r32s[l], m.m32[l]}; }

// x mod q for any x < 2^64 (q < 2^30): the high word times 2^32 mod q by Shoup's method and the
// low word by a 32-bit Barrett step, each in [0, 2q), summed below 4q and corrected twice.
__device__ __forceinline__ uint32_t reduce_red(uint64_t x, const Red& r) {
    const uint32_t xl = (uint32_t)x;
    const uint32_t t = mul_shoup_lazy((uint32_t)(x >> 32), r.r32, r.r32s, r.q);
    const uint32_t u = xl - __umulhi(xl, r.m32) * r.q;
    return csub(csub(t + u, 2 * r.q), r.q);
}
// Montgomery step: for x < 2^64, m = x_lo q^-1 mod 2^32 makes m q agree with x in its low word,
// so x_hi - floor(m q / 2^32) is exactly (x - m q) / 2^32, congruent to x 2^-32 mod q and above
// -q. Returned as that value plus q (GUARD false: the caller knows x_hi + q < 2^32), or plus q
// only where it is negative (GUARD true).
template <bool GUARD>
__device__ __forceinline__ uint32_t redc(uint64_t x, uint32_t q, uint32_t qinv) {
    const uint32_t hi = (uint32_t)(x >> 32), u = __umulhi((uint32_t)x * qinv, q);
    if constexpr (GUARD)
        return hi - u + (hi < u ? q : 0u);
    else
        return hi - u + q;
}
// v mod q for v < 2^32 (32-bit Barrett, one correction above [0, 2q)).
__device__ __forceinline__ uint32_t reduce32(uint32_t v, const Red& r) {
    return csub(v - __umulhi(v, r.m32) * r.q, r.q);
}

// 16-byte word i of p: the read-only path, or (COH) through L2.
template <bool COH = false>
__device__ __forceinline__ uint4 ld4(const uint32_t* p, size_t i) {
    if constexpr (COH)
        return __ldcg(reinterpret_cast<const uint4*>(p) + i);
    else
        return __ldg(reinterpret_cast<const uint4*>(p) + i);
}
__device__ __forceinline__ void st4(uint32_t* p, size_t i, uint4 v) {
    reinterpret_cast<uint4*>(p)[i] = v;
}
__device__ __forceinline__ uint32_t get(const uint4& v, int k) {
    return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w;
}
__device__ __forceinline__ void set(uint4& v, int k, uint32_t x) {
    if (k == 0) v.x = x;
    else if (k == 1) v.y = x;
    else if (k == 2) v.z = x;
    else v.w = x;
}

// ---- HM-1: tensor product (Hada-Mult + Ele-Add), d2 written twice (NTT form + copy for INTT).
// dscale (nullable): limbs l < scale_lt write d0 and d1 multiplied by dscale[l] (Shoup pair).
struct TensorArgs {
    const uint32_t* a;
    const uint32_t* b;
    uint32_t* d0;
    uint32_t* d1;
    uint32_t* d2;
    uint32_t* d2c;  // a second copy of d2, or null
    size_t L4, comp4;
    ModVec m;
    const uint2* dscale;
    int scale_lt;
};

// The inputs a, b are never written by the pipeline, so they are read through the read-only path.
__device__ __forceinline__ void tensor_range(const TensorArgs& t, int l, size_t i, size_t end, size_t step) {
    const Red rd = red_of(t.m, l);
    const bool scaled = t.dscale != nullptr && l < t.scale_lt;
    const uint2 sc = scaled ? __ldg(&t.dscale[l]) : make_uint2(0, 0);
    const uint32_t q = t.m.q[l];
    for (; i < end; i += step) {
        const size_t idx = (size_t)l * t.L4 + i;
        uint4 a0 = ld4(t.a, idx), a1 = ld4(t.a, t.comp4 + idx), b0 = ld4(t.b, idx), b1 = ld4(t.b, t.comp4 + idx);
        uint4 r0, r1, r2;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint32_t x0 = get(a0, k), x1 = get(a1, k), y0 = get(b0, k), y1 = get(b1, k);
            uint32_t v0 = reduce_red((uint64_t)x0 * y0, rd), v1 = reduce_red((uint64_t)x0 * y1 + (uint64_t)x1 * y0, rd);
            if (scaled) {
                v0 = mul_shoup(v0, sc.x, sc.y, q);
                v1 = mul_shoup(v1, sc.x, sc.y, q);
            }
            set(r0, k, v0);
            set(r1, k, v1);
            set(r2, k, reduce_red((uint64_t)x1 * y1, rd));
        }
        st4(t.d0, idx, r0);
        st4(t.d1, idx, r1);
        st4(t.d2, idx, r2);
        if (t.d2c) st4(t.d2c, idx, r2);
    }
}

// ---- KS-2 / KS-5: Conv (fast basis conversion, Sec. IV-A)
//   y_i = [x_i * (B/b_i)^-1]_{b_i};  out_t = sum_i y_i * [B/b_i]_t  mod t
struct ConvArgs {
    const uint32_t* src;
    size_t src_stride;  // elements between source limbs
    int nsrc;
    uint32_t src_q[16];
    uint2 hat_inv[16];
    const uint32_t* hat_mod;  // [nsrc][nmod]
    int nmod;
    uint32_t* dst;
    size_t dst_stride;
    int ndst;
    uint8_t dst_mod[kMaxLimbs];
    ModVec dm;
    size_t L4;  // residues per limb / 4
    // destinations t < scale_lt come out multiplied by s1[t] s2[t] (Shoup pairs mod q_t, folded
    // into the constants [B/b_i]_t; s2 may be null); 0 leaves every destination unscaled
    const uint2* s1;
    const uint2* s2;
    int scale_lt;
};

// The constants [B/b_i]_t of every (source, destination) pair, scaled where asked, into the
// CTA's shared memory s_hat[nsrc][ndst], in Montgomery form (times 2^32 mod q_t: conv_range
// reduces its sums with one Montgomery step). The caller synchronises the CTA before using them.
__device__ __forceinline__ void conv_load_hat(const ConvArgs& a, int nsrc, uint32_t* s_hat) {
    for (int k = threadIdx.x; k < nsrc * a.ndst; k += blockDim.x) {
        int i = k / a.ndst, t = k % a.ndst;
        uint32_t h = a.hat_mod[(size_t)i * a.nmod + a.dst_mod[t]];
        if (t < a.scale_lt) {
            const uint32_t q = a.dm.q[t];
            const uint2 u = a.s1[a.dst_mod[t]];
            h = mul_shoup(h, u.x, u.y, q);
            if (a.s2) {
                const uint2 v = a.s2[a.dst_mod[t]];
                h = mul_shoup(h, v.x, v.y, q);
            }
        }
        s_hat[k] = mul_shoup(h, a.dm.r32[t], a.dm.r32s[t], a.dm.q[t]);
    }
}

// VW consecutive words of p starting at word VW * i (VW = 2 or 4), loaded and stored as one
// 8- or 16-byte access.
template <int VW, bool COH>
__device__ __forceinline__ void ldv(const uint32_t* p, size_t i, uint32_t (&o)[VW]) {
    if constexpr (VW == 4) {
        const uint4 v = ld4<COH>(p, i);
        o[0] = v.x, o[1] = v.y, o[2] = v.z, o[3] = v.w;
    } else {
        static_assert(VW == 2, "VW is 2 or 4");
        uint2 v;
        if constexpr (COH)
            v = __ldcg(reinterpret_cast<const uint2*>(p) + i);
        else
            v = __ldg(reinterpret_cast<const uint2*>(p) + i);
        o[0] = v.x, o[1] = v.y;
    }
}
template <int VW>
__device__ __forceinline__ void stv(uint32_t* p, size_t i, const uint32_t (&v)[VW]) {
    if constexpr (VW == 4)
        reinterpret_cast<uint4*>(p)[i] = make_uint4(v[0], v[1], v[2], v[3]);
    else
        reinterpret_cast<uint2*>(p)[i] = make_uint2(v[0], v[1]);
}

// NS = number of source limbs (a compile-time constant so no issue slot is spent on
// predicated-off source terms); VW-word groups [n, end) of every limb (VW = 4 in the
// stand-alone kernel; 2 in the persistent kernel, whose register budget is half as large).
template <int NS, bool COH, int VW = 4>
__device__ __forceinline__ void conv_range(const ConvArgs& a, const uint32_t* s_hat, size_t n, size_t end,
                                           size_t step) {
    static_assert(NS >= 1 && NS <= 15, "the 64-bit sums hold at most 15 products below 2^60");
    for (; n < end; n += step) {
        uint32_t y[NS][VW];
#pragma unroll
        for (int i = 0; i < NS; ++i) {
            uint32_t x[VW];
            ldv<VW, COH>(a.src, i * (a.src_stride / VW) + n, x);
            const uint32_t b = a.src_q[i];
            const uint2 h = a.hat_inv[i];
#pragma unroll
            for (int k = 0; k < VW; ++k) y[i][k] = mul_shoup(x[k], h.x, h.y, b);
        }
        for (int t = 0; t < a.ndst; ++t) {
            uint64_t acc[VW];
#pragma unroll
            for (int k = 0; k < VW; ++k) acc[k] = 0;
#pragma unroll
            for (int i = 0; i < NS; ++i) {
                const uint64_t h = s_hat[i * a.ndst + t];
#pragma unroll
                for (int k = 0; k < VW; ++k) acc[k] += (uint64_t)y[i][k] * h;
            }
            // acc < NS 2^30 q_t (y_i < 2^30, constants below q_t), so its high word is below
            // NS q_t / 4: the Montgomery step leaves [0, 4 q_t) (for NS > 12 with its guard)
            uint32_t r[VW];
            const uint32_t q = a.dm.q[t], qinv = a.dm.qinv[t];
#pragma unroll
            for (int k = 0; k < VW; ++k) r[k] = csub(csub(redc<(NS > 12)>(acc[k], q, qinv), 2 * q), q);
            stv<VW>(a.dst, t * (a.dst_stride / VW) + n, r);
        }
    }
}

// ---- KS-4: inner product with the evaluation key (Hada-Mult + Ele-Add), all slices at once:
//   ks_c[t] = sum_j d~_j[t] * evk_{j,c}[t],  d~_j[t] = d2[t] on slice j's own limbs, else the
//   NTT of slice j's ModUp output. One pass reads every slice and writes ks0, ks1 once.
struct IpArgs {
    const uint32_t* d2;   // (nl, B, N) NTT domain
    const uint32_t* tmp;  // (dnum, ext, B, N): slice j's converted limbs at j*ext (q limbs outside the slice, then P)
    const uint32_t* evk;  // (dnum_ctx, 2, nmod, N)
    uint32_t* ks;         // (2, ext, B, N)
    int nl, alpha, dnum, ext, nq, nmod;
    size_t L4, N4;        // residues per limb / 4, N / 4
    ModVec m;             // per extended limb t < ext
    // per extended limb t: 2^32 s_t mod q_t with its Shoup quotient, the factor each sum takes
    // after its Montgomery step (which leaves it times 2^-32); s_t = P^-1 q_l^-1 on the limbs the
    // fused HMULT tail scales, P^-1 on those of a fused ModDown combine, else 1 (ip_set_post)
    uint2 post[kMaxLimbs];
};

// The post factors of an inner product over ext extended limbs whose first nl are q limbs,
// with P^-1 on limbs t < scale_lt, times q_l^-1 (l = nl - 1) for the fused HMULT tail (with_ql).
inline void ip_set_post(const fhe_ctx* ctx, IpArgs& ia, int nl, int ext, int scale_lt, bool with_ql) {
    for (int t = 0; t < ext; ++t) {
        const uint32_t q = ia.m.q[t];
        uint32_t c = (uint32_t)((1ull << 32) % q);
        if (t < scale_lt) {
            c = mulmod_h(c, ctx->p_inv_h[t].x, q);
            if (with_ql) c = mulmod_h(c, invmod_h(ctx->mods[nl - 1] % q, q), q);
        }
        ia.post[t] = make_uint2(c, shoup_h(c, q));
    }
}

// DN > 0: the slice count as a compile-time constant, so the slice loop unrolls and every
// slice's loads can issue before the first product; 0: a.dnum, a runtime loop.
template <bool COH, int DN = 0>
__device__ __forceinline__ void ip_range(const IpArgs& a, int t, size_t i, size_t end, size_t step) {
    const int dnum = DN > 0 ? DN : a.dnum;
    const Red rd = red_of(a.m, t);
    const uint32_t q = a.m.q[t], qinv = a.m.qinv[t];
    const uint2 post = a.post[t];
    const int mod = t < a.nl ? t : a.nq + (t - a.nl);
    const size_t limb = a.L4 * 4;
    uint32_t* k0 = a.ks + (size_t)t * limb;
    uint32_t* k1 = a.ks + (size_t)(a.ext + t) * limb;
    for (; i < end; i += step) {
        const size_t n4 = i % a.N4;
        // products < 2^60: up to 15 of them accumulate exactly in 64 bits, then one reduction
        uint64_t r0[4] = {0, 0, 0, 0}, r1[4] = {0, 0, 0, 0};
#pragma unroll
        for (int j = 0; j < dnum; ++j) {
            if (j > 0 && j % 15 == 0) {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    r0[k] = reduce_red(r0[k], rd);
                    r1[k] = reduce_red(r1[k], rd);
                }
            }
            const int lo = j * a.alpha, hi = min(a.nl, lo + a.alpha);
            const uint32_t* src = (t >= lo && t < hi)
                                      ? a.d2 + (size_t)t * limb
                                      : a.tmp + ((size_t)j * a.ext + (t < lo ? t : t - (hi - lo))) * limb;
            const uint4 x = ld4<COH>(src, i);
            const uint4 w0 = ld4(a.evk + ((size_t)(j * 2 + 0) * a.nmod + mod) * a.N4 * 4, n4);
            const uint4 w1 = ld4(a.evk + ((size_t)(j * 2 + 1) * a.nmod + mod) * a.N4 * 4, n4);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                r0[k] += (uint64_t)get(x, k) * get(w0, k);
                r1[k] += (uint64_t)get(x, k) * get(w1, k);
            }
        }
        // one Montgomery step per sum (guarded: the sums of more than 12 slices could pass
        // 2^32 with q added unconditionally), then the post factor, whose lazy Shoup product
        // takes any word: 14 FMA-pipe cycles per warp and sum instead of 14 plus 16 for the
        // 64-bit reduction and the two scaling products
        uint4 o0, o1;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            set(o0, k, csub(mul_shoup_lazy(redc<true>(r0[k], q, qinv), post.x, post.y, q), q));
            set(o1, k, csub(mul_shoup_lazy(redc<true>(r1[k], q, qinv), post.x, post.y, q), q));
        }
        st4(k0, i, o0);
        st4(k1, i, o1);
    }
}

// ---- the last limb of the fused HMULT tail (see hmult_fused in ckks.cu), component c:
//   relin_last: last = ks_l P^-1 + d_l (NTT domain, without the ModDown term y);
//   last_fix:   last = INTT(last) - y_l P^-1 mod q_l (coefficient domain).
struct LastArgs {
    const uint32_t* d;   // (2, nl, B, N)
    const uint32_t* ks;  // (2, ext, B, N)
    const uint32_t* y;   // (2, nl, B, N)
    uint32_t* last;      // (2, B, N)
    uint2 pinv;          // [P^-1]_{q_l} with its Shoup quotient
    uint32_t q;          // q_l
    int nl, ext;
    size_t L4;
};

template <bool COH>
__device__ __forceinline__ void relin_last_range(const LastArgs& a, int c, size_t n, size_t end, size_t step) {
    const int l = a.nl - 1;
    const uint32_t* dp = a.d + ((size_t)c * a.nl + l) * a.L4 * 4;
    const uint32_t* kp = a.ks + ((size_t)c * a.ext + l) * a.L4 * 4;
    uint32_t* op = a.last + (size_t)c * a.L4 * 4;
    for (; n < end; n += step) {
        uint4 dv = ld4<COH>(dp, n), kv = ld4<COH>(kp, n), r;
#pragma unroll
        for (int k = 0; k < 4; ++k) set(r, k, csub(mul_shoup(get(kv, k), a.pinv.x, a.pinv.y, a.q) + get(dv, k), a.q));
        st4(op, n, r);
    }
}

template <bool COH>
__device__ __forceinline__ void last_fix_range(const LastArgs& a, int c, size_t n, size_t end, size_t step) {
    const int l = a.nl - 1;
    const uint32_t* yp = a.y + ((size_t)c * a.nl + l) * a.L4 * 4;
    uint32_t* op = a.last + (size_t)c * a.L4 * 4;
    for (; n < end; n += step) {
        uint4 yv = ld4<COH>(yp, n), lv = ld4<COH>(op, n), r;
#pragma unroll
        for (int k = 0; k < 4; ++k)
            set(r, k, csub(get(lv, k) + a.q - mul_shoup(get(yv, k), a.pinv.x, a.pinv.y, a.q), a.q));
        st4(op, n, r);
    }
}

}  // namespace
}  // namespace fhe

// CKKS HMULT pipeline on the GPU: tensor product, generalized key switching (Dcomp/ModUp,
// inner product, ModDown) and RESCALE, composed from the kernels named in Sec. IV-A
// (Hada-Mult, Ele-Add, Ele-Sub, Conv, NTT).
//
// Every elementwise / basis-conversion stage is a coalesced, 16-byte vectorised stream over
// the (L, B, N) layout of Sec. IV-D: grid.y is the limb (so the modulus is uniform per block)
// and grid.x strides over the B*N residues of that limb.
#include <algorithm>

#include "ckks_kernels.cuh"

namespace fhe {
namespace {

// ---- HM-1: tensor product (tensor_range in ckks_kernels.cuh), one limb per grid row
__global__ void k_tensor(const TensorArgs t) {
    tensor_range(t, blockIdx.y, blockIdx.x * (size_t)blockDim.x + threadIdx.x, t.L4, (size_t)gridDim.x * blockDim.x);
}

// ---- KS-2 / KS-5: Conv (conv_range in ckks_kernels.cuh)
template <int NS>
__global__ void __launch_bounds__(256) k_conv(const ConvArgs a) {
    extern __shared__ uint32_t s_hat[];  // [nsrc][ndst]
    conv_load_hat(a, NS, s_hat);
    __syncthreads();
    conv_range<NS, false>(a, s_hat, blockIdx.x * (size_t)blockDim.x + threadIdx.x, a.L4, (size_t)gridDim.x * blockDim.x);
}

int launch_conv(const ConvArgs& ca, dim3 grid, size_t smem, cudaStream_t st) {
    switch (ca.nsrc) {
#define FHE_CONV_CASE(K) \
    case K: k_conv<K><<<grid, 256, smem, st>>>(ca); break;
        FHE_CONV_CASE(1) FHE_CONV_CASE(2) FHE_CONV_CASE(3) FHE_CONV_CASE(4) FHE_CONV_CASE(5)
        FHE_CONV_CASE(6) FHE_CONV_CASE(7) FHE_CONV_CASE(8) FHE_CONV_CASE(9) FHE_CONV_CASE(10)
        FHE_CONV_CASE(11) FHE_CONV_CASE(12) FHE_CONV_CASE(13) FHE_CONV_CASE(14) FHE_CONV_CASE(15)
#undef FHE_CONV_CASE
        default: return set_error(FHE_EINVAL, "Conv source count out of [1, 15]");
    }
    FHE_CUDA_TRY(cudaGetLastError());
    return FHE_OK;
}

// The context's basis-conversion kernel: tensor cores (conv_tc.cu) or the CUDA-core k_conv.
int run_conv(const fhe_ctx* ctx, const ConvArgs& ca, const ConvTable& ct, dim3 grid, size_t smem, cudaStream_t st) {
    if (ctx->conv_path == FHE_CONV_TC && ct.bdig && ca.ndst <= 64 && ca.scale_lt == 0) {
        TcConvArgs t;
        memset(&t, 0, sizeof(t));
        t.src = ca.src;
        t.src_stride = ca.src_stride;
        t.nsrc = ca.nsrc;
        for (int i = 0; i < ca.nsrc; ++i) {
            t.src_q[i] = ca.src_q[i];
            t.hat_inv[i] = ca.hat_inv[i];
        }
        t.bdig = ct.bdig;
        t.dst = ca.dst;
        t.dst_stride = ca.dst_stride;
        t.ndst = ca.ndst;
        for (int d = 0; d < ca.ndst; ++d) {
            t.dst_mod[d] = ca.dst_mod[d];
            t.dst_q[d] = ca.dm.q[d];
        }
        t.ncoef = ca.L4 * 4;
        return launch_conv_tc(ctx, t, st);
    }
    return launch_conv(ca, grid, smem, st);
}

// ---- KS-4: inner product with the evaluation key (ip_range in ckks_kernels.cuh). It waits on
// memory. With the slice count fixed at compile time (1 to 4) the slice loop unrolls, so every
// slice's loads issue before the first product, at five CTAs per SM (at most 48 registers, no
// spill). Larger counts spill when unrolled and take the loop as it is, at eight CTAs per SM
// (32 registers).
template <int DN>
__global__ void __launch_bounds__(256, DN > 0 ? 5 : 8) k_inner_product(const IpArgs a) {
    ip_range<false, DN>(a, blockIdx.y, blockIdx.x * (size_t)blockDim.x + threadIdx.x, a.L4,
                        (size_t)gridDim.x * blockDim.x);
}

int launch_inner_product(const IpArgs& ia, dim3 g, cudaStream_t st) {
    switch (ia.dnum) {
        case 1: k_inner_product<1><<<g, 256, 0, st>>>(ia); break;
        case 2: k_inner_product<2><<<g, 256, 0, st>>>(ia); break;
        case 3: k_inner_product<3><<<g, 256, 0, st>>>(ia); break;
        case 4: k_inner_product<4><<<g, 256, 0, st>>>(ia); break;
        default: k_inner_product<0><<<g, 256, 0, st>>>(ia); break;
    }
    FHE_CUDA_TRY(cudaGetLastError());
    return FHE_OK;
}

// ---- KS-5 tail + HM-2: out_c[i] (+)= (ks_c[i] - y_c[i]) * [P^-1]_{q_i}
__global__ void k_moddown_combine(const uint32_t* __restrict__ ks, const uint32_t* __restrict__ y,
                                  uint32_t* __restrict__ out, const uint2* __restrict__ pinv, int nl,
                                  int ext, int accumulate, size_t L4, ModVec m) {
    const int c = blockIdx.y / nl, i = blockIdx.y % nl;
    const uint32_t q = m.q[i];
    const uint2 pi = __ldg(&pinv[i]);
    const uint32_t* kp = ks + ((size_t)c * ext + i) * L4 * 4;
    const uint32_t* yp = y + ((size_t)c * nl + i) * L4 * 4;
    uint32_t* op = out + ((size_t)c * nl + i) * L4 * 4;
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < L4; n += (size_t)gridDim.x * blockDim.x) {
        uint4 kv = ld4(kp, n), yv = ld4(yp, n);
        uint4 ov = accumulate ? ld4(op, n) : make_uint4(0, 0, 0, 0);
        uint4 r;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint32_t d = get(kv, k) + q - get(yv, k);                 // [1, 2q)
            uint32_t v = mul_shoup(d, pi.x, pi.y, q) + get(ov, k);    // [0, 2q)
            set(r, k, csub(v, q));
        }
        st4(op, n, r);
    }
}

// ---- RS-1: gather the last limb of both components
__global__ void k_copy_limb(const uint32_t* __restrict__ ct, uint32_t* __restrict__ out, int nl, size_t L4) {
    const int c = blockIdx.y;
    const uint32_t* src = ct + ((size_t)c * nl + (nl - 1)) * L4 * 4;
    uint32_t* dst = out + (size_t)c * L4 * 4;
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < L4; n += (size_t)gridDim.x * blockDim.x)
        st4(dst, n, ld4(src, n));
}

// x in [0, q_l) -> centred value (x - q_l if x > (q_l - 1)/2) reduced mod q_i, for i < nl - 1
__global__ void k_rescale_broadcast(const uint32_t* __restrict__ last, uint32_t* __restrict__ xb,
                                    uint32_t ql, int nout, size_t L4, ModVec m) {
    const int c = blockIdx.y / nout, i = blockIdx.y % nout;
    const uint32_t q = m.q[i];
    const uint32_t* src = last + (size_t)c * L4 * 4;
    uint32_t* dst = xb + ((size_t)c * nout + i) * L4 * 4;
    const uint32_t half = (ql - 1) / 2;
    const uint32_t ql_mod = ql % q;
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < L4; n += (size_t)gridDim.x * blockDim.x) {
        uint4 x = ld4(src, n), r;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint32_t v = get(x, k);
            // v <= half: v mod q;  v > half: (v - ql) mod q = (v mod q) - (ql mod q) mod q
            uint32_t vm = reduce32(v, red_of(m, i));
            uint32_t o = v > half ? (vm + q - ql_mod) : vm;
            set(r, k, csub(o, q));
        }
        st4(dst, n, r);
    }
}

// out_c[i] = (ct_c[i] - xb_c[i]) * [q_l^-1]_{q_i}
__global__ void k_rescale_final(const uint32_t* __restrict__ ct, const uint32_t* __restrict__ xb,
                                uint32_t* __restrict__ out, const uint2* __restrict__ qlinv, int nl,
                                size_t L4, ModVec m) {
    const int nout = nl - 1;
    const int c = blockIdx.y / nout, i = blockIdx.y % nout;
    const uint32_t q = m.q[i];
    const uint2 w = __ldg(&qlinv[i]);
    const uint32_t* cp = ct + ((size_t)c * nl + i) * L4 * 4;
    const uint32_t* xp = xb + ((size_t)c * nout + i) * L4 * 4;
    uint32_t* op = out + ((size_t)c * nout + i) * L4 * 4;
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < L4; n += (size_t)gridDim.x * blockDim.x) {
        uint4 cv = ld4(cp, n), xv = ld4(xp, n), r;
#pragma unroll
        for (int k = 0; k < 4; ++k) set(r, k, mul_shoup(get(cv, k) + q - get(xv, k), w.x, w.y, q));
        st4(op, n, r);
    }
}

// ---- HMULT tail, fused (the ModDown combine folded into RESCALE): the relinearised result
// d_c + (ks_c - y_c) P^-1 is formed only for the last limb l = nl - 1 (it feeds the rescale's
// INTT) and, for the other limbs, inside the rescale's final step, so the relinearised
// ciphertext is never written out. With rel_i = (ks_i - y^_i) P^-1 + d_i the relinearised
// limb i (NTT domain) and x_i the centred last limb broadcast to q_i,
// the output is (rel_i - x^_i) q_l^-1 = (ks_i P^-1 + d_i - NTT(y_i P^-1 + x_i)) q_l^-1 by the
// linearity of the NTT mod q_i, so one forward NTT of z_i = y_i P^-1 + x_i replaces the NTTs
// of y (ModDown) and of x (RESCALE). The constant factors are applied where they cost no
// extra pass: for i < l the tensor product writes d'_i = d_i q_l^-1, the inner product
// ks'_i = ks_i P^-1 q_l^-1 and ModDown's Conv y'_i = y_i P^-1 q_l^-1, so with
// z'_i = y'_i + x_i q_l^-1 the output is ks'_i + d'_i - NTT(z'_i), additions only.
//
// u = ks_l P^-1 + d_l, the last limb of both components without the y term (NTT domain), and
// last = INTT(u) - y_l P^-1 mod q_l: the last relinearised limb in the coefficient domain
// (relin_last_range / last_fix_range in ckks_kernels.cuh).
__global__ void k_relin_last(const LastArgs a) {
    relin_last_range<false>(a, blockIdx.y, blockIdx.x * (size_t)blockDim.x + threadIdx.x, a.L4,
                            (size_t)gridDim.x * blockDim.x);
}

__global__ void k_last_fix(const LastArgs a) {
    last_fix_range<false>(a, blockIdx.y, blockIdx.x * (size_t)blockDim.x + threadIdx.x, a.L4,
                          (size_t)gridDim.x * blockDim.x);
}

// z'_i = y'_i + [last]_centred q_l^-1 mod q_i (coefficient domain), i < l.
__global__ void k_rescale_prep(const uint32_t* __restrict__ last, const uint32_t* __restrict__ y,
                               uint32_t* __restrict__ z, const uint2* __restrict__ qlinv, uint32_t ql, int nl,
                               size_t L4, ModVec m) {
    const int nout = nl - 1;
    const int c = blockIdx.y / nout, i = blockIdx.y % nout;
    const uint32_t q = m.q[i];
    const uint2 qi = __ldg(&qlinv[i]);
    const uint32_t* lp = last + (size_t)c * L4 * 4;
    const uint32_t* yp = y + ((size_t)c * nl + i) * L4 * 4;
    uint32_t* zp = z + ((size_t)c * nout + i) * L4 * 4;
    const uint32_t half = (ql - 1) / 2;
    const uint32_t ql_mod = ql % q;
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < L4; n += (size_t)gridDim.x * blockDim.x) {
        uint4 lv = ld4(lp, n), yv = ld4(yp, n), r;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t v = get(lv, k);
            const uint32_t vm = reduce32(v, red_of(m, i));
            const uint32_t x = csub(v > half ? (vm + q - ql_mod) : vm, q);  // (v - ql) mod q above half
            set(r, k, csub(get(yv, k) + mul_shoup(x, qi.x, qi.y, q), q));
        }
        st4(zp, n, r);
    }
}

// out_i = ks'_i + d'_i - z'^_i, i < l, where ks'_i = ks_i P^-1 q_l^-1 and d'_i = d_i q_l^-1 were
// scaled when they were written and z'^ is the NTT of z'.
__global__ void k_hmult_final(const uint32_t* __restrict__ d, const uint32_t* __restrict__ ks,
                              const uint32_t* __restrict__ zh, uint32_t* __restrict__ out, int nl, int ext,
                              size_t L4, ModVec m) {
    const int nout = nl - 1;
    const int c = blockIdx.y / nout, i = blockIdx.y % nout;
    const uint32_t q = m.q[i];
    const size_t limb = L4 * 4;
    const uint32_t* dp = d + ((size_t)c * nl + i) * limb;
    const uint32_t* kp = ks + ((size_t)c * ext + i) * limb;
    const uint32_t* zp = zh + ((size_t)c * nout + i) * limb;
    uint32_t* op = out + ((size_t)c * nout + i) * limb;
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < L4; n += (size_t)gridDim.x * blockDim.x) {
        uint4 dv = ld4(dp, n), kv = ld4(kp, n), zv = ld4(zp, n), r;
#pragma unroll
        for (int k = 0; k < 4; ++k) set(r, k, csub(csub(get(kv, k) + get(dv, k), q) + q - get(zv, k), q));
        st4(op, n, r);
    }
}

// ------------------------------------------------------------------ host orchestration

dim3 stream_grid(const fhe_ctx* ctx, size_t L4, int limbs) {
    // enough blocks per limb to cover ~4 waves of the GPU across all limbs
    size_t want = (size_t)ctx->num_sms * 8 * 4 / (size_t)std::max(1, limbs) + 1;
    size_t need = (L4 + 255) / 256;
    size_t gx = std::min(want, need);
    if (gx < 1) gx = 1;
    return dim3((unsigned)gx, (unsigned)limbs, 1);
}

struct Sizes {
    size_t N, limb;  // residues per limb (B * N)
    int nl, K, ext;
};

size_t ks_scratch_limbs(int nl, int K, int alpha) {
    // d2c (nl) + ModUp outputs (dnum slices of nl + K) + ks (2 (nl + K)) + y (2 nl)
    const size_t dnum = (size_t)((nl + alpha - 1) / alpha);
    return (size_t)nl + dnum * (nl + K) + 2 * (size_t)(nl + K) + 2 * (size_t)nl;
}

// KS-1..KS-3: INTT into d2c (nl limbs: of src when given, else of d2c in place; NTT form in)
// and, per slice j, Conv
// Q_j -> (Q_l \ Q_j) u P and the NTT of the converted limbs into `digits` (dnum, ext, B, N):
// slice j's converted limbs at j * ext, the q limbs outside the slice first, then P.
int ks_modup(const fhe_ctx* ctx, uint32_t logN, int nl, int batch, uint32_t* d2c, uint32_t* digits,
             cudaStream_t st, NttScratch ns, const uint32_t* src = nullptr) {
    const size_t N = 1ull << logN, limb = N * batch, L4 = limb / 4;
    const int K = ctx->np, ext = nl + K, alpha = ctx->alpha, nq = ctx->nq;
    const int nmod = (int)ctx->mods.size();
    const int dnum = (nl + alpha - 1) / alpha;
    int rc;
    // KS-1: INTT(d2)
    if (src)
        rc = ntt_inv_from(ctx, logN, d2c, src, nl, batch, contiguous_map(ctx, 0, nl), st, ns);
    else
        rc = ntt_any(ctx, FHE_NTT_DEFAULT, logN, true, d2c, nl, batch, contiguous_map(ctx, 0, nl), st, ns);
    if (rc) return rc;
    for (int j = 0; j < dnum; ++j) {
        const int lo = j * alpha, hi = std::min(nl, (j + 1) * alpha);
        uint32_t* tmp = digits + (size_t)j * ext * limb;
        const ConvTable& ct = ctx->modup[j][hi - lo - 1];
        // KS-2: Conv Q_j -> (Q_l \ Q_j) u P
        ConvArgs ca;
        ca.s1 = ca.s2 = nullptr;
        ca.scale_lt = 0;
        ca.src = d2c + (size_t)lo * limb;
        ca.src_stride = limb;
        ca.nsrc = hi - lo;
        for (int i = 0; i < ca.nsrc; ++i) {
            ca.src_q[i] = ctx->mods[lo + i];
            ca.hat_inv[i] = ct.hat_inv_h[i];
        }
        ca.hat_mod = ct.hat_mod;
        ca.nmod = nmod;
        ca.dst = tmp;
        ca.dst_stride = limb;
        int dmod[kMaxLimbs];
        int nd = 0;
        for (int t = 0; t < nl; ++t)
            if (t < lo || t >= hi) dmod[nd++] = t;
        for (int k = 0; k < K; ++k) dmod[nd++] = nq + k;
        ca.ndst = nd;
        for (int t = 0; t < nd; ++t) ca.dst_mod[t] = (uint8_t)dmod[t];
        ca.dm = modvec(ctx, dmod, nd);
        ca.L4 = L4;
        size_t smem = (size_t)ca.nsrc * nd * 4;
        dim3 g = stream_grid(ctx, L4, 1);
        g.x = std::min<unsigned>(g.x * 4, (unsigned)((L4 + 255) / 256));
        if ((rc = run_conv(ctx, ca, ct, g, smem, st))) return rc;
        // KS-3: NTT of the converted limbs
        LimbMap lm;
        for (int t = 0; t < nd; ++t) {
            lm.mod[t] = (uint8_t)dmod[t];
            lm.q[t] = ctx->mods[dmod[t]];
        }
        if ((rc = ntt_any(ctx, FHE_NTT_DEFAULT, logN, false, tmp, nd, batch, lm, st, ns))) return rc;
    }
    return FHE_OK;
}

int launch_automorph(const fhe_ctx* ctx, const uint32_t* in, uint32_t* out, uint32_t k, uint32_t logN, size_t rows,
                     cudaStream_t st);

// KS-4, KS-5: the inner product of the ModUp digits with evk (slice j's own limbs taken from d2,
// NTT form) and ModDown into `out` (2, nl, B, N); accumulate != 0 adds to out. ks (2 ext limbs)
// and y (2 nl limbs) are scratch. scale_lt > 0 (the fused HMULT + RESCALE tail, out == nullptr):
// q limbs t < scale_lt of ks and of y come out multiplied by P^-1 q_{nl-1}^-1.
// galois != 0 (hoisted rotations): the inner product writes ks_pre (2 ext limbs), whose
// automorphism X -> X^galois then becomes ks; with evk permuted by the inverse automorphism this
// equals the inner product of the permuted digits with evk, since the product is pointwise.
int ks_finish(const fhe_ctx* ctx, uint32_t logN, int nl, int batch, const uint32_t* d2, const uint32_t* digits,
              const uint32_t* evk, uint32_t* out, int accumulate, uint32_t* ks, uint32_t* y, cudaStream_t st,
              NttScratch ns, int scale_lt, uint32_t galois = 0, uint32_t* ks_pre = nullptr) {
    const size_t N = 1ull << logN, limb = N * batch, L4 = limb / 4;
    const int K = ctx->np, ext = nl + K, alpha = ctx->alpha, nq = ctx->nq;
    const int nmod = (int)ctx->mods.size();
    const int dnum = (nl + alpha - 1) / alpha;
    int ext_mod[kMaxLimbs];
    for (int t = 0; t < ext; ++t) ext_mod[t] = t < nl ? t : nq + (t - nl);
    ModVec ext_m = modvec(ctx, ext_mod, ext);
    int rc;
    // The combine out += (ks - NTT(y)) P^-1 can ride on the forward NTT of y, as the HMULT's
    // RESCALE tail does (z' = y' loaded, out = ks' + out - z'^ stored): the inner product then
    // writes ks' = ks P^-1 on the q limbs and ModDown's Conv y' = y P^-1, so that neither NTT(y)
    // nor a separate combine pass reaches HBM.
    const bool fuse_combine = out != nullptr && accumulate && scale_lt == 0 &&
                              ntt_tail_fusable(ctx, FHE_NTT_DEFAULT, logN);
    const int ip_scale = fuse_combine ? nl : scale_lt;
    // KS-4: inner product over all slices
    {
        IpArgs ia;
        ia.d2 = d2;
        ia.tmp = digits;
        ia.evk = evk;
        ia.ks = galois ? ks_pre : ks;
        ia.nl = nl;
        ia.alpha = alpha;
        ia.dnum = dnum;
        ia.ext = ext;
        ia.nq = nq;
        ia.nmod = nmod;
        ia.L4 = L4;
        ia.N4 = N / 4;
        ia.m = ext_m;
        ip_set_post(ctx, ia, nl, ext, ip_scale, !fuse_combine);
        if ((rc = launch_inner_product(ia, stream_grid(ctx, L4, ext), st))) return rc;
        if (galois && (rc = launch_automorph(ctx, ks_pre, ks, galois, logN, 2 * (size_t)ext * batch, st))) return rc;
    }
    // KS-5: ModDown of ks0, ks1
    LimbMap pm = contiguous_map(ctx, nq, K);
    for (int c = 0; c < 2; ++c)
        if ((rc = ntt_any(ctx, FHE_NTT_DEFAULT, logN, true, ks + ((size_t)c * ext + nl) * limb, K, batch, pm, st, ns)))
            return rc;
    for (int c = 0; c < 2; ++c) {
        ConvArgs ca;
        ca.s1 = ctx->p_inv;
        ca.s2 = scale_lt > 0 ? ctx->ql_inv + (size_t)(nl - 1) * nq : nullptr;
        ca.scale_lt = ip_scale;
        ca.src = ks + ((size_t)c * ext + nl) * limb;
        ca.src_stride = limb;
        ca.nsrc = K;
        for (int k = 0; k < K; ++k) {
            ca.src_q[k] = ctx->mods[nq + k];
            ca.hat_inv[k] = ctx->moddown.hat_inv_h[k];
        }
        ca.hat_mod = ctx->moddown.hat_mod;
        ca.nmod = nmod;
        ca.dst = y + (size_t)c * nl * limb;
        ca.dst_stride = limb;
        ca.ndst = nl;
        int dmod[kMaxLimbs];
        for (int t = 0; t < nl; ++t) {
            dmod[t] = t;
            ca.dst_mod[t] = (uint8_t)t;
        }
        ca.dm = modvec(ctx, dmod, nl);
        ca.L4 = L4;
        dim3 g = stream_grid(ctx, L4, 1);
        g.x = std::min<unsigned>(g.x * 4, (unsigned)((L4 + 255) / 256));
        if ((rc = run_conv(ctx, ca, ctx->moddown, g, (size_t)K * nl * 4, st))) return rc;
    }
    if (2 * nl > kMaxLimbs) return set_error(FHE_EINVAL, "too many limbs");
    LimbMap qm2;
    for (int c = 0; c < 2; ++c)
        for (int i = 0; i < nl && i < FHE_MAX_MODULI; ++i) {
            qm2.mod[c * nl + i] = (uint8_t)i;
            qm2.q[c * nl + i] = ctx->mods[i];
        }
    // the caller fuses the ModDown combine into RESCALE and takes y in the coefficient domain
    if (out == nullptr) return FHE_OK;
    if (fuse_combine) {
        HmultTail tl;
        tl.y = y;
        tl.last = nullptr;
        tl.ks = ks;
        tl.d = out;
        tl.out = out;
        tl.qlinv = nullptr;
        tl.ql = 0;
        tl.nl = nl;
        tl.nout = nl;
        tl.ext = ext;
        return ntt_u32_l2_tail(ctx, logN, 2 * nl * batch, batch, qm2, st, ns, tl);
    }
    if ((rc = ntt_any(ctx, FHE_NTT_DEFAULT, logN, false, y, 2 * nl, batch, qm2, st, ns))) return rc;
    int qidx[kMaxLimbs];
    for (int i = 0; i < nl; ++i) qidx[i] = i;
    k_moddown_combine<<<stream_grid(ctx, L4, 2 * nl), 256, 0, st>>>(ks, y, out, ctx->p_inv, nl, ext, accumulate,
                                                                  L4, modvec(ctx, qidx, nl));
    FHE_CUDA_TRY(cudaGetLastError());
    return FHE_OK;
}

// Key switching of d2 (NTT form) into `out` (2, nl, B, N); accumulate != 0 adds to out.
// d2c (nl limbs of scratch) may already hold a copy of d2 when d2c_ready != 0; otherwise the
// INTT reads d2 itself (or a copy of it, where the inverse cannot run out of place).
// scale_lt > 0 (the fused HMULT + RESCALE tail, out == nullptr): q limbs t < scale_lt of ks and
// of y come out multiplied by P^-1 q_{nl-1}^-1, the factors the tail would otherwise apply.
// Scratch: d2c (nl limbs), ModUp digits (dnum (nl + K)), ks (2 (nl + K)), y (2 nl).
int keyswitch_impl(const fhe_ctx* ctx, uint32_t logN, int nl, int batch, const uint32_t* d2,
                   const uint32_t* evk, uint32_t* out, int accumulate, uint32_t* scratch,
                   bool d2c_ready, cudaStream_t st, NttScratch ns, int scale_lt = 0) {
    const size_t limb = ((size_t)1 << logN) * batch;
    const int ext = nl + ctx->np;
    const int dnum = (nl + ctx->alpha - 1) / ctx->alpha;
    uint32_t* d2c = scratch;
    uint32_t* tmp_all = d2c + (size_t)nl * limb;
    uint32_t* ks = tmp_all + (size_t)dnum * ext * limb;
    uint32_t* y = ks + 2 * (size_t)ext * limb;
    int rc;
    if ((rc = ks_modup(ctx, logN, nl, batch, d2c, tmp_all, st, ns, d2c_ready ? nullptr : d2))) return rc;
    return ks_finish(ctx, logN, nl, batch, d2, tmp_all, evk, out, accumulate, ks, y, st, ns, scale_lt);
}

size_t rescale_scratch_limbs(int nl) { return 2 + 2 * (size_t)(nl - 1); }

// RESCALE needs no extra NTT region: the INTT of the last limb chunks through the (still
// unused) broadcast buffer, and the NTT of the broadcast through the last-limb buffer once
// the broadcast has consumed it.
int rescale_impl(const fhe_ctx* ctx, uint32_t logN, int nl, int batch, const uint32_t* ct, uint32_t* out,
                 uint32_t* scratch, cudaStream_t st) {
    const size_t N = 1ull << logN, limb = N * batch, L4 = limb / 4;
    const int nout = nl - 1;
    uint32_t* last = scratch;
    uint32_t* xb = last + 2 * limb;
    NttScratch ns_last, ns_xb;
    ns_last.p = xb;
    ns_last.bytes = 2 * (size_t)nout * limb * 4;
    ns_xb.p = last;
    ns_xb.bytes = 2 * limb * 4;
    int rc;
    k_copy_limb<<<stream_grid(ctx, L4, 2), 256, 0, st>>>(ct, last, nl, L4);
    FHE_CUDA_TRY(cudaGetLastError());
    LimbMap lm;
    lm.mod[0] = lm.mod[1] = (uint8_t)(nl - 1);
    lm.q[0] = lm.q[1] = ctx->mods[nl - 1];
    if ((rc = ntt_any(ctx, FHE_NTT_DEFAULT, logN, true, last, 2, batch, lm, st, ns_last))) return rc;
    int qidx[kMaxLimbs];
    for (int i = 0; i < nout; ++i) qidx[i] = i;
    ModVec qm = modvec(ctx, qidx, nout);
    k_rescale_broadcast<<<stream_grid(ctx, L4, 2 * nout), 256, 0, st>>>(last, xb, ctx->mods[nl - 1], nout, L4, qm);
    FHE_CUDA_TRY(cudaGetLastError());
    if (2 * nout > kMaxLimbs) return set_error(FHE_EINVAL, "too many limbs");
    LimbMap qm2;
    for (int c = 0; c < 2; ++c)
        for (int i = 0; i < nout && i < FHE_MAX_MODULI; ++i) {
            qm2.mod[c * nout + i] = (uint8_t)i;
            qm2.q[c * nout + i] = ctx->mods[i];
        }
    if ((rc = ntt_any(ctx, FHE_NTT_DEFAULT, logN, false, xb, 2 * nout, batch, qm2, st, ns_xb))) return rc;
    k_rescale_final<<<stream_grid(ctx, L4, 2 * nout), 256, 0, st>>>(ct, xb, out, ctx->ql_inv + (size_t)(nl - 1) * ctx->nq,
                                                                   nl, L4, qm);
    FHE_CUDA_TRY(cudaGetLastError());
    return FHE_OK;
}

int hmult_relin_impl(const fhe_ctx* ctx, uint32_t logN, int nl, int batch, const uint32_t* a, const uint32_t* b,
                     const uint32_t* evk, uint32_t* out, uint32_t* scratch, cudaStream_t st, NttScratch ns) {
    const size_t N = 1ull << logN, limb = N * batch, L4 = limb / 4;
    uint32_t* d2 = scratch;
    uint32_t* ks_scratch = d2 + (size_t)nl * limb;  // begins with d2c
    int qidx[kMaxLimbs];
    for (int i = 0; i < nl; ++i) qidx[i] = i;
    // the tensor product writes the copy of d2 that the INTT transforms in place, unless the
    // INTT can read d2 itself
    const bool oop = ntt_inv_out_of_place(ctx, logN);
    k_tensor<<<stream_grid(ctx, L4, nl), 256, 0, st>>>(TensorArgs{a, b, out, out + (size_t)nl * limb, d2,
                                                                oop ? nullptr : ks_scratch,
                                                                L4, (size_t)nl * L4, modvec(ctx, qidx, nl), nullptr, 0});
    FHE_CUDA_TRY(cudaGetLastError());
    return keyswitch_impl(ctx, logN, nl, batch, d2, evk, out, 1, ks_scratch, !oop, st, ns);
}

// HMULT + RESCALE with the fused tail (k_relin_last .. k_hmult_final above): one forward NTT of
// 2 (nl - 1) limbs after key switching instead of ModDown's 2 nl and RESCALE's 2 (nl - 1).
// Scratch: relin-d (2 nl limbs: d0, d1), d2 (nl), then the key-switching scratch (d2c, ModUp
// outputs, ks, y); after the inner product the d2c / ModUp region is reused for the last limb
// and z (2 + 2 (nl - 1) limbs, which fit: nl + dnum (nl + K) >= 2 nl).
int hmult_fused(const fhe_ctx* ctx, uint32_t logN, int nl, int batch, const uint32_t* a, const uint32_t* b,
                const uint32_t* evk, uint32_t* out, uint32_t* scratch, cudaStream_t st, NttScratch ns) {
    const size_t N = 1ull << logN, limb = N * batch, L4 = limb / 4;
    const int K = ctx->np, ext = nl + K, alpha = ctx->alpha;
    const int dnum = (nl + alpha - 1) / alpha;
    uint32_t* dd = scratch;                       // (2, nl): d0, d1
    uint32_t* d2 = dd + 2 * (size_t)nl * limb;    // (nl)
    uint32_t* ksx = d2 + (size_t)nl * limb;       // key-switching scratch, begins with d2c
    uint32_t* ks = ksx + ((size_t)nl + (size_t)dnum * ext) * limb;
    uint32_t* y = ks + 2 * (size_t)ext * limb;
    uint32_t* last = ksx;                         // reuses d2c / ModUp space
    uint32_t* xb = last + 2 * limb;
    int qidx[kMaxLimbs];
    for (int i = 0; i < nl; ++i) qidx[i] = i;
    // the limbs i < l of d0, d1, ks and y carry the tail's factors from the start: q_l^-1 on d,
    // P^-1 q_l^-1 on ks and y (folded into HBM-bound passes and into Conv's constants), so that
    // the combine below needs no multiplication
    const uint2* qlinv = ctx->ql_inv + (size_t)(nl - 1) * ctx->nq;
    const bool oop = ntt_inv_out_of_place(ctx, logN);  // else the tensor product also writes d2c
    k_tensor<<<stream_grid(ctx, L4, nl), 256, 0, st>>>(TensorArgs{a, b, dd, dd + (size_t)nl * limb, d2,
                                                                oop ? nullptr : ksx, L4, (size_t)nl * L4,
                                                                modvec(ctx, qidx, nl), qlinv, nl - 1});
    FHE_CUDA_TRY(cudaGetLastError());
    int rc = keyswitch_impl(ctx, logN, nl, batch, d2, evk, nullptr, 0, ksx, !oop, st, ns, nl - 1);
    if (rc) return rc;
    const uint32_t ql = ctx->mods[nl - 1];
    const uint2 pinv_l = ctx->p_inv_h[nl - 1];
    const LastArgs la{dd, ks, y, last, pinv_l, ql, nl, ext, L4};
    k_relin_last<<<stream_grid(ctx, L4, 2), 256, 0, st>>>(la);
    FHE_CUDA_TRY(cudaGetLastError());
    LimbMap lm;
    lm.mod[0] = lm.mod[1] = (uint8_t)(nl - 1);
    lm.q[0] = lm.q[1] = ql;
    if ((rc = ntt_any(ctx, FHE_NTT_DEFAULT, logN, true, last, 2, batch, lm, st, ns))) return rc;
    k_last_fix<<<stream_grid(ctx, L4, 2), 256, 0, st>>>(la);
    FHE_CUDA_TRY(cudaGetLastError());
    const int nout = nl - 1;
    LimbMap qm2;
    for (int c = 0; c < 2; ++c)
        for (int i = 0; i < nout && i < FHE_MAX_MODULI; ++i) {
            qm2.mod[c * nout + i] = (uint8_t)i;
            qm2.q[c * nout + i] = ctx->mods[i];
        }
    if (ntt_tail_fusable(ctx, FHE_NTT_DEFAULT, logN)) {
        // z is built while the forward NTT loads it and the output combined while it stores
        // z^: the same arithmetic as k_rescale_prep / k_hmult_final without their HBM passes
        HmultTail tl;
        tl.y = y;
        tl.last = last;
        tl.ks = ks;
        tl.d = dd;
        tl.out = out;
        tl.qlinv = qlinv;
        tl.ql = ql;
        tl.nl = nl;
        tl.nout = nout;
        tl.ext = ext;
        return ntt_u32_l2_tail(ctx, logN, 2 * nout * batch, batch, qm2, st, ns, tl);
    }
    ModVec qm = modvec(ctx, qidx, nout);
    k_rescale_prep<<<stream_grid(ctx, L4, 2 * nout), 256, 0, st>>>(last, y, xb, qlinv, ql, nl, L4, qm);
    FHE_CUDA_TRY(cudaGetLastError());
    if ((rc = ntt_any(ctx, FHE_NTT_DEFAULT, logN, false, xb, 2 * nout, batch, qm2, st, ns))) return rc;
    k_hmult_final<<<stream_grid(ctx, L4, 2 * nout), 256, 0, st>>>(dd, ks, xb, out, nl, ext, L4, qm);
    FHE_CUDA_TRY(cudaGetLastError());
    return FHE_OK;
}

// ---- FrobeniusMap (X -> X^k, k odd) in the NTT domain, where it only permutes: Eq. (4)
// evaluates at psi^(2j+1), and a(X^k) at psi^(2j+1) is a at psi^((2j+1) k), so output j takes
// input j' with 2j' + 1 = (2j + 1) k mod 2N. The product is taken mod 2^32, a multiple of
// 2N, so its wrap-around does not change it mod 2N. Rows are independent of the modulus.
__global__ void k_automorph(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, uint32_t k, int logN,
                            size_t rows) {
    const uint32_t N = 1u << logN, mask = 2 * N - 1;
    for (size_t r = blockIdx.y; r < rows; r += gridDim.y) {
        const uint32_t* src = in + (r << logN);
        uint32_t* dst = out + (r << logN);
        for (uint32_t j4 = blockIdx.x * blockDim.x + threadIdx.x; j4 < N / 4; j4 += gridDim.x * blockDim.x) {
            uint4 v;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const uint32_t j = 4 * j4 + kk;
                set(v, kk, __ldg(&src[(((2 * j + 1) * k) & mask) >> 1]));
            }
            st4(dst, j4, v);
        }
    }
}

// One CTA per 1024 outputs of a row (each thread one uint4), the CTAs of a row adjacent in
// launch order: the rows in flight at once (about 19 at N = 2^16) then hold a few MB, so the
// stride-k gather of each row is served from L2. With one CTA walking a whole row, some 1200
// rows of 256 KB would be in flight, far above the 129 MB of L2, and gathered sectors would be
// fetched from DRAM several times.
int launch_automorph(const fhe_ctx* ctx, const uint32_t* in, uint32_t* out, uint32_t k, uint32_t logN, size_t rows,
                     cudaStream_t st) {
    (void)ctx;
    if (rows == 0) return FHE_OK;
    const size_t L4 = ((size_t)1 << logN) / 4;
    const dim3 g((unsigned)((L4 + 255) / 256), (unsigned)std::min<size_t>(rows, 65535), 1);
    k_automorph<<<g, 256, 0, st>>>(in, out, k, (int)logN, rows);
    FHE_CUDA_TRY(cudaGetLastError());
    return FHE_OK;
}

// ---- CMULT (Hada-Mult of both components by a plaintext) and HADD (Ele-Add), NTT domain.
__global__ void k_cmult(const uint32_t* __restrict__ ct, const uint32_t* __restrict__ pt, uint32_t* __restrict__ out,
                        size_t L4, size_t comp4, ModVec m) {
    const int l = blockIdx.y;
    const Red rd = red_of(m, l);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < L4; i += (size_t)gridDim.x * blockDim.x) {
        const size_t idx = (size_t)l * L4 + i;
        const uint4 p = ld4(pt, idx), c0 = ld4(ct, idx), c1 = ld4(ct, comp4 + idx);
        uint4 r0, r1;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            set(r0, k, reduce_red((uint64_t)get(c0, k) * get(p, k), rd));
            set(r1, k, reduce_red((uint64_t)get(c1, k) * get(p, k), rd));
        }
        st4(out, idx, r0);
        st4(out, comp4 + idx, r1);
    }
}

__global__ void k_hadd(const uint32_t* __restrict__ a, const uint32_t* __restrict__ b, uint32_t* __restrict__ out,
                       size_t L4, size_t comp4, ModVec m) {
    const int l = blockIdx.y % (gridDim.y / 2), c = blockIdx.y / (gridDim.y / 2);
    const uint32_t q = m.q[l];
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < L4; i += (size_t)gridDim.x * blockDim.x) {
        const size_t idx = c * comp4 + (size_t)l * L4 + i;
        const uint4 x = ld4(a, idx), y = ld4(b, idx);
        uint4 r;
#pragma unroll
        for (int k = 0; k < 4; ++k) set(r, k, csub(get(x, k) + get(y, k), q));
        st4(out, idx, r);
    }
}

// HROTATE / conjugation: out = (c0(X^k) + ks0, ks1), (ks0, ks1) = KeySwitch(c1(X^k)) under the
// key from s(X^k) to s. Scratch: c1(X^k) (nl limbs), then the key-switching scratch.
size_t hrotate_scratch_limbs(int nl, int K, int alpha) { return (size_t)nl + ks_scratch_limbs(nl, K, alpha); }

int hrotate_impl(const fhe_ctx* ctx, uint32_t logN, int nl, int batch, uint32_t k, const uint32_t* ct,
                 const uint32_t* ksk, uint32_t* out, uint32_t* scratch, cudaStream_t st, NttScratch ns) {
    const size_t limb = ((size_t)1 << logN) * batch, rows = (size_t)nl * batch;
    uint32_t* c1k = scratch;
    int rc;
    if ((rc = launch_automorph(ctx, ct, out, k, logN, rows, st))) return rc;
    if ((rc = launch_automorph(ctx, ct + (size_t)nl * limb, c1k, k, logN, rows, st))) return rc;
    FHE_CUDA_TRY(cudaMemsetAsync(out + (size_t)nl * limb, 0, (size_t)nl * limb * 4, st));
    return keyswitch_impl(ctx, logN, nl, batch, c1k, ksk, out, 1, c1k + (size_t)nl * limb, false, st, ns);
}

// Hoisted HROTATE: n_rot rotations of one ciphertext share one ModUp. The NTT-domain digits
// ModUp_j(c1) are formed once; each rotation's key switch is that of the digits permuted by
// the automorphism X -> X^k (a permutation of NTT-domain values, the same under every
// modulus). Since the inner product is pointwise, sum_j d_j[sigma(n)] evk_j[n] is ks'[sigma(n)]
// with ks'[m] = sum_j d_j[m] evk_j[sigma^-1(m)]: each rotation permutes its key by the inverse
// automorphism (once, shared by the whole batch), takes the inner product of the unpermuted
// digits and c1 (the own-slice limbs), and permutes the 2 (nl + K) limbs of ks' instead of the
// nl + dnum (nl + K) - nl limbs of c1 and the digits; c0 is permuted into the output, and
// ModDown finishes as in hrotate_impl. The approximate Conv does not commute exactly with
// X -> X^k (where a coefficient is negated, its lift changes by a multiple of Q_j), so this is
// a valid key switch of c1(X^k) that differs from hrotate_impl's result.
// Scratch: c1 (coefficients; nl limbs), digits (dnum ext), ks' (2 ext), ks (2 ext), y (2 nl),
// then the permuted key (dnum x 2 x nmod rows of N words, in whole limbs of the batch).
size_t hoisted_key_limbs(const fhe_ctx* ctx, int nl, int batch) {
    const size_t dnum = (size_t)((nl + ctx->alpha - 1) / ctx->alpha);
    const size_t rows = dnum * 2 * ctx->mods.size();
    return batch > 0 ? (rows + batch - 1) / batch : 0;
}
size_t hoisted_scratch_limbs(const fhe_ctx* ctx, int nl, int batch) {
    const size_t dnum = (size_t)((nl + ctx->alpha - 1) / ctx->alpha), ext = (size_t)(nl + ctx->np);
    return (size_t)nl + dnum * ext + 4 * ext + 2 * (size_t)nl + hoisted_key_limbs(ctx, nl, batch);
}

// The inverse of an odd k modulo 2^bits (bits <= 32), by Newton's iteration.
uint32_t inv_pow2(uint32_t k, int bits) {
    uint32_t x = k;
    for (int i = 0; i < 5; ++i) x *= 2u - k * x;
    return bits >= 32 ? x : x & ((1u << bits) - 1);
}

int hrotate_hoisted_impl(const fhe_ctx* ctx, uint32_t logN, int nl, int batch, int nrot, const uint32_t* galois,
                         const uint32_t* ct, const uint32_t* const* ksk, uint32_t* out, uint32_t* scratch,
                         cudaStream_t st, NttScratch ns) {
    const size_t N = (size_t)1 << logN, limb = N * batch, rows = (size_t)nl * batch;
    const int ext = nl + ctx->np, alpha = ctx->alpha, dnum = (nl + alpha - 1) / alpha;
    const uint32_t* c1 = ct + (size_t)nl * limb;
    uint32_t* c1c = scratch;
    uint32_t* digits = c1c + (size_t)nl * limb;
    uint32_t* kp = digits + (size_t)dnum * ext * limb;
    uint32_t* ks = kp + 2 * (size_t)ext * limb;
    uint32_t* y = ks + 2 * (size_t)ext * limb;
    uint32_t* key = y + 2 * (size_t)nl * limb;
    const size_t key_rows = (size_t)dnum * 2 * ctx->mods.size();
    int rc;
    if ((rc = ks_modup(ctx, logN, nl, batch, c1c, digits, st, ns, c1))) return rc;
    for (int r = 0; r < nrot; ++r) {
        const uint32_t k = galois[r];
        uint32_t* o = out + (size_t)r * 2 * nl * limb;
        if ((rc = launch_automorph(ctx, ksk[r], key, inv_pow2(k, (int)logN + 1), logN, key_rows, st))) return rc;
        if ((rc = launch_automorph(ctx, ct, o, k, logN, rows, st))) return rc;
        FHE_CUDA_TRY(cudaMemsetAsync(o + (size_t)nl * limb, 0, (size_t)nl * limb * 4, st));
        if ((rc = ks_finish(ctx, logN, nl, batch, c1, digits, key, o, 1, ks, y, st, ns, 0, k, kp))) return rc;
    }
    return FHE_OK;
}

bool al16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

int check_ckks(const fhe_ctx* ctx, uint32_t logN, int nl, int batch, int min_nl) {
    FHE_CHECK(ctx != nullptr, "ctx is NULL");
    FHE_CHECK(ctx->np > 0, "context has no special primes");
    FHE_CHECK(logN >= FHE_LOGN_MIN && logN <= ctx->logN_max, "logN out of [10, logN_max]");
    FHE_CHECK(nl >= min_nl && nl <= ctx->nq, "n_limbs out of range");
    FHE_CHECK(batch >= 0, "batch < 0");
    return FHE_OK;
}

int check_ptrs(std::initializer_list<const void*> ps) {
    for (const void* p : ps) FHE_CHECK(p != nullptr && al16(p), "pointer NULL or not 16-byte aligned");
    return FHE_OK;
}

// Rows of the largest NTT call an operation makes, per ciphertext of the batch.
// RESCALE chunks through its own buffers (rescale_impl) and needs none.
size_t ntt_rows(const fhe_ctx* ctx, int op, int nl) { return op == FHE_OP_RESCALE ? 0 : 2 * ((size_t)nl + ctx->np); }

size_t scratch_limbs(const fhe_ctx* ctx, int op, int nl, int batch) {
    const int K = ctx->np;
    switch (op) {
        case FHE_OP_KEYSWITCH: return ks_scratch_limbs(nl, K, ctx->alpha);
        case FHE_OP_HMULT_RELIN: return (size_t)nl + ks_scratch_limbs(nl, K, ctx->alpha);
        case FHE_OP_RESCALE: return rescale_scratch_limbs(nl);
        case FHE_OP_HMULT: return 2 * (size_t)nl + (size_t)nl + ks_scratch_limbs(nl, K, ctx->alpha);
        case FHE_OP_HROTATE: return hrotate_scratch_limbs(nl, K, ctx->alpha);
        case FHE_OP_HROTATE_HOISTED: return hoisted_scratch_limbs(ctx, nl, batch);
        default: return 0;
    }
}

// The two-pass NTT region of an operation's caller scratch (after the operation's limbs).
NttScratch op_ntt_scratch(const fhe_ctx* ctx, int op, uint32_t logN, int nl, int batch, void* scratch) {
    NttScratch s;
    s.bytes = op_region_bytes(ctx, logN, ntt_rows(ctx, op, nl) * batch);
    if (s.bytes) s.p = (uint32_t*)((uint8_t*)scratch + scratch_limbs(ctx, op, nl, batch) * ((size_t)batch << logN) * 4);
    return s;
}

}  // namespace
}  // namespace fhe

using namespace fhe;

extern "C" {

size_t fhe_scratch_bytes(const fhe_ctx* ctx, int op, uint32_t logN, int n_limbs, int batch) {
    if (!ctx || ctx->np == 0 || logN < FHE_LOGN_MIN || logN > ctx->logN_max || n_limbs < 1 ||
        n_limbs > ctx->nq || batch < 0)
        return 0;
    if ((op == FHE_OP_RESCALE || op == FHE_OP_HMULT) && n_limbs < 2) return 0;
    const size_t limbs = scratch_limbs(ctx, op, n_limbs, batch);
    if (limbs == 0) return 0;
    // the operation's limbs, then the two-pass NTT region of its NTT calls
    return limbs * ((size_t)batch << logN) * 4 + op_region_bytes(ctx, logN, ntt_rows(ctx, op, n_limbs) * batch);
}

int fhe_keyswitch(const fhe_ctx* ctx, uint32_t logN, int n_limbs, int batch, const uint32_t* d2,
                  const uint32_t* evk, uint32_t* ks_out, void* scratch, size_t scratch_bytes, void* stream) {
    int rc = check_ckks(ctx, logN, n_limbs, batch, 1);
    if (rc || batch == 0) return rc;
    if ((rc = check_ptrs({d2, evk, ks_out, scratch}))) return rc;
    if (scratch_bytes < fhe_scratch_bytes(ctx, FHE_OP_KEYSWITCH, logN, n_limbs, batch))
        return set_error(FHE_ENOMEM, "scratch too small");
    return keyswitch_impl(ctx, logN, n_limbs, batch, d2, evk, ks_out, 0, (uint32_t*)scratch, false,
                          (cudaStream_t)stream, op_ntt_scratch(ctx, FHE_OP_KEYSWITCH, logN, n_limbs, batch, scratch));
}

int fhe_hmult_relin(const fhe_ctx* ctx, uint32_t logN, int n_limbs, int batch, const uint32_t* ct_a,
                    const uint32_t* ct_b, const uint32_t* evk, uint32_t* out, void* scratch,
                    size_t scratch_bytes, void* stream) {
    int rc = check_ckks(ctx, logN, n_limbs, batch, 1);
    if (rc || batch == 0) return rc;
    if ((rc = check_ptrs({ct_a, ct_b, evk, out, scratch}))) return rc;
    if (scratch_bytes < fhe_scratch_bytes(ctx, FHE_OP_HMULT_RELIN, logN, n_limbs, batch))
        return set_error(FHE_ENOMEM, "scratch too small");
    return hmult_relin_impl(ctx, logN, n_limbs, batch, ct_a, ct_b, evk, out, (uint32_t*)scratch,
                            (cudaStream_t)stream,
                            op_ntt_scratch(ctx, FHE_OP_HMULT_RELIN, logN, n_limbs, batch, scratch));
}

int fhe_rescale(const fhe_ctx* ctx, uint32_t logN, int n_limbs, int batch, const uint32_t* ct_in,
                uint32_t* ct_out, void* scratch, size_t scratch_bytes, void* stream) {
    int rc = check_ckks(ctx, logN, n_limbs, batch, 2);
    if (rc || batch == 0) return rc;
    if ((rc = check_ptrs({ct_in, ct_out, scratch}))) return rc;
    if (scratch_bytes < fhe_scratch_bytes(ctx, FHE_OP_RESCALE, logN, n_limbs, batch))
        return set_error(FHE_ENOMEM, "scratch too small");
    return rescale_impl(ctx, logN, n_limbs, batch, ct_in, ct_out, (uint32_t*)scratch, (cudaStream_t)stream);
}

int fhe_hmult(const fhe_ctx* ctx, uint32_t logN, int n_limbs, int batch, const uint32_t* ct_a,
              const uint32_t* ct_b, const uint32_t* evk, uint32_t* ct_out, void* scratch,
              size_t scratch_bytes, void* stream) {
    int rc = check_ckks(ctx, logN, n_limbs, batch, 2);
    if (rc || batch == 0) return rc;
    if ((rc = check_ptrs({ct_a, ct_b, evk, ct_out, scratch}))) return rc;
    if (scratch_bytes < fhe_scratch_bytes(ctx, FHE_OP_HMULT, logN, n_limbs, batch))
        return set_error(FHE_ENOMEM, "scratch too small");
    return hmult_fused(ctx, logN, n_limbs, batch, ct_a, ct_b, evk, ct_out, (uint32_t*)scratch, (cudaStream_t)stream,
                       op_ntt_scratch(ctx, FHE_OP_HMULT, logN, n_limbs, batch, scratch));
}

int fhe_automorph(const fhe_ctx* ctx, uint32_t logN, long long rows, uint32_t galois, const uint32_t* in,
                  uint32_t* out, void* stream) {
    FHE_CHECK(ctx != nullptr, "ctx is NULL");
    FHE_CHECK(logN >= FHE_LOGN_MIN && logN <= ctx->logN_max, "logN out of [10, logN_max]");
    FHE_CHECK(rows >= 0, "rows < 0");
    FHE_CHECK((galois & 1u) == 1u && galois < (2u << logN), "galois element must be odd and below 2N");
    if (rows == 0) return FHE_OK;
    int rc = check_ptrs({in, out});
    if (rc) return rc;
    FHE_CHECK(in != out, "fhe_automorph cannot run in place");
    return launch_automorph(ctx, in, out, galois, logN, (size_t)rows, (cudaStream_t)stream);
}

int fhe_hrotate(const fhe_ctx* ctx, uint32_t logN, int n_limbs, int batch, uint32_t galois, const uint32_t* ct_in,
                const uint32_t* ksk, uint32_t* ct_out, void* scratch, size_t scratch_bytes, void* stream) {
    int rc = check_ckks(ctx, logN, n_limbs, batch, 1);
    if (rc || batch == 0) return rc;
    FHE_CHECK((galois & 1u) == 1u && galois < (2u << logN), "galois element must be odd and below 2N");
    if ((rc = check_ptrs({ct_in, ksk, ct_out, scratch}))) return rc;
    FHE_CHECK(ct_in != ct_out, "fhe_hrotate cannot run in place");
    if (scratch_bytes < fhe_scratch_bytes(ctx, FHE_OP_HROTATE, logN, n_limbs, batch))
        return set_error(FHE_ENOMEM, "scratch too small");
    return hrotate_impl(ctx, logN, n_limbs, batch, galois, ct_in, ksk, ct_out, (uint32_t*)scratch,
                        (cudaStream_t)stream, op_ntt_scratch(ctx, FHE_OP_HROTATE, logN, n_limbs, batch, scratch));
}

int fhe_hrotate_hoisted(const fhe_ctx* ctx, uint32_t logN, int n_limbs, int batch, int n_rot, const uint32_t* galois,
                        const uint32_t* ct_in, const uint32_t* const* ksk, uint32_t* ct_out, void* scratch,
                        size_t scratch_bytes, void* stream) {
    int rc = check_ckks(ctx, logN, n_limbs, batch, 1);
    if (rc) return rc;
    FHE_CHECK(n_rot >= 0, "n_rot < 0");
    if (batch == 0 || n_rot == 0) return FHE_OK;
    FHE_CHECK(galois != nullptr && ksk != nullptr, "galois or ksk array is NULL");
    for (int r = 0; r < n_rot; ++r) {
        FHE_CHECK((galois[r] & 1u) == 1u && galois[r] < (2u << logN), "galois element must be odd and below 2N");
        if ((rc = check_ptrs({ksk[r]}))) return rc;
    }
    if ((rc = check_ptrs({ct_in, ct_out, scratch}))) return rc;
    const uintptr_t in0 = (uintptr_t)ct_in, out0 = (uintptr_t)ct_out;
    const size_t ct_bytes = 2 * (size_t)n_limbs * ((size_t)batch << logN) * 4;
    FHE_CHECK(out0 + (size_t)n_rot * ct_bytes <= in0 || in0 + ct_bytes <= out0, "ct_out overlaps ct_in");
    if (scratch_bytes < fhe_scratch_bytes(ctx, FHE_OP_HROTATE_HOISTED, logN, n_limbs, batch))
        return set_error(FHE_ENOMEM, "scratch too small");
    return hrotate_hoisted_impl(ctx, logN, n_limbs, batch, n_rot, galois, ct_in, ksk, ct_out, (uint32_t*)scratch,
                                (cudaStream_t)stream,
                                op_ntt_scratch(ctx, FHE_OP_HROTATE_HOISTED, logN, n_limbs, batch, scratch));
}

int fhe_cmult(const fhe_ctx* ctx, uint32_t logN, int n_limbs, int batch, const uint32_t* ct, const uint32_t* pt,
              uint32_t* ct_out, void* stream) {
    FHE_CHECK(ctx != nullptr, "ctx is NULL");
    FHE_CHECK(logN >= FHE_LOGN_MIN && logN <= ctx->logN_max, "logN out of [10, logN_max]");
    FHE_CHECK(n_limbs >= 1 && n_limbs <= ctx->nq, "n_limbs out of range");
    FHE_CHECK(batch >= 0, "batch < 0");
    if (batch == 0) return FHE_OK;
    int rc = check_ptrs({ct, pt, ct_out});
    if (rc) return rc;
    const size_t L4 = ((size_t)batch << logN) / 4;
    int qidx[kMaxLimbs];
    for (int i = 0; i < n_limbs; ++i) qidx[i] = i;
    k_cmult<<<stream_grid(ctx, L4, n_limbs), 256, 0, (cudaStream_t)stream>>>(ct, pt, ct_out, L4, (size_t)n_limbs * L4,
                                                                           modvec(ctx, qidx, n_limbs));
    FHE_CUDA_TRY(cudaGetLastError());
    return FHE_OK;
}

int fhe_hadd(const fhe_ctx* ctx, uint32_t logN, int n_limbs, int batch, const uint32_t* ct_a, const uint32_t* ct_b,
             uint32_t* ct_out, void* stream) {
    FHE_CHECK(ctx != nullptr, "ctx is NULL");
    FHE_CHECK(logN >= FHE_LOGN_MIN && logN <= ctx->logN_max, "logN out of [10, logN_max]");
    FHE_CHECK(n_limbs >= 1 && n_limbs <= ctx->nq, "n_limbs out of range");
    FHE_CHECK(batch >= 0, "batch < 0");
    if (batch == 0) return FHE_OK;
    int rc = check_ptrs({ct_a, ct_b, ct_out});
    if (rc) return rc;
    const size_t L4 = ((size_t)batch << logN) / 4;
    int qidx[kMaxLimbs];
    for (int i = 0; i < n_limbs; ++i) qidx[i] = i;
    k_hadd<<<stream_grid(ctx, L4, 2 * n_limbs), 256, 0, (cudaStream_t)stream>>>(ct_a, ct_b, ct_out, L4,
                                                                              (size_t)n_limbs * L4,
                                                                              modvec(ctx, qidx, n_limbs));
    FHE_CUDA_TRY(cudaGetLastError());
    return FHE_OK;
}

}  // extern "C"

// Plain 32-bit NTT for N >= 2^15 in two passes through L2 (no thread-block clusters).
//
// The merged Cooley-Tukey transform of ntt_u32.cu is split at the quarter boundary
// (C = N / 2^14 quarters of NC = 2^14 residues, or 2 x 2^13 .. per kernel shape):
//   forward: cross pass  -- the first log2(C) stages couple the C quarters of a row; a
//                           streaming kernel applies them and writes the row to a scratch
//                           buffer sized to stay in L2;
//            quarter pass -- every quarter finishes its remaining stages in one CTA (the same
//                           register/shared-memory rounds as the single-CTA kernel) and stores
//                           its outputs k = k_local * C + rev(c) back into the row (in place:
//                           the cross pass has already read the whole chunk);
//   inverse: the same two passes in reverse order (quarter pass from the row into scratch,
//            cross pass from scratch back into the row, with the N^-1 scaling).
// Rows are processed in chunks whose scratch fits in L2, so the intermediate never reaches
// HBM: each residue is read and written in HBM once, as in the cluster kernels, but every CTA
// is independent and all SMs are usable.
#include "common.cuh"
#include "ptx.cuh"

namespace fhe {
namespace {

struct L2Args {
    uint32_t* data;      // LimbMap mode: row r at data + r * N
    int batch;
    const RowRef* rowtab;  // row-table mode
    const uint32_t* mod_q;
    uint32_t* temp;      // chunk scratch: row r0 + i at temp + i * N
    int r0, nrows;       // rows of this chunk
    const uint2* tw;     // [nmod][N]
    const uint2* twC;    // [nmod][C][31][T]
    const uint2* ninv;   // [nmod]
    LimbMap map;
};

template <int N>
__device__ __forceinline__ uint32_t* l2_row(const L2Args& a, int row, uint32_t* q, int* mod) {
    if (a.rowtab) {
        const RowRef r = a.rowtab[row];
        *mod = (int)r.mod;
        *q = __ldg(&a.mod_q[r.mod]);
        return r.ptr;
    }
    const int limb = row / a.batch;
    *q = a.map.q[limb];
    *mod = a.map.mod[limb];
    return a.data + (size_t)row * N;
}

template <int BITS>
__device__ __forceinline__ uint32_t rbits(uint32_t x) {
    return __brev(x) >> (32 - BITS);
}
__device__ __forceinline__ void ct2(uint32_t& x, uint32_t& y, uint2 w, uint32_t q) {
    uint32_t x2 = csub(x, 2 * q);
    uint32_t t = mul_shoup_lazy(y, w.x, w.y, q);
    x = x2 + t;
    y = x2 - t + 2 * q;
}
__device__ __forceinline__ void gs2(uint32_t& x, uint32_t& y, uint2 w, uint32_t q) {
    uint32_t s = csub(x + y, 2 * q);
    uint32_t d = x - y + 2 * q;
    x = s;
    y = mul_shoup_lazy(d, w.x, w.y, q);
}

// ---- cross pass: grid (blocks over NC/4 quad positions, chunk rows); 4 positions per thread
template <int LOG_NC, int LOG_C, bool INV>
__global__ void __launch_bounds__(256) ntt_cross_kernel(const L2Args a) {
    constexpr int NC = 1 << LOG_NC, C = 1 << LOG_C, N = NC * C;
    const int i = blockIdx.y;
    uint32_t q;
    int mod;
    uint32_t* row = l2_row<N>(a, a.r0 + i, &q, &mod);
    uint32_t* tmp = a.temp + (size_t)i * N;
    const uint2* tw = a.tw + (size_t)mod * N;
    const uint32_t* src = INV ? tmp : row;
    uint32_t* dst = INV ? row : tmp;
    uint2 ni = make_uint2(0, 0);
    if (INV) ni = __ldg(&a.ninv[mod]);
    for (int p4 = blockIdx.x * blockDim.x + threadIdx.x; p4 < NC / 4; p4 += gridDim.x * blockDim.x) {
        uint4 x[C];
#pragma unroll
        for (int qq = 0; qq < C; ++qq) x[qq] = __ldg(reinterpret_cast<const uint4*>(src + qq * NC) + p4);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint32_t y[C];
#pragma unroll
            for (int qq = 0; qq < C; ++qq) y[qq] = k == 0 ? x[qq].x : k == 1 ? x[qq].y : k == 2 ? x[qq].z : x[qq].w;
            if (!INV) {
#pragma unroll
                for (int s = 0; s < LOG_C; ++s) {
                    const int tq = C >> (s + 1);
#pragma unroll
                    for (int qq = 0; qq < C; ++qq)
                        if ((qq / tq) % 2 == 0) ct2(y[qq], y[qq + tq], __ldg(&tw[(1 << s) + qq / (2 * tq)]), q);
                }
            } else {
#pragma unroll
                for (int s = LOG_C - 1; s >= 0; --s) {
                    const int tq = C >> (s + 1);
#pragma unroll
                    for (int qq = 0; qq < C; ++qq)
                        if ((qq / tq) % 2 == 0) gs2(y[qq], y[qq + tq], __ldg(&tw[(1 << s) + qq / (2 * tq)]), q);
                }
#pragma unroll
                for (int qq = 0; qq < C; ++qq) y[qq] = mul_shoup(y[qq], ni.x, ni.y, q);
            }
#pragma unroll
            for (int qq = 0; qq < C; ++qq) {
                if (k == 0) x[qq].x = y[qq];
                else if (k == 1) x[qq].y = y[qq];
                else if (k == 2) x[qq].z = y[qq];
                else x[qq].w = y[qq];
            }
        }
#pragma unroll
        for (int qq = 0; qq < C; ++qq) reinterpret_cast<uint4*>(dst + qq * NC)[p4] = x[qq];
    }
}

template <int LOG_T>
constexpr int kMinB = (1 << (14 - LOG_T)) / 32 > 0 ? (1 << (14 - LOG_T)) / 32 : 1;

// ---- quarter pass, forward: scratch quarter c -> remaining stages -> row (stride C)
template <int LOG_T, int LOG_C>
__global__ void __launch_bounds__(1 << LOG_T, kMinB<LOG_T>) ntt_quarter_fwd_kernel(const L2Args a) {
    constexpr int T = 1 << LOG_T, C = 1 << LOG_C, NC = 32 * T, N = NC * C, RB = LOG_T - 5;
    extern __shared__ __align__(128) uint32_t work[];
    const int tid = threadIdx.x, c = blockIdx.x, i = blockIdx.y;
    const int rc = rbits<LOG_C>(c);
    using L = PadLayout<LOG_T>;
    const int pA = L::pad(tid);
    uint32_t q;
    int mod;
    uint32_t* row = l2_row<N>(a, a.r0 + i, &q, &mod);
    const uint32_t* tmp = a.temp + (size_t)i * N + c * NC;
    const uint2* tw = a.tw + (size_t)mod * N;
    uint32_t v[32];
#pragma unroll
    for (int e = 0; e < 32; ++e) v[e] = __ldcg(&tmp[tid + T * e]);
    // round A
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const int half = 16 >> k;
#pragma unroll
        for (int e = 0; e < 32; ++e)
            if ((e & half) == 0) ct2(v[e], v[e + half], __ldg(&tw[(1 << k) * (C + c) + (e >> (5 - k))]), q);
    }
#pragma unroll
    for (int e = 0; e < 32; ++e) work[pA + L::kSA * e] = v[e];
    __syncthreads();
    // round B
    if constexpr (RB > 0) {
        constexpr int GPT = 32 >> RB, EG = 1 << RB;
        const int lane = tid & 31, w_ = tid >> 5;
#pragma unroll
        for (int gi = 0; gi < GPT; ++gi) {
            const int g = w_ * GPT + gi;
            uint32_t* vv = v + gi * EG;
#pragma unroll
            for (int e = 0; e < EG; ++e) vv[e] = work[g * L::kSA + lane + 33 * e];
#pragma unroll
            for (int k = 0; k < RB; ++k) {
                const int half = EG >> (k + 1);
#pragma unroll
                for (int e = 0; e < EG; ++e)
                    if ((e & half) == 0)
                        ct2(vv[e], vv[e + half], __ldg(&tw[(1 << k) * (32 * (C + c) + g) + (e >> (RB - k))]), q);
            }
#pragma unroll
            for (int e = 0; e < EG; ++e) work[g * L::kSA + lane + 33 * e] = vv[e];
        }
        __syncthreads();
    }
    // round C
    {
        const int gidx = rbits<LOG_T>(tid);
        const int pC = L::pad(32 * gidx);
#pragma unroll
        for (int e = 0; e < 32; ++e) v[e] = work[pC + e];
        const uint2* twc = a.twC + (((size_t)mod * C + c) * 31) * T + tid;
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const int half = 16 >> k;
#pragma unroll
            for (int e = 0; e < 32; ++e)
                if ((e & half) == 0) ct2(v[e], v[e + half], __ldg(&twc[(size_t)((1 << k) - 1 + (e >> (5 - k))) * T]), q);
        }
    }
#pragma unroll
    for (int e = 0; e < 32; ++e) row[(rbits<5>(e) * T + tid) * C + rc] = csub(csub(v[e], 2 * q), q);
}

// ---- quarter pass, inverse: row (stride C, quarter c's bit-reversed share) -> GS stages -> scratch
template <int LOG_T, int LOG_C>
__global__ void __launch_bounds__(1 << LOG_T, kMinB<LOG_T>) ntt_quarter_inv_kernel(const L2Args a) {
    constexpr int T = 1 << LOG_T, C = 1 << LOG_C, NC = 32 * T, N = NC * C, RB = LOG_T - 5;
    extern __shared__ __align__(128) uint32_t work[];
    const int tid = threadIdx.x, c = blockIdx.x, i = blockIdx.y;
    const int rc = rbits<LOG_C>(c);
    using L = PadLayout<LOG_T>;
    const int pA = L::pad(tid);
    uint32_t q;
    int mod;
    const uint32_t* row = l2_row<N>(a, a.r0 + i, &q, &mod);
    uint32_t* tmp = a.temp + (size_t)i * N + c * NC;
    const uint2* tw = a.tw + (size_t)mod * N;
    uint32_t v[32];
#pragma unroll
    for (int e = 0; e < 32; ++e) v[e] = __ldg(&row[(rbits<5>(e) * T + tid) * C + rc]);
    // round C'
    {
        const int gidx = rbits<LOG_T>(tid);
        const int pC = L::pad(32 * gidx);
        const uint2* twc = a.twC + (((size_t)mod * C + c) * 31) * T + tid;
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const int half = 1 << k, kf = 4 - k;
#pragma unroll
            for (int e = 0; e < 32; ++e)
                if ((e & half) == 0)
                    gs2(v[e], v[e + half], __ldg(&twc[(size_t)((1 << kf) - 1 + (e >> (5 - kf))) * T]), q);
        }
#pragma unroll
        for (int e = 0; e < 32; ++e) work[pC + e] = v[e];
        __syncthreads();
    }
    // round B'
    if constexpr (RB > 0) {
        constexpr int GPT = 32 >> RB, EG = 1 << RB;
        const int lane = tid & 31, w_ = tid >> 5;
#pragma unroll
        for (int gi = 0; gi < GPT; ++gi) {
            const int g = w_ * GPT + gi;
            uint32_t* vv = v + gi * EG;
#pragma unroll
            for (int e = 0; e < EG; ++e) vv[e] = work[g * L::kSA + lane + 33 * e];
#pragma unroll
            for (int k = RB - 1; k >= 0; --k) {
                const int half = EG >> (k + 1);
#pragma unroll
                for (int e = 0; e < EG; ++e)
                    if ((e & half) == 0)
                        gs2(vv[e], vv[e + half], __ldg(&tw[(1 << k) * (32 * (C + c) + g) + (e >> (RB - k))]), q);
            }
#pragma unroll
            for (int e = 0; e < EG; ++e) work[g * L::kSA + lane + 33 * e] = vv[e];
        }
        __syncthreads();
    }
    // round A'
#pragma unroll
    for (int e = 0; e < 32; ++e) v[e] = work[pA + L::kSA * e];
#pragma unroll
    for (int k = 4; k >= 0; --k) {
        const int half = 16 >> k;
#pragma unroll
        for (int e = 0; e < 32; ++e)
            if ((e & half) == 0) gs2(v[e], v[e + half], __ldg(&tw[(1 << k) * (C + c) + (e >> (5 - k))]), q);
    }
#pragma unroll
    for (int e = 0; e < 32; ++e) __stcg(&tmp[tid + T * e], v[e]);
}

template <int LOG_T, int LOG_C>
int run_l2(const fhe_ctx* ctx, const NttTables& t, int shape, bool inverse, uint32_t* d, int rows, int batch,
           const LimbMap& map, const RowRef* rowtab, cudaStream_t st) {
    constexpr int T = 1 << LOG_T, C = 1 << LOG_C, NC = 32 * T, N = NC * C;
    constexpr int smem = PadLayout<LOG_T>::kWords * 4;
    auto qk = inverse ? ntt_quarter_inv_kernel<LOG_T, LOG_C> : ntt_quarter_fwd_kernel<LOG_T, LOG_C>;
    auto xk = inverse ? ntt_cross_kernel<LOG_T + 5, LOG_C, true> : ntt_cross_kernel<LOG_T + 5, LOG_C, false>;
    FHE_CUDA_TRY(cudaFuncSetAttribute(qk, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    int carve = (int)((kMinB<LOG_T> * (smem + 1024) * 100 + 228 * 1024 - 1) / (228 * 1024));
    FHE_CUDA_TRY(cudaFuncSetAttribute(qk, cudaFuncAttributePreferredSharedMemoryCarveout, carve > 100 ? 100 : carve));
    L2Args a;
    a.data = d;
    a.batch = batch;
    a.rowtab = rowtab;
    a.mod_q = ctx->d_mods;
    a.temp = ctx->ntt_temp;
    a.tw = inverse ? t.inv : t.fwd;
    a.twC = inverse ? t.invC[shape] : t.fwdC[shape];
    a.ninv = t.ninv;
    a.map = map;
    const int chunk = (int)(kNttTempBytes / ((size_t)N * 4));
    const int gx = (NC / 4 + 255) / 256;
    for (int r0 = 0; r0 < rows; r0 += chunk) {
        a.r0 = r0;
        a.nrows = rows - r0 < chunk ? rows - r0 : chunk;
        if (!inverse) {
            xk<<<dim3(gx, a.nrows), 256, 0, st>>>(a);
            FHE_CUDA_TRY(cudaGetLastError());
        }
        qk<<<dim3(C, a.nrows), T, smem, st>>>(a);
        FHE_CUDA_TRY(cudaGetLastError());
        if (inverse) {
            xk<<<dim3(gx, a.nrows), 256, 0, st>>>(a);
            FHE_CUDA_TRY(cudaGetLastError());
        }
    }
    return FHE_OK;
}

}  // namespace

int ntt_u32_l2(const fhe_ctx* ctx, uint32_t logN, int shape, bool inverse, uint32_t* d, int rows, int batch,
               const LimbMap& map, const RowRef* rowtab, cudaStream_t st) {
    const NttTables& t = ctx->ntt[logN];
    if (!ctx->ntt_temp) return set_error(FHE_EINVAL, "no two-pass scratch in this context");
    int log_t, log_c;
    if (!ntt_variant_shape(logN, shape, &log_t, &log_c) || log_c == 0)
        return set_error(FHE_EINVAL, "two-pass NTT needs N >= 2^15");
    if (log_t == 9 && log_c == 2) return run_l2<9, 2>(ctx, t, shape, inverse, d, rows, batch, map, rowtab, st);
    if (log_t == 9 && log_c == 1) return run_l2<9, 1>(ctx, t, shape, inverse, d, rows, batch, map, rowtab, st);
    if (log_t == 8 && log_c == 3) return run_l2<8, 3>(ctx, t, shape, inverse, d, rows, batch, map, rowtab, st);
    if (log_t == 8 && log_c == 2) return run_l2<8, 2>(ctx, t, shape, inverse, d, rows, batch, map, rowtab, st);
    return set_error(FHE_EINVAL, "no two-pass kernel for this shape");
}

}  // namespace fhe

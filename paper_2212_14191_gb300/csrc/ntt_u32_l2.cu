// Plain 32-bit NTT for N >= 2^15 in two passes through L2 (no thread-block clusters).
//
// A row of N = C * NC residues (NC = 2^14, or 2^13 for the 256-thread shape) is transformed
// as C sub-transforms of NC points plus a C-point combination, in one launch per chunk of rows:
//   forward (decimation in time): local pass -- every CTA runs the single-CTA NC-point
//            transform (root psi^C, the library's root for that ring degree) on the
//            decimated sequence a[j + C m] and writes it in natural order to a scratch buffer;
//            cross pass -- twist B_j[k'] by psi^((2k'+1) j), C-point cyclic DFT, write
//            A[k' + NC t] back into the row;
//   inverse (decimation in frequency): quarter pass -- every CTA gathers the outputs
//            k = k_local * C + rev(c) of its quarter, runs the Gentleman-Sande stages of the
//            quarter and writes the scratch; cross pass -- the last log2(C) stages couple the
//            quarters and apply N^-1, writing the row.
// The cross pass of a row is run by whichever of its C CTAs finishes the local pass last
// (an atomic count per row, no waiting), so it reads the row's scratch from L2 and no second
// launch is needed. Every CTA is independent, all SMs are usable and no cluster barrier is
// involved. The strided side of both forms is a read (the C CTAs of a row share every sector
// through L2): stores stay contiguous. Rows go through in chunks of up to 1 GiB of scratch.
#include <algorithm>

#include "ntt_u32_l2.cuh"


namespace fhe {
namespace {

// Stand-alone cross passes, one launch after the local passes: used for chunks too small to
// fill the GPU, where the fused form would leave one CTA per row doing all of its cross work.
template <int LOG_NC, int LOG_C>
__global__ void __launch_bounds__(256) ntt_cross_inv_kernel(const L2Args a) {
    cross_inv_row<LOG_NC, LOG_C>(a, blockIdx.y, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

template <int LOG_T, int LOG_C>
__global__ void __launch_bounds__(1 << LOG_T, kMinB<LOG_T>) ntt_quarter_inv_kernel(const L2Args a) {
    quarter_inv<LOG_T, LOG_C, false>(a, blockIdx.y, blockIdx.x);
}

template <int LOG_NC, int LOG_C, bool TAIL>
__global__ void __launch_bounds__(256) ntt_dit_cross_kernel(const L2Args a) {
    dit_cross_row<LOG_NC, LOG_C, TAIL>(a, blockIdx.y, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

template <int LOG_T, int LOG_C, bool TAIL, bool LAST = true>
__global__ void __launch_bounds__(1 << LOG_T, kMinB<LOG_T>) ntt_dit_local_kernel(const L2Args a) {
    dit_local<LOG_T, LOG_C, TAIL, false, LAST>(a, blockIdx.y, blockIdx.x);
}


template <int LOG_T, int LOG_C, bool TAIL>
int run_l2(const fhe_ctx* ctx, const NttTables& t, int shape, bool inverse, uint32_t* d, int rows, int batch,
           const LimbMap& map, const RowRef* rowtab, cudaStream_t st, uint32_t* temp, size_t temp_bytes,
           const HmultTail* tail, const uint32_t* src) {
    constexpr int T = 1 << LOG_T, C = 1 << LOG_C, NC = 32 * T, N = NC * C;
    constexpr int smem = PadLayout<LOG_T>::kWords * 4;
    // forward: decimation in time (local NC-point transforms, then twist + C-point DFT);
    // inverse: decimation in frequency (quarter pass, then cross stages with N^-1)
    if (TAIL && (inverse || rowtab || !tail)) return set_error(FHE_EINVAL, "fused tail: forward, limb-map rows only");
    if (src && (!inverse || rowtab)) return set_error(FHE_EINVAL, "out-of-place two-pass NTT: inverse, limb-map rows only");
    auto qk = inverse ? ntt_quarter_inv_kernel<LOG_T, LOG_C>
                      : (TAIL && !tail->last) ? ntt_dit_local_kernel<LOG_T, LOG_C, TAIL, false>
                                              : ntt_dit_local_kernel<LOG_T, LOG_C, TAIL>;
    FHE_CUDA_TRY(cudaFuncSetAttribute(qk, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    int carve = (int)((kMinB<LOG_T> * (smem + 1024) * 100 + 228 * 1024 - 1) / (228 * 1024));
    FHE_CUDA_TRY(cudaFuncSetAttribute(qk, cudaFuncAttributePreferredSharedMemoryCarveout, carve > 100 ? 100 : carve));
    const NttTables& ts = ctx->ntt[LOG_T + 5];  // the NC-point ring degree of the local passes
    if (!inverse && (!ts.fwd || !ts.fwdC[0] || (C > 1 && (!t.dit_twist[shape] || !t.dit_omega[shape]))))
        return set_error(FHE_EINVAL, "two-pass forward tables missing");
    L2Args a;
    a.data = d;
    a.batch = batch;
    a.rowtab = rowtab;
    a.mod_q = ctx->d_mods;
    a.temp = temp;
    a.tw = inverse ? t.inv : t.fwd;
    a.twC = inverse ? t.invC[shape] : t.fwdC[shape];
    a.ninv = t.ninv;
    a.ninv_w1 = t.ninv_w1;
    a.tw_sub = ts.fwd;
    a.twC_sub = ts.fwdC[0];
    a.twist = t.dit_twist[shape];
    a.omega = t.dit_omega[shape];
    a.map = map;
    a.src_off = src ? src - d : 0;
    memset(&a.tail, 0, sizeof(a.tail));
    if (TAIL) a.tail = *tail;
    // chunk rows: N residues of scratch and one completion counter each
    const size_t chunk_rows = temp_bytes / ((size_t)N * 4 + 4);
    if (chunk_rows < 1) return set_error(FHE_EINVAL, "two-pass NTT scratch smaller than one row");
    const int chunk = (int)std::min<size_t>(chunk_rows, (size_t)1 << 30);
    a.cnt = reinterpret_cast<int*>(temp + (size_t)chunk * N);
    const int gx = (NC / 4 + 255) / 256;
    for (int r0 = 0; r0 < rows; r0 += chunk) {
        a.r0 = r0;
        a.nrows = rows - r0 < chunk ? rows - r0 : chunk;
        // fused cross passes need enough rows for the other CTAs to hide them: at least four
        // waves of local-pass CTAs
        a.fuse = (size_t)a.nrows * C >= (size_t)4 * ctx->num_sms * kMinB<LOG_T>;
        if (a.fuse) FHE_CUDA_TRY(cudaMemsetAsync(a.cnt, 0, (size_t)a.nrows * sizeof(int), st));
        qk<<<dim3(C, a.nrows), T, smem, st>>>(a);
        FHE_CUDA_TRY(cudaGetLastError());
        if (!a.fuse) {
            if (inverse)
                ntt_cross_inv_kernel<LOG_T + 5, LOG_C><<<dim3(gx, a.nrows), 256, 0, st>>>(a);
            else
                ntt_dit_cross_kernel<LOG_T + 5, LOG_C, TAIL><<<dim3(gx, a.nrows), 256, 0, st>>>(a);
            FHE_CUDA_TRY(cudaGetLastError());
        }
    }
    return FHE_OK;
}

}  // namespace

namespace {
template <bool TAIL>
int ntt_u32_l2_impl(const fhe_ctx* ctx, uint32_t logN, int shape, bool inverse, uint32_t* d, int rows, int batch,
                    const LimbMap& map, const RowRef* rowtab, cudaStream_t st, NttScratch scr, const HmultTail* tail,
                    const uint32_t* src = nullptr) {
    const NttTables& t = ctx->ntt[logN];
    uint32_t* temp = scr.p ? scr.p : ctx->ntt_temp;
    const size_t temp_bytes = scr.p ? scr.bytes : kNttTempBytes;
    if (!temp) return set_error(FHE_EINVAL, "no two-pass scratch in this context");
    int log_t, log_c;
    if (!ntt_variant_shape(logN, shape, &log_t, &log_c) || (log_c == 0 && !TAIL))
        return set_error(FHE_EINVAL, "two-pass NTT needs N >= 2^15");
    // N <= 2^14 with a tail: one CTA of N / 32 threads per row runs the whole transform and
    // then the tail's store side as a one-part cross pass
    if constexpr (TAIL) {
        if (log_t == 9 && log_c == 0)
            return run_l2<9, 0, TAIL>(ctx, t, shape, inverse, d, rows, batch, map, rowtab, st, temp, temp_bytes, tail,
                                      src);
        if (log_t == 8 && log_c == 0)
            return run_l2<8, 0, TAIL>(ctx, t, shape, inverse, d, rows, batch, map, rowtab, st, temp, temp_bytes, tail,
                                      src);
        if (log_t == 7 && log_c == 0)
            return run_l2<7, 0, TAIL>(ctx, t, shape, inverse, d, rows, batch, map, rowtab, st, temp, temp_bytes, tail,
                                      src);
    }
    if (log_t == 9 && log_c == 2)
        return run_l2<9, 2, TAIL>(ctx, t, shape, inverse, d, rows, batch, map, rowtab, st, temp, temp_bytes, tail, src);
    if (log_t == 9 && log_c == 1)
        return run_l2<9, 1, TAIL>(ctx, t, shape, inverse, d, rows, batch, map, rowtab, st, temp, temp_bytes, tail, src);
    if (log_t == 8 && log_c == 3)
        return run_l2<8, 3, TAIL>(ctx, t, shape, inverse, d, rows, batch, map, rowtab, st, temp, temp_bytes, tail, src);
    if (log_t == 8 && log_c == 2)
        return run_l2<8, 2, TAIL>(ctx, t, shape, inverse, d, rows, batch, map, rowtab, st, temp, temp_bytes, tail, src);
    return set_error(FHE_EINVAL, "no two-pass kernel for this shape");
}
}  // namespace

int ntt_u32_l2(const fhe_ctx* ctx, uint32_t logN, int shape, bool inverse, uint32_t* d, int rows, int batch,
               const LimbMap& map, const RowRef* rowtab, cudaStream_t st, NttScratch scr) {
    return ntt_u32_l2_impl<false>(ctx, logN, shape, inverse, d, rows, batch, map, rowtab, st, scr, nullptr);
}

bool ntt_inv_out_of_place(const fhe_ctx* ctx, uint32_t logN) {
    if (logN < 15 || logN > FHE_LOGN_MAX || ctx->ntt_variant[1][logN] >= kNttVariants) return false;
    const int v = ctx->plain_variant[1][logN];
    int log_t, log_c;
    return ntt_variant_exchange(v) == 3 && ntt_variant_shape(logN, v, &log_t, &log_c) && log_c > 0;
}

int ntt_inv_from(const fhe_ctx* ctx, uint32_t logN, uint32_t* dst, const uint32_t* src, int n_limbs, int batch,
                 const LimbMap& map, cudaStream_t st, NttScratch scr) {
    if (ntt_inv_out_of_place(ctx, logN)) {
        if (n_limbs == 0 || batch == 0) return FHE_OK;
        const int v = ctx->plain_variant[1][logN];
        return ntt_u32_l2_impl<false>(ctx, logN, v & 1, true, dst, n_limbs * batch, batch, map, nullptr, st, scr,
                                      nullptr, src);
    }
    FHE_CUDA_TRY(cudaMemcpyAsync(dst, src, ((size_t)n_limbs * batch << logN) * 4, cudaMemcpyDeviceToDevice, st));
    return ntt_any(ctx, FHE_NTT_DEFAULT, logN, true, dst, n_limbs, batch, map, st, scr);
}

bool ntt_tail_fusable(const fhe_ctx* ctx, int path, uint32_t logN) {
    if (logN < 12 || logN > FHE_LOGN_MAX) return false;
    if (path == FHE_NTT_DEFAULT && ctx->ntt_variant[0][logN] >= kNttVariants) return false;  // tensor cores
    if (path != FHE_NTT_DEFAULT && path != FHE_NTT_U32) return false;
    if (logN <= 14) return ctx->ntt[logN].fwd != nullptr;  // the one-CTA-per-row shape, whatever the variant
    const int v = ctx->plain_variant[0][logN];
    int log_t, log_c;
    return ntt_variant_exchange(v) == 3 && ntt_variant_shape(logN, v, &log_t, &log_c) && log_c > 0;
}

int ntt_u32_l2_tail(const fhe_ctx* ctx, uint32_t logN, int rows, int batch, const LimbMap& map, cudaStream_t st,
                    NttScratch scr, const HmultTail& tail) {
    if (!ntt_tail_fusable(ctx, FHE_NTT_U32, logN)) return set_error(FHE_EINVAL, "fused tail needs the two-pass NTT");
    if (rows == 0) return FHE_OK;
    const int v = ctx->plain_variant[0][logN];
    // the data pointer is not read or written by the TAIL kernels (rows come from y / go to out)
    return ntt_u32_l2_impl<true>(ctx, logN, logN <= 14 ? 0 : v & 1, false, tail.out, rows, batch, map, nullptr, st, scr,
                                 &tail);
}

}  // namespace fhe

// Tensor-core NTT (Sec. IV-B Eq. (9) and Sec. IV-C, Stages 1-5) on sm_103a tcgen05.
//
// Four-step form, N = N1 * N2 (N1 = 2^ceil(logN/2), N2 = 2^floor(logN/2)), index maps
// n = N2*n1 + n2 and k = k1 + N1*k2:
//   forward  A[k1 + N1 k2] = sum_n2 w^(n2 k2) psi^((2k1+1) n2) sum_n1 psi^(N2 (2k1+1) n1) a[N2 n1 + n2]
//   inverse  a[N2 n1 + n2] = N^-1 sum_k1 psi^(-N2 (2k1+1) n1) psi^(-(2k1+1) n2) sum_k2 psi^(-2 N1 n2 k2) A[k1 + N1 k2]
// (w = psi^(2 N1)). Each direction is two persistent GEMM kernels per chunk of polynomials:
//   gemm 1 (Stages 1-3): TMA brings the u32 residues, converter warps split them into four
//          8-bit digits (Stage 1) laid out with the reduction index contiguous (K-major
//          operand) in shared memory only; tcgen05 GEMM against the first twiddle matrix; the
//          epilogue rebuilds each output mod q, multiplies by the twiddle and re-splits it into
//          digit planes for the next GEMM (transposed);
//   gemm 2 (Stages 4-5): tcgen05 GEMM against the second matrix; the epilogue rebuilds mod q
//          and stores natural-order u32 results.
//
// Segment fusion on this GPU: sm_103a has no tcgen05 integer MMA (ptxas rejects kind::i8),
// so the 8-bit segments are carried exactly in fp16 (kind::f16, fp32 accumulation in TMEM).
// Data digits are balanced base-256 digits in [-128, 127]; twiddle-matrix digits are balanced
// base-255 digits in [-127, 127]. The j-th data digit's weight 256^j is folded into the
// constant matrix (W 256^j mod q), so one accumulator per twiddle digit i remains:
//   acc_i = sum_{n, j} d_j(x_n) e_i(W_n 256^j mod q),    y = sum_i 255^i acc_i = W x (mod q).
// |d e| <= 128 * 127 = 16256 and K' = 4K <= 1024 terms keep every partial sum below
// 16,646,144 < 2^24, so the fp32 accumulation is exact (integers below 2^24 are exact).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "ptx.cuh"

namespace fhe {
namespace {

constexpr int kTileM = 128;
constexpr int kChunk = 64;             // K' elements (fp16) per pipeline stage = 128 bytes
constexpr int kMaxChunkLimbs = 64;

struct GemmArgs {
    int rows;     // polynomials per limb in this launch
    int Y;        // A rows per polynomial
    int X4;       // K' = 4 X
    int cols;     // output columns of the matrix
    int N;
    int mode;     // 1: twiddle + re-split into planes; 2: u32 output
    size_t out_limb_stride;  // mode 2: elements between limbs of `out`
    const uint2* tw;         // mode 1: [nmod][cols][Y]
    uint2* planes;           // mode 1: [limb][rows][cols][Y] groups of four fp16 digits
    uint32_t* out;           // mode 2: first row of the chunk
    int X;                   // first GEMM: reduction size (source rows per polynomial)
    int src_batch;           // first GEMM: polynomials between limbs of the source
    int* status;
    uint32_t q[kMaxChunkLimbs];
    uint64_t mu[kMaxChunkLimbs];
    uint64_t off[kMaxChunkLimbs];  // multiple of q above 2^49 that makes the rebuilt value positive
    int mod[kMaxChunkLimbs];
};

// Epilogue of both GEMM kernels, run by one warp over all of the CTA's tiles: the warp reads
// TMEM lanes [32 quarter, 32 quarter + 32) (= tile rows) of the accumulator buffer lt & 1 once
// acc_full says its MMAs are complete, rebuilds each value mod q, then either multiplies by the
// twiddle and stores the four fp16 digits into the planes (mode 1) or stores the u32 result in
// natural order (mode 2), and hands the buffer back through acc_empty. CB = TMEM columns per
// load (8 keeps the fused kernel within its register budget). Every wait is bounded.
template <int NT, int CB>
__device__ __forceinline__ void epilogue_warp(const GemmArgs& a, uint32_t tmem, uint64_t* acc_full,
                                              uint64_t* acc_empty, int quarter, int lane, int tiles_m,
                                              int tiles_n, int ntiles) {
    constexpr int kAccCols = 4 * NT;
    int lt = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++lt) {
        const int buf = lt & 1;
        // warp-uniform verdict: the tcgen05.ld below is .sync.aligned
        const bool ok = __all_sync(
            0xffffffffu, ptx::mbar_wait(&acc_full[buf], (uint32_t)((lt >> 1) & 1), a.status, FHE_ETIMEOUT));
        if (!ok) break;
        ptx::tc_fence_after();
        const int mt = t % tiles_m, nt = (t / tiles_m) % tiles_n, z = t / (tiles_m * tiles_n);
        const int n0 = nt * NT;
        const int mrow = mt * kTileM + quarter * 32 + lane;
        const bool valid = mrow < a.rows * a.Y;
        const int poly = mrow / a.Y, y = mrow % a.Y;
        const uint32_t q = a.q[z];
        const uint64_t mu = a.mu[z], off = a.off[z];
        const uint32_t lane_base = tmem + buf * kAccCols + ((uint32_t)(quarter * 32) << 16);
        // mode 1: this thread's twiddles for column block cb (CB columns, stride Y), loaded one
        // block ahead so their L2 latency overlaps the TMEM loads and the previous block's work
        const uint2* twp = a.tw + ((size_t)a.mod[z] * a.cols + n0) * a.Y + y;
        uint2 wnext[CB];
        if (a.mode == 1 && valid) {
#pragma unroll
            for (int j = 0; j < CB; ++j) wnext[j] = __ldg(&twp[(size_t)j * a.Y]);
        }
#pragma unroll 1
        for (int cb = 0; cb < NT / CB; ++cb) {
            uint32_t r[4][CB];
            uint2 wcur[CB];
#pragma unroll
            for (int j = 0; j < CB; ++j) wcur[j] = wnext[j];
            if (a.mode == 1 && valid && cb + 1 < NT / CB) {
#pragma unroll
                for (int j = 0; j < CB; ++j) wnext[j] = __ldg(&twp[(size_t)((cb + 1) * CB + j) * a.Y]);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) ptx::tmem_ld<CB>(lane_base + i * NT + cb * CB, r[i]);
            ptx::tmem_wait_ld();
            if (!valid) continue;
#pragma unroll
            for (int j = 0; j < CB; ++j) {
                const int col = n0 + cb * CB + j;
                const long long a0 = __float2int_rn(__uint_as_float(r[0][j]));
                const long long a1 = __float2int_rn(__uint_as_float(r[1][j]));
                const long long a2 = __float2int_rn(__uint_as_float(r[2][j]));
                const long long a3 = __float2int_rn(__uint_as_float(r[3][j]));
                const long long yv = a0 + 255 * a1 + 65025 * a2 + 16581375 * a3;
                uint32_t v = reduce_u64((uint64_t)(yv + (long long)off), mu, q);
                if (a.mode == 1) {
                    v = mul_shoup(v, wcur[j].x, wcur[j].y, q);
                    a.planes[(((size_t)z * a.rows + poly) * a.cols + col) * a.Y + y] = split_f16x4(v);
                } else {
                    a.out[z * a.out_limb_stride + (size_t)poly * a.N + (size_t)col * a.Y + y] = v;
                }
            }
        }
        ptx::tc_fence_before();
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(&acc_empty[buf]);  // this warp's rows of the buffer are read
    }
}

// Stages 4-5 (and the digit-plane form of Stages 2-3), persistent: one CTA per SM walks the
// 128 x NT output tiles of all limbs, t = blockIdx.x + k gridDim.x (row tiles fastest, so the
// CTAs running at one time share their B tiles in L2). Warp 0 issues the TMA loads of A (digit
// planes) and B through a 4-stage shared-memory ring, warp 1 issues the MMAs, warps 2-5 run
// the epilogue. The accumulators are double-buffered in TMEM (2 x 4 NT columns), so the MMAs
// of tile k+1 run while the epilogue drains tile k.
template <int NT>
struct GemmCfg {
    static constexpr int kABytes = kTileM * 128;
    static constexpr int kBBytes = 4 * NT * 128;
    static constexpr int kStageBytes = kABytes + kBBytes;
    static constexpr int kStages = (200 * 1024) / kStageBytes > 4 ? 4 : (200 * 1024) / kStageBytes;
    static constexpr int kSmem = kStages * kStageBytes + 1024;
    static constexpr int kAccCols = 4 * NT;
    static constexpr int kTmemCols = 2 * kAccCols;  // a power of two: 256 or 512
};

// The four digit planes of the constant matrix are consecutive rows of one B tile, so a single
// M=128, N=4*NT MMA per K step (K = 16) fills all four accumulators of a buffer (its TMEM
// columns [i*NT, (i+1)*NT) hold acc_i) and reads the A tile once.
template <int NT>
__device__ __forceinline__ void mma_chunk(uint32_t acc, uint32_t As, uint32_t Bs, bool first) {
    constexpr uint32_t idesc = ptx::idesc_f16(kTileM, 4 * NT);
#pragma unroll
    for (int kk = 0; kk < kChunk / 16; ++kk) {
        const uint64_t adesc = ptx::sdesc_sw128(As + kk * 32);
        const uint64_t bdesc = ptx::sdesc_sw128(Bs + kk * 32);
        ptx::mma_f16(acc, adesc, bdesc, idesc, (!first || kk > 0) ? 1u : 0u);
    }
}

template <int NT>
__global__ void __launch_bounds__(192, 1)
tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               const GemmArgs a, int tiles_m, int tiles_n, int nl) {
    using Cfg = GemmCfg<NT>;
    constexpr int S = Cfg::kStages;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    __shared__ uint64_t full[S], empty[S], acc_full[2], acc_empty[2], drained;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntiles = tiles_m * tiles_n * nl;
    const int nchunks = a.X4 / kChunk;

    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            ptx::mbar_init(&full[s], 1);
            ptx::mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            ptx::mbar_init(&acc_full[b], 1);
            ptx::mbar_init(&acc_empty[b], 4);
        }
        ptx::mbar_init(&drained, 1);
        ptx::fence_mbar_init();
    }
    if (warp == 0) {
        ptx::tmem_alloc(&tmem_base, Cfg::kTmemCols);
        ptx::tmem_relinquish();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = tmem_base;

    if (warp == 0 && lane == 0) {
        // ---- TMA producer
        ptx::prefetch_tmap(&tmA);
        ptx::prefetch_tmap(&tmB);
        bool ok = true;
        long long issued = 0;
        for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
            const int mt = t % tiles_m, nt = (t / tiles_m) % tiles_n, z = t / (tiles_m * tiles_n);
            const int a_row0 = z * a.rows * a.Y + mt * kTileM;
            const int b_row0 = a.mod[z] * 4 * a.cols + nt * NT;
            for (int c = 0; c < nchunks; ++c, ++issued) {
                const int s = (int)(issued % S);
                if (issued >= S) ok = ptx::mbar_wait(&empty[s], (uint32_t)(((issued / S) - 1) & 1), a.status, FHE_ETIMEOUT);
                if (!ok) break;
                uint8_t* As = sm + s * Cfg::kStageBytes;
                uint8_t* Bs = As + Cfg::kABytes;
                ptx::mbar_arrive_expect_tx(&full[s], Cfg::kStageBytes);
                ptx::tma_load_2d(As, &tmA, c * kChunk, a_row0, &full[s]);
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    ptx::tma_load_2d(Bs + i * NT * 128, &tmB, c * kChunk, b_row0 + i * a.cols, &full[s]);
            }
        }
        if (!ok) {
            // drain the copies that may still be in flight (bounded) before the CTA may exit
            for (long long c = (issued > S ? issued - S : 0); c < issued; ++c)
                ptx::mbar_wait(&full[c % S], (uint32_t)((c / S) & 1), nullptr, 0);
        }
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer
        bool ok = true;
        long long consumed = 0;
        int lt = 0;
        for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++lt) {
            const int buf = lt & 1;
            if (lt >= 2) ok = ptx::mbar_wait(&acc_empty[buf], (uint32_t)(((lt >> 1) - 1) & 1), a.status, FHE_ETIMEOUT);
            if (!ok) break;
            ptx::tc_fence_after();
            for (int c = 0; c < nchunks; ++c, ++consumed) {
                const int s = (int)(consumed % S);
                ok = ptx::mbar_wait(&full[s], (uint32_t)((consumed / S) & 1), a.status, FHE_ETIMEOUT);
                if (!ok) break;
                ptx::tc_fence_after();
                const uint32_t As = ptx::smem_u32(sm + s * Cfg::kStageBytes);
                mma_chunk<NT>(tmem + buf * Cfg::kAccCols, As, As + Cfg::kABytes, c == 0);
                ptx::mma_commit(&empty[s]);
            }
            if (ok) ptx::mma_commit(&acc_full[buf]);
        }
        // every MMA issued above has completed before TMEM can be released
        ptx::mma_commit(&drained);
        ptx::mbar_wait(&drained, 0, nullptr, 0);
    } else if (warp >= 2) {
        epilogue_warp<NT, 16>(a, tmem, acc_full, acc_empty, warp & 3, lane, tiles_m, tiles_n, ntiles);
    }

    __syncwarp();
    ptx::tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        __syncwarp();
        ptx::tmem_dealloc(tmem, Cfg::kTmemCols);
    }
}

// Stages 1-3 fused, persistent (same tile walk and TMEM double buffering as tc_gemm_kernel):
// the A operand is built on chip from the caller's u32 residues, so their digit planes never
// reach HBM. Three shared-memory rings, each sized for the latency it has to cover:
//   B   (4 x 4 NT rows x 128 B): warp 0 loads the constant-matrix planes by TMA;
//   raw (per converter warp, 2 x 2 KB): each converter warp TMA-loads the 16 reduction indices
//       x 32 rows of its quarter of the A tile, and refills a slot as soon as it has read it,
//       so the raw loads run ahead of the conversion;
//   A   (4 x 16 KB): the converter warps (6-13, two groups of four taking alternate stages)
//       split the residues into fp16 digits and store them in the 128-byte swizzled K-major
//       layout of the MMA descriptors; each stage ends with a proxy fence, whose latency the
//       other group's stage overlaps.
// Warp 1 issues the MMAs once A and B of a stage are both full; warps 2-5 run the epilogue.
// Every wait is bounded.
template <int NT>
struct FusedCfg {
    static constexpr int kGroups = 2;                  // converter warp groups (alternate stages)
    static constexpr int kSA = 4, kSB = 4, kSR = 2;    // kSR: source slots per converter warp
    static constexpr int kABytes = kTileM * 128;
    static constexpr int kBBytes = 4 * NT * 128;
    static constexpr int kRawBytes = 32 * (kChunk / 4) * 4;  // one converter warp's 32 rows
    static constexpr int kOffB = kSA * kABytes;
    static constexpr int kOffRaw = kOffB + kSB * kBBytes;
    static constexpr int kSmem = kOffRaw + 4 * kGroups * kSR * kRawBytes + 1024;
    static constexpr int kThreads = 32 * (6 + 4 * kGroups);
    static constexpr int kAccCols = 4 * NT;
    static constexpr int kTmemCols = 2 * kAccCols;
};

template <int NT>
__global__ void __launch_bounds__(FusedCfg<NT>::kThreads, 1)
tc_gemm_fused_kernel(const __grid_constant__ CUtensorMap tmS, const __grid_constant__ CUtensorMap tmB,
                     const GemmArgs a, int tiles_m, int tiles_n, int nl) {
    using Cfg = FusedCfg<NT>;
    constexpr int SA = Cfg::kSA, SB = Cfg::kSB, SR = Cfg::kSR;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    __shared__ uint64_t a_full[SA], a_empty[SA], b_full[SB], b_empty[SB], raw_full[4 * Cfg::kGroups][SR];
    __shared__ uint64_t acc_full[2], acc_empty[2], drained;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntiles = tiles_m * tiles_n * nl;
    const int nchunks = a.X4 / kChunk;

    if (tid == 0) {
        for (int s = 0; s < SA; ++s) {
            ptx::mbar_init(&a_full[s], 4);  // one arrival per converter warp of the stage's group
            ptx::mbar_init(&a_empty[s], 1);
        }
        for (int s = 0; s < SB; ++s) {
            ptx::mbar_init(&b_full[s], 1);
            ptx::mbar_init(&b_empty[s], 1);
        }
        for (int w = 0; w < 4 * Cfg::kGroups; ++w)
            for (int s = 0; s < SR; ++s) ptx::mbar_init(&raw_full[w][s], 1);
        for (int b = 0; b < 2; ++b) {
            ptx::mbar_init(&acc_full[b], 1);
            ptx::mbar_init(&acc_empty[b], 4);
        }
        ptx::mbar_init(&drained, 1);
        ptx::fence_mbar_init();
    }
    if (warp == 0) {
        ptx::tmem_alloc(&tmem_base, Cfg::kTmemCols);
        ptx::tmem_relinquish();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = tmem_base;

    if (warp == 0 && lane == 0) {
        // ---- TMA producer of B
        ptx::prefetch_tmap(&tmB);
        bool ok = true;
        long long issued = 0;
        for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
            const int nt = (t / tiles_m) % tiles_n, z = t / (tiles_m * tiles_n);
            const int b_row0 = a.mod[z] * 4 * a.cols + nt * NT;
            for (int c = 0; c < nchunks; ++c, ++issued) {
                const int s = (int)(issued % SB);
                if (issued >= SB)
                    ok = ptx::mbar_wait(&b_empty[s], (uint32_t)(((issued / SB) - 1) & 1), a.status, FHE_ETIMEOUT);
                if (!ok) break;
                uint8_t* Bs = sm + Cfg::kOffB + s * Cfg::kBBytes;
                ptx::mbar_arrive_expect_tx(&b_full[s], Cfg::kBBytes);
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    ptx::tma_load_2d(Bs + i * NT * 128, &tmB, c * kChunk, b_row0 + i * a.cols, &b_full[s]);
            }
        }
        if (!ok) {
            for (long long c = (issued > SB ? issued - SB : 0); c < issued; ++c)
                ptx::mbar_wait(&b_full[c % SB], (uint32_t)((c / SB) & 1), nullptr, 0);
        }
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer
        bool ok = true;
        long long k = 0;
        int lt = 0;
        for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++lt) {
            const int buf = lt & 1;
            if (lt >= 2) ok = ptx::mbar_wait(&acc_empty[buf], (uint32_t)(((lt >> 1) - 1) & 1), a.status, FHE_ETIMEOUT);
            if (!ok) break;
            ptx::tc_fence_after();
            for (int c = 0; c < nchunks; ++c, ++k) {
                const int sa = (int)(k % SA), sb = (int)(k % SB);
                ok = ptx::mbar_wait(&a_full[sa], (uint32_t)((k / SA) & 1), a.status, FHE_ETIMEOUT) &&
                     ptx::mbar_wait(&b_full[sb], (uint32_t)((k / SB) & 1), a.status, FHE_ETIMEOUT);
                if (!ok) break;
                ptx::tc_fence_after();
                mma_chunk<NT>(tmem + buf * Cfg::kAccCols, ptx::smem_u32(sm + sa * Cfg::kABytes),
                              ptx::smem_u32(sm + Cfg::kOffB + sb * Cfg::kBBytes), c == 0);
                ptx::mma_commit(&a_empty[sa]);
                ptx::mma_commit(&b_empty[sb]);
            }
            if (ok) ptx::mma_commit(&acc_full[buf]);
        }
        ptx::mma_commit(&drained);
        ptx::mbar_wait(&drained, 0, nullptr, 0);
    } else if (warp >= 2 && warp < 6) {
        epilogue_warp<NT, 8>(a, tmem, acc_full, acc_empty, warp & 3, lane, tiles_m, tiles_n, ntiles);
    } else if (warp >= 6) {
        // ---- Stage 1 converters: two groups of four warps take alternate stages (k = g mod 2),
        // so the conversion of one stage overlaps the proxy fence of the other. Warp (g, cw) owns
        // A rows r = 32 cw + lane (TMEM lanes): per stage each thread splits its 16 residues
        // (reduction indices x = 16 c .. 16 c + 15) into 64 fp16 digits, K' = 4 x + j, stored as
        // eight 16-byte chunks, chunk i at position i ^ (r % 8) of the row (the 128-byte swizzle).
        constexpr int G = Cfg::kGroups;
        const int cw = (warp - 6) & 3, g = (warp - 6) >> 2, r = 32 * cw + lane;
        uint8_t* raw = sm + Cfg::kOffRaw + (warp - 6) * SR * Cfg::kRawBytes;
        uint64_t* rfull = raw_full[warp - 6];
        // issue cursor: the next of this warp's stages whose source box it loads (32 n-indices of
        // one polynomial x 16 reduction indices; rows of the source map are (limb, polynomial, x))
        int it = blockIdx.x, ic = g, irow = 0, iy0 = 0;
        long long jnext = 0;
        auto place = [&]() {
            const int mt = it % tiles_m, z = it / (tiles_m * tiles_n);
            const int m = mt * kTileM + 32 * cw;
            irow = (z * a.src_batch + m / a.Y) * a.X;
            iy0 = m % a.Y;
        };
        auto issue_next = [&]() {  // lane 0
            const int s = (int)(jnext % SR);
            ptx::mbar_arrive_expect_tx(&rfull[s], Cfg::kRawBytes);
            ptx::tma_load_2d(raw + s * Cfg::kRawBytes, &tmS, iy0, irow + ic * (kChunk / 4), &rfull[s]);
            ++jnext;
            if ((ic += G) >= nchunks) {
                ic = g;
                it += gridDim.x;
                if (it < ntiles) place();
            }
        };
        const int my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
        const long long total = (long long)my_tiles * (nchunks / G);  // this warp's stages
        if (lane == 0 && total > 0) {
            ptx::prefetch_tmap(&tmS);
            place();
            while (jnext < SR && jnext < total) issue_next();
        }
        __syncwarp();
        long long j = 0;
        bool ok = true;
        for (; j < total; ++j) {
            const long long k = g + (long long)G * j;  // the CTA's stage index
            const int s = (int)(j % SR), sa = (int)(k % SA);
            ok = __all_sync(0xffffffffu, ptx::mbar_wait(&rfull[s], (uint32_t)((j / SR) & 1), a.status, FHE_ETIMEOUT));
            if (!ok) break;
            const uint32_t* src = reinterpret_cast<const uint32_t*>(raw + s * Cfg::kRawBytes) + lane;
            uint4 d[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const uint2 p0 = split_f16x4(src[(2 * i) * 32]);
                const uint2 p1 = split_f16x4(src[(2 * i + 1) * 32]);
                d[i] = make_uint4(p0.x, p0.y, p1.x, p1.y);
            }
            // the slot's values are in registers (the splits consumed them): refill it with this
            // warp's stage SR ahead
            __syncwarp();
            if (lane == 0 && j + SR < total) issue_next();
            if (k >= SA)
                ok = __all_sync(0xffffffffu,
                                ptx::mbar_wait(&a_empty[sa], (uint32_t)(((k / SA) - 1) & 1), a.status, FHE_ETIMEOUT));
            if (!ok) {
                ++j;  // stage j is consumed; stages j + 1 .. jnext - 1 are in flight
                break;
            }
            uint8_t* arow = sm + sa * Cfg::kABytes + r * 128;
#pragma unroll
            for (int i = 0; i < 8; ++i) *reinterpret_cast<uint4*>(arow + ((i ^ (r & 7)) << 4)) = d[i];
            ptx::fence_proxy_async();  // the MMA reads these bytes through the async proxy
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(&a_full[sa]);
        }
        if (!ok && lane == 0) {
            // drain this warp's source copies still in flight (bounded) before the CTA may exit
            for (long long jj = j; jj < jnext; ++jj)
                ptx::mbar_wait(&rfull[jj % SR], (uint32_t)((jj / SR) & 1), nullptr, 0);
        }
    }

    __syncwarp();
    ptx::tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        __syncwarp();
        ptx::tmem_dealloc(tmem, Cfg::kTmemCols);
    }
}

// ------------------------------------------------------------------ host side

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult qr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &qr) ==
                cudaSuccess &&
            qr == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    });
    return fn;
}

// 2-D fp16 tensor map over a row-major [rows][inner] array, box = 64 x box_rows, 128B swizzle.
int make_map(CUtensorMap* m, const void* base, uint64_t inner, uint64_t rows, uint32_t box_rows) {
    auto fn = encode_fn();
    if (!fn) return set_error(FHE_ECUDA, "cuTensorMapEncodeTiled is unavailable");
    cuuint64_t dims[2] = {inner, rows};
    cuuint64_t strides[1] = {inner * 2};
    cuuint32_t box[2] = {(cuuint32_t)kChunk, box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(FHE_ECUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
    return FHE_OK;
}

// 2-D u32 tensor map over the caller's residues viewed as [rows][inner] (inner = the A rows of
// one polynomial), box = box_inner x 16 rows, no swizzle; rows past the end read as zero.
int make_src_map(CUtensorMap* m, const uint32_t* base, uint64_t inner, uint64_t rows, uint32_t box_inner) {
    auto fn = encode_fn();
    if (!fn) return set_error(FHE_ECUDA, "cuTensorMapEncodeTiled is unavailable");
    cuuint64_t dims[2] = {inner, rows};
    cuuint64_t strides[1] = {inner * 4};
    cuuint32_t box[2] = {box_inner, (cuuint32_t)(kChunk / 4)};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, const_cast<uint32_t*>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(FHE_ECUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
    return FHE_OK;
}

// Balanced base-255 digits of w < 2^30: w = e0 + 255 e1 + 255^2 e2 + 255^3 e3, |e_i| <= 127.
void digits255(uint32_t w, int e[4]) {
    int64_t x = w;
    for (int i = 0; i < 3; ++i) {
        int64_t d = ((x + 127) % 255) - 127;
        e[i] = (int)d;
        x = (x - d) / 255;
    }
    e[3] = (int)x;
}

int tc_cols(uint32_t logN, int kind, int* n1, int* n2) {
    *n1 = 1 << ((logN + 1) / 2);
    *n2 = 1 << (logN / 2);
    return (kind == 0 || kind == 3) ? *n1 : *n2;
}

std::mutex g_tc_mu;

}  // namespace

// Matrices (cols x K), kind 0: W1 forward, 1: W3 forward, 2: W3 inverse, 3: W1 inverse.
int build_tc_tables(fhe_ctx* ctx, uint32_t logN) {
    TcTables& t = ctx->tc[logN];
    if (t.built) return FHE_OK;
    const int nmod = (int)ctx->mods.size();
    const uint32_t N = 1u << logN;
    int n1, n2;
    tc_cols(logN, 0, &n1, &n2);
    t.n1 = n1;
    t.n2 = n2;
    int rc;
    if (!ctx->tc_planes) {
        if ((rc = dev_alloc(ctx, (uint8_t**)&ctx->tc_planes, kTcPlaneBytes))) return rc;
    }
    for (int kind = 0; kind < 4; ++kind) {
        const int cols = (kind == 0 || kind == 3) ? n1 : n2;
        const int K = cols;
        const size_t per_mod = (size_t)4 * cols * 4 * K;
        std::vector<uint16_t> h((size_t)nmod * per_mod);
        for (int m = 0; m < nmod; ++m) {
            const uint32_t q = ctx->mods[m];
            const uint32_t psi = root_2n(q, logN);
            const uint32_t psi_inv = invmod_h(psi, q);
            const uint64_t two_n = 2ull * N;
            for (int c = 0; c < cols; ++c)
                for (int n = 0; n < K; ++n) {
                    uint64_t e;
                    uint32_t base;
                    switch (kind) {
                        case 0: e = (uint64_t)n2 * (2ull * c + 1) * n % two_n; base = psi; break;
                        case 1: e = 2ull * n1 * n * c % two_n; base = psi; break;
                        case 2: e = 2ull * n1 * c * n % two_n; base = psi_inv; break;
                        default: e = (uint64_t)n2 * (2ull * n + 1) * c % two_n; base = psi_inv; break;
                    }
                    uint32_t w = powmod_h(base, e, q);
                    for (int j = 0; j < 4; ++j) {
                        uint32_t wj = mulmod_h(w, powmod_h(256, j, q), q);
                        int dg[4];
                        digits255(wj, dg);
                        for (int i = 0; i < 4; ++i)
                            h[(size_t)m * per_mod + (((size_t)i * cols + c) * 4 * K) + (size_t)n * 4 + j] =
                                f16_bits_of_small_int(dg[i]);
                    }
                }
        }
        if ((rc = dev_upload(ctx, &t.mat[kind], h))) return rc;
        // the B tiles of a GEMM with NT-column output tiles are 4 TMA boxes of NT rows (one per
        // digit plane), so each tile width has its own map
        if ((rc = make_map(&t.map_b[kind], t.mat[kind], (uint64_t)4 * K, (uint64_t)nmod * 4 * cols,
                           cols >= 64 ? 64 : 32)))
            return rc;
        if ((rc = make_map(&t.map_b32[kind], t.mat[kind], (uint64_t)4 * K, (uint64_t)nmod * 4 * cols, 32)))
            return rc;
    }
    // twiddles for the first-GEMM epilogue: forward [k1][n2] psi^((2k1+1) n2);
    // inverse [n2][k1] psi^(-(2k1+1) n2) N^-1
    std::vector<uint2> twf((size_t)nmod * N), twi((size_t)nmod * N);
    for (int m = 0; m < nmod; ++m) {
        const uint32_t q = ctx->mods[m];
        const uint32_t psi = root_2n(q, logN);
        const uint32_t psi_inv = invmod_h(psi, q);
        const uint32_t ninv = invmod_h(N % q, q);
        for (int k1 = 0; k1 < n1; ++k1)
            for (int x = 0; x < n2; ++x) {
                const uint64_t e = (2ull * k1 + 1) * x % (2ull * N);
                uint32_t wf = powmod_h(psi, e, q);
                uint32_t wi = mulmod_h(powmod_h(psi_inv, e, q), ninv, q);
                twf[(size_t)m * N + (size_t)k1 * n2 + x] = make_uint2(wf, shoup_h(wf, q));
                twi[(size_t)m * N + (size_t)x * n1 + k1] = make_uint2(wi, shoup_h(wi, q));
            }
    }
    if ((rc = dev_upload(ctx, &t.tw_fwd, twf))) return rc;
    if ((rc = dev_upload(ctx, &t.tw_inv, twi))) return rc;
    // second-GEMM operand maps over the plane buffer: [rows][4X] for X = n1 and X = n2
    const uint64_t cap_n1 = kTcPlaneBytes / 2 / (4ull * n1), cap_n2 = kTcPlaneBytes / 2 / (4ull * n2);
    if ((rc = make_map(&t.map_a[0], ctx->tc_planes, 4ull * n1, cap_n1, kTileM))) return rc;
    if ((rc = make_map(&t.map_a[1], ctx->tc_planes, 4ull * n2, cap_n2, kTileM))) return rc;
    t.built = true;
    return FHE_OK;
}

template <int NT>
int launch_gemm(const fhe_ctx* ctx, const CUtensorMap& ma, const CUtensorMap& mb, const GemmArgs& g, int nl,
                cudaStream_t st) {
    using Cfg = GemmCfg<NT>;
    FHE_CUDA_TRY(cudaFuncSetAttribute(tc_gemm_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::kSmem));
    FHE_CUDA_TRY(cudaFuncSetAttribute(tc_gemm_kernel<NT>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    const int tiles_m = (g.rows * g.Y + kTileM - 1) / kTileM, tiles_n = g.cols / NT;
    const int ntiles = tiles_m * tiles_n * nl;
    const int grid = ntiles < ctx->num_sms ? ntiles : ctx->num_sms;
    tc_gemm_kernel<NT><<<grid, 192, Cfg::kSmem, st>>>(ma, mb, g, tiles_m, tiles_n, nl);
    FHE_CUDA_TRY(cudaGetLastError());
    return FHE_OK;
}

template <int NT>
int launch_gemm_fused(const fhe_ctx* ctx, const CUtensorMap& ms, const CUtensorMap& mb, const GemmArgs& g, int nl,
                      cudaStream_t st) {
    using Cfg = FusedCfg<NT>;
    if ((g.X4 / kChunk) % Cfg::kGroups) return set_error(FHE_EINVAL, "tensor-core NTT: reduction size too small");
    FHE_CUDA_TRY(
        cudaFuncSetAttribute(tc_gemm_fused_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::kSmem));
    FHE_CUDA_TRY(cudaFuncSetAttribute(tc_gemm_fused_kernel<NT>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    const int tiles_m = (g.rows * g.Y + kTileM - 1) / kTileM, tiles_n = g.cols / NT;
    const int ntiles = tiles_m * tiles_n * nl;
    const int grid = ntiles < ctx->num_sms ? ntiles : ctx->num_sms;
    tc_gemm_fused_kernel<NT><<<grid, Cfg::kThreads, Cfg::kSmem, st>>>(ms, mb, g, tiles_m, tiles_n, nl);
    FHE_CUDA_TRY(cudaGetLastError());
    return FHE_OK;
}

int ntt_tc(const fhe_ctx* cctx, uint32_t logN, bool inverse, uint32_t* d, int n_limbs, int batch,
           const LimbMap& map, cudaStream_t st, NttScratch scr) {
    fhe_ctx* ctx = const_cast<fhe_ctx*>(cctx);
    {
        std::lock_guard<std::mutex> lock(g_tc_mu);
        int rc = build_tc_tables(ctx, logN);
        if (rc) return rc;
    }
    const TcTables& t = ctx->tc[logN];
    const int n1 = t.n1, n2 = t.n2;
    const int nt = ctx->tc_nt[inverse ? 1 : 0][logN];  // output tile width (64 or 32 columns)
    const size_t N = (size_t)1 << logN;
    // X: first-GEMM reduction size, Y: its rows per polynomial; the second GEMM swaps them.
    const int X1 = inverse ? n2 : n1, Y1 = inverse ? n1 : n2;
    const int cols1 = inverse ? n2 : n1, cols2 = inverse ? n1 : n2;
    const int kind1 = inverse ? 2 : 0, kind2 = inverse ? 3 : 1;
    // the digit planes: the caller's region when given (calls may then overlap on other
    // streams), else the context's buffer, with the second GEMM's operand map over it
    uint2* planes = (uint2*)ctx->tc_planes;
    size_t plane_bytes = kTcPlaneBytes;
    CUtensorMap own_a;
    const CUtensorMap* a2 = &t.map_a[inverse ? 0 : 1];
    if (scr.p) {
        plane_bytes = std::min(scr.bytes, kTcPlaneBytes);
        if (plane_bytes < N * 8) return set_error(FHE_EINVAL, "tensor-core NTT: scratch region below 8 N bytes");
        planes = (uint2*)scr.p;
        const uint64_t inner = 4ull * (inverse ? n1 : n2);
        int rc0 = make_map(&own_a, planes, inner, plane_bytes / 2 / inner, kTileM);
        if (rc0) return rc0;
        a2 = &own_a;
    }
    const size_t cap_polys = plane_bytes / (N * 8);  // fp16 x 4 digits per residue
    int nb = batch, nlc = (int)(cap_polys / batch);
    if (nlc < 1) {
        nlc = 1;
        nb = (int)cap_polys;
    }
    if (nlc > kMaxChunkLimbs) nlc = kMaxChunkLimbs;
    int rc;
    for (int l0 = 0; l0 < n_limbs; l0 += nlc) {
        const int nl = std::min(nlc, n_limbs - l0);
        for (int b0 = 0; b0 < batch; b0 += nb) {
            const int rows = std::min(nb, batch - b0);
            uint32_t* base = d + ((size_t)l0 * batch + b0) * N;
            GemmArgs g;
            memset(&g, 0, sizeof(g));
            g.rows = rows;
            g.N = (int)N;
            g.status = ctx->d_status;
            for (int z = 0; z < nl; ++z) {
                const uint32_t q = map.q[l0 + z];
                g.q[z] = q;
                g.mu[z] = ~0ull / q;
                g.off[z] = (((1ull << 49) + q - 1) / q) * q;
                g.mod[z] = map.mod[l0 + z];
            }
            // Stage 1 runs inside the first GEMM: its source map views this chunk's residues as
            // rows (limb, polynomial, x) of Y1 values
            CUtensorMap src;
            if ((rc = make_src_map(&src, base, (uint64_t)Y1, ((uint64_t)(nl - 1) * batch + rows) * X1, 32)))
                return rc;
            g.X = X1;
            g.src_batch = batch;
            // Stages 2-3
            g.Y = Y1;
            g.X4 = 4 * X1;
            g.cols = cols1;
            g.mode = 1;
            g.tw = inverse ? t.tw_inv : t.tw_fwd;
            g.planes = planes;
            rc = (cols1 >= 64 && nt == 64) ? launch_gemm_fused<64>(ctx, src, t.map_b[kind1], g, nl, st)
                                           : launch_gemm_fused<32>(ctx, src, t.map_b32[kind1], g, nl, st);
            if (rc) return rc;
            // Stages 4-5
            g.Y = cols1;
            g.X4 = 4 * Y1;
            g.cols = cols2;
            g.mode = 2;
            g.out = base;
            g.out_limb_stride = (size_t)batch * N;
            rc = (cols2 >= 64 && nt == 64) ? launch_gemm<64>(ctx, *a2, t.map_b[kind2], g, nl, st)
                                           : launch_gemm<32>(ctx, *a2, t.map_b32[kind2], g, nl, st);
            if (rc) return rc;
        }
    }
    return FHE_OK;
}

}  // namespace fhe

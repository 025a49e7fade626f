// Tensor-core NTT (Sec. IV-B Eq. (9) and Sec. IV-C, Stages 1-5) on sm_103a tcgen05.
//
// Four-step form, N = N1 * N2 (N1 = 2^ceil(logN/2), N2 = 2^floor(logN/2)), index maps
// n = N2*n1 + n2 and k = k1 + N1*k2:
//   forward  A[k1 + N1 k2] = sum_n2 w^(n2 k2) psi^((2k1+1) n2) sum_n1 psi^(N2 (2k1+1) n1) a[N2 n1 + n2]
//   inverse  a[N2 n1 + n2] = N^-1 sum_k1 psi^(-N2 (2k1+1) n1) psi^(-(2k1+1) n2) sum_k2 psi^(-2 N1 n2 k2) A[k1 + N1 k2]
// (w = psi^(2 N1)). Each direction is three kernels per chunk of polynomials:
//   split  (Stage 1): u32 residues -> four 8-bit digit planes, transposed so that the
//          reduction index is contiguous (K-major operand);
//   gemm 1 (Stages 2-3): tcgen05 GEMM against the first twiddle matrix; the epilogue rebuilds
//          each output mod q, multiplies by the twiddle and re-splits it into digit planes
//          for the next GEMM (again transposed);
//   gemm 2 (Stages 4-5): tcgen05 GEMM against the second matrix; the epilogue rebuilds mod q
//          and stores natural-order u32 results.
//
// Segment fusion on this GPU: sm_103a has no tcgen05 integer MMA (ptxas rejects kind::i8),
// so the 8-bit segments are carried exactly in bf16 (kind::f16, fp32 accumulation in TMEM).
// Data digits are balanced base-256 digits in [-128, 127]; twiddle-matrix digits are balanced
// base-255 digits in [-127, 127]. The j-th data digit's weight 256^j is folded into the
// constant matrix (W 256^j mod q), so one accumulator per twiddle digit i remains:
//   acc_i = sum_{n, j} d_j(x_n) e_i(W_n 256^j mod q),    y = sum_i 255^i acc_i = W x (mod q).
// |d e| <= 128 * 127 = 16256 and K' = 4K <= 1024 terms keep every partial sum below
// 16,646,144 < 2^24, so the fp32 accumulation is exact (integers below 2^24 are exact).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "common.cuh"
#include "ptx.cuh"

namespace fhe {
namespace {

constexpr int kTileM = 128;
constexpr int kChunk = 64;             // K' elements (bf16) per pipeline stage = 128 bytes
constexpr int kMaxChunkLimbs = 64;
constexpr size_t kPlaneBytes = 256ull << 20;  // each of the two digit-plane scratch buffers

struct GemmArgs {
    int rows;     // polynomials per limb in this launch
    int Y;        // A rows per polynomial
    int X4;       // K' = 4 X
    int cols;     // output columns of the matrix
    int N;
    int mode;     // 1: twiddle + re-split into planes; 2: u32 output
    size_t out_limb_stride;  // mode 2: elements between limbs of `out`
    const uint2* tw;         // mode 1: [nmod][cols][Y]
    uint2* planes;           // mode 1: [limb][rows][cols][Y] groups of four bf16 digits
    uint32_t* out;           // mode 2: first row of the chunk
    int* status;
    uint32_t q[kMaxChunkLimbs];
    uint64_t mu[kMaxChunkLimbs];
    uint64_t off[kMaxChunkLimbs];  // multiple of q above 2^49 that makes the rebuilt value positive
    int mod[kMaxChunkLimbs];
};

__device__ __forceinline__ uint2 split_bf16x4(uint32_t v) {
    int x = (int)v;
    const int d0 = ((x + 128) & 255) - 128;
    x = (x - d0) >> 8;
    const int d1 = ((x + 128) & 255) - 128;
    x = (x - d1) >> 8;
    const int d2 = ((x + 128) & 255) - 128;
    x = (x - d2) >> 8;
    __nv_bfloat162 lo = __floats2bfloat162_rn((float)d0, (float)d1);
    __nv_bfloat162 hi = __floats2bfloat162_rn((float)d2, (float)x);
    return make_uint2(*reinterpret_cast<uint32_t*>(&lo), *reinterpret_cast<uint32_t*>(&hi));
}

// Stage 1: in[limb][poly] viewed as X x Y (row-major) -> planes[limb][poly][Y][X] of four
// bf16 digits each. Block (32, 8) transposes a TS x TS tile (TS = 32 or 64; each thread has
// TS * TS / 256 loads in flight) through shared memory; every thread then writes whole
// 32-byte groups of four consecutive x.
template <int TS>
__global__ void __launch_bounds__(256) tc_split_kernel(const uint32_t* __restrict__ in, uint2* __restrict__ planes,
                                                       int X, int Y, int rows, size_t in_limb_stride, int N) {
    __shared__ uint32_t tile[TS][TS + 1];
    const int z = blockIdx.z;
    const int limb = z / rows, poly = z % rows;
    const uint32_t* src = in + limb * in_limb_stride + (size_t)poly * N;
    const int x0 = blockIdx.y * TS, y0 = blockIdx.x * TS;
    const int tx = threadIdx.x, ty = threadIdx.y;
#pragma unroll
    for (int i = ty; i < TS; i += 8)
#pragma unroll
        for (int h = 0; h < TS / 32; ++h) tile[i][tx + 32 * h] = __ldg(&src[(size_t)(x0 + i) * Y + y0 + tx + 32 * h]);
    __syncthreads();
    constexpr int XG = TS / 4;  // groups of four x per y
    const int t = ty * 32 + tx;
#pragma unroll
    for (int u = t; u < TS * XG; u += 256) {
        const int yy = u / XG, xg = u % XG;
        uint2* dst = planes + ((size_t)z * Y + y0 + yy) * X + x0 + xg * 4;
        const uint2 p0 = split_bf16x4(tile[xg * 4 + 0][yy]), p1 = split_bf16x4(tile[xg * 4 + 1][yy]);
        const uint2 p2 = split_bf16x4(tile[xg * 4 + 2][yy]), p3 = split_bf16x4(tile[xg * 4 + 3][yy]);
        reinterpret_cast<uint4*>(dst)[0] = make_uint4(p0.x, p0.y, p1.x, p1.y);
        reinterpret_cast<uint4*>(dst)[1] = make_uint4(p2.x, p2.y, p3.x, p3.y);
    }
}

// Stages 2-5, persistent: one CTA per SM walks the 128 x NT output tiles of all limbs,
// t = blockIdx.x + k gridDim.x (row tiles fastest, so the CTAs running at one time share their
// B tiles in L2).
// Warp 0 issues the TMA loads through a 4-stage ring, warp 1 issues the MMAs, warps 2-5 run
// the epilogue. The accumulators are double-buffered in TMEM (2 x 4 NT columns), so the MMAs
// of tile k+1 run while the epilogue drains tile k; acc_full[b] / acc_empty[b] hand each
// buffer between the MMA warp and the four epilogue warps. Every wait is bounded.
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
        // the four digit planes of the constant matrix are consecutive rows of one B tile, so
        // a single M=128, N=4*NT MMA per K step fills all four accumulators of buffer lt & 1
        // (its TMEM columns [i*NT, (i+1)*NT) hold acc_i) and reads the A tile once
        constexpr uint32_t idesc = ptx::idesc_bf16(kTileM, 4 * NT);
        bool ok = true;
        long long consumed = 0;
        int lt = 0;
        for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++lt) {
            const int buf = lt & 1;
            if (lt >= 2) ok = ptx::mbar_wait(&acc_empty[buf], (uint32_t)(((lt >> 1) - 1) & 1), a.status, FHE_ETIMEOUT);
            if (!ok) break;
            ptx::tc_fence_after();
            const uint32_t acc = tmem + buf * Cfg::kAccCols;
            for (int c = 0; c < nchunks; ++c, ++consumed) {
                const int s = (int)(consumed % S);
                ok = ptx::mbar_wait(&full[s], (uint32_t)((consumed / S) & 1), a.status, FHE_ETIMEOUT);
                if (!ok) break;
                ptx::tc_fence_after();
                const uint32_t As = ptx::smem_u32(sm + s * Cfg::kStageBytes);
                const uint32_t Bs = As + Cfg::kABytes;
#pragma unroll
                for (int kk = 0; kk < kChunk / 16; ++kk) {
                    const uint64_t adesc = ptx::sdesc_sw128(As + kk * 32);
                    const uint64_t bdesc = ptx::sdesc_sw128(Bs + kk * 32);
                    ptx::mma_bf16(acc, adesc, bdesc, idesc, (c > 0 || kk > 0) ? 1u : 0u);
                }
                ptx::mma_commit(&empty[s]);
            }
            if (ok) ptx::mma_commit(&acc_full[buf]);
        }
        // every MMA issued above has completed before TMEM can be released
        ptx::mma_commit(&drained);
        ptx::mbar_wait(&drained, 0, nullptr, 0);
    } else if (warp >= 2) {
        // ---- epilogue: warp w reads TMEM lanes [32 (w % 4), 32 (w % 4) + 32) = tile rows
        const int quarter = warp & 3;
        int lt = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++lt) {
            const int buf = lt & 1;
            // warp-uniform verdict: the tcgen05.ld below is .sync.aligned
            const bool ok =
                __all_sync(0xffffffffu, ptx::mbar_wait(&acc_full[buf], (uint32_t)((lt >> 1) & 1), a.status, FHE_ETIMEOUT));
            if (!ok) break;
            ptx::tc_fence_after();
            const int mt = t % tiles_m, nt = (t / tiles_m) % tiles_n, z = t / (tiles_m * tiles_n);
            const int n0 = nt * NT;
            const int mrow = mt * kTileM + quarter * 32 + lane;
            const bool valid = mrow < a.rows * a.Y;
            const int poly = mrow / a.Y, y = mrow % a.Y;
            const uint32_t q = a.q[z];
            const uint64_t mu = a.mu[z], off = a.off[z];
            const uint32_t lane_base = tmem + buf * Cfg::kAccCols + ((uint32_t)(quarter * 32) << 16);
            const uint2* twp = a.tw + ((size_t)a.mod[z] * a.cols + n0) * a.Y + y;
            uint2 wnext[16];
            if (a.mode == 1 && valid) {
#pragma unroll
                for (int j = 0; j < 16; ++j) wnext[j] = __ldg(&twp[(size_t)j * a.Y]);
            }
#pragma unroll 1
            for (int cb = 0; cb < NT / 16; ++cb) {
                uint32_t r[4][16];
                uint2 wcur[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) wcur[j] = wnext[j];
                if (a.mode == 1 && valid && cb + 1 < NT / 16) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) wnext[j] = __ldg(&twp[(size_t)((cb + 1) * 16 + j) * a.Y]);
                }
#pragma unroll
                for (int i = 0; i < 4; ++i) ptx::tmem_ld16(lane_base + i * NT + cb * 16, r[i]);
                ptx::tmem_wait_ld();
                if (!valid) continue;
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int col = n0 + cb * 16 + j;
                    const long long a0 = __float2int_rn(__uint_as_float(r[0][j]));
                    const long long a1 = __float2int_rn(__uint_as_float(r[1][j]));
                    const long long a2 = __float2int_rn(__uint_as_float(r[2][j]));
                    const long long a3 = __float2int_rn(__uint_as_float(r[3][j]));
                    const long long yv = a0 + 255 * a1 + 65025 * a2 + 16581375 * a3;
                    uint32_t v = reduce_u64((uint64_t)(yv + (long long)off), mu, q);
                    if (a.mode == 1) {
                        v = mul_shoup(v, wcur[j].x, wcur[j].y, q);
                        a.planes[(((size_t)z * a.rows + poly) * a.cols + col) * a.Y + y] = split_bf16x4(v);
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

// 2-D bf16 tensor map over a row-major [rows][inner] array, box = 64 x box_rows, 128B swizzle.
int make_map(CUtensorMap* m, const void* base, uint64_t inner, uint64_t rows, uint32_t box_rows) {
    auto fn = encode_fn();
    if (!fn) return set_error(FHE_ECUDA, "cuTensorMapEncodeTiled is unavailable");
    cuuint64_t dims[2] = {inner, rows};
    cuuint64_t strides[1] = {inner * 2};
    cuuint32_t box[2] = {(cuuint32_t)kChunk, box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(FHE_ECUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
    return FHE_OK;
}

uint16_t bf16_bits_of_small_int(int e) {
    float f = (float)e;
    uint32_t b;
    memcpy(&b, &f, 4);
    return (uint16_t)(b >> 16);  // exact: |e| <= 256 has at most 8 significant bits
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
    if (!ctx->tc_planes[0]) {
        if ((rc = dev_alloc(ctx, (uint8_t**)&ctx->tc_planes[0], kPlaneBytes))) return rc;
        if ((rc = dev_alloc(ctx, (uint8_t**)&ctx->tc_planes[1], kPlaneBytes))) return rc;
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
                                bf16_bits_of_small_int(dg[i]);
                    }
                }
        }
        if ((rc = dev_upload(ctx, &t.mat[kind], h))) return rc;
        if ((rc = make_map(&t.map_b[kind], t.mat[kind], (uint64_t)4 * K, (uint64_t)nmod * 4 * cols,
                           cols >= 64 ? 64 : 32)))
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
    // operand maps over the plane buffers: [rows][4X] for X = n1 and X = n2
    const uint64_t cap_n1 = kPlaneBytes / 2 / (4ull * n1), cap_n2 = kPlaneBytes / 2 / (4ull * n2);
    for (int p = 0; p < 2; ++p) {
        if ((rc = make_map(&t.map_a[p][0], ctx->tc_planes[p], 4ull * n1, cap_n1, kTileM))) return rc;
        if ((rc = make_map(&t.map_a[p][1], ctx->tc_planes[p], 4ull * n2, cap_n2, kTileM))) return rc;
    }
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

int ntt_tc(const fhe_ctx* cctx, uint32_t logN, bool inverse, uint32_t* d, int n_limbs, int batch,
           const LimbMap& map, cudaStream_t st) {
    fhe_ctx* ctx = const_cast<fhe_ctx*>(cctx);
    {
        std::lock_guard<std::mutex> lock(g_tc_mu);
        int rc = build_tc_tables(ctx, logN);
        if (rc) return rc;
    }
    const TcTables& t = ctx->tc[logN];
    const int n1 = t.n1, n2 = t.n2;
    const size_t N = (size_t)1 << logN;
    // X: first-GEMM reduction size, Y: its rows per polynomial; the second GEMM swaps them.
    const int X1 = inverse ? n2 : n1, Y1 = inverse ? n1 : n2;
    const int cols1 = inverse ? n2 : n1, cols2 = inverse ? n1 : n2;
    const int kind1 = inverse ? 2 : 0, kind2 = inverse ? 3 : 1;
    const size_t cap_polys = kPlaneBytes / (N * 8);  // bf16 x 4 digits per residue
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
            // Stage 1
            if (X1 >= 64 && Y1 >= 64) {
                dim3 sg(Y1 / 64, X1 / 64, nl * rows);
                tc_split_kernel<64><<<sg, dim3(32, 8), 0, st>>>(base, (uint2*)ctx->tc_planes[0], X1, Y1, rows,
                                                                (size_t)batch * N, (int)N);
            } else {
                dim3 sg(Y1 / 32, X1 / 32, nl * rows);
                tc_split_kernel<32><<<sg, dim3(32, 8), 0, st>>>(base, (uint2*)ctx->tc_planes[0], X1, Y1, rows,
                                                                (size_t)batch * N, (int)N);
            }
            FHE_CUDA_TRY(cudaGetLastError());
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
            // Stages 2-3
            g.Y = Y1;
            g.X4 = 4 * X1;
            g.cols = cols1;
            g.mode = 1;
            g.tw = inverse ? t.tw_inv : t.tw_fwd;
            g.planes = (uint2*)ctx->tc_planes[1];
            const CUtensorMap& a1 = t.map_a[0][inverse ? 1 : 0];
            rc = cols1 >= 64 ? launch_gemm<64>(ctx, a1, t.map_b[kind1], g, nl, st)
                             : launch_gemm<32>(ctx, a1, t.map_b[kind1], g, nl, st);
            if (rc) return rc;
            // Stages 4-5
            g.Y = cols1;
            g.X4 = 4 * Y1;
            g.cols = cols2;
            g.mode = 2;
            g.out = base;
            g.out_limb_stride = (size_t)batch * N;
            const CUtensorMap& a2 = t.map_a[1][inverse ? 0 : 1];
            rc = cols2 >= 64 ? launch_gemm<64>(ctx, a2, t.map_b[kind2], g, nl, st)
                             : launch_gemm<32>(ctx, a2, t.map_b[kind2], g, nl, st);
            if (rc) return rc;
        }
    }
    return FHE_OK;
}

}  // namespace fhe

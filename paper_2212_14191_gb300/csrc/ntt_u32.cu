// Plain 32-bit negacyclic NTT / INTT on CUDA cores (the comparison path of Sec. IV-B;
// butterflies as in Sec. II-A, Fig. 1: Cooley-Tukey forward, Gentleman-Sande inverse).
//
// Transform (Eq. (4)):  A_k = sum_n a_n psi^((2k+1) n) mod q, natural order in and out.
//
// Design (GB300): one polynomial limb is transformed by a cluster of C = N / 2^14 CTAs
// (C = 1 for N <= 2^14) that keep the whole limb in shared memory, so each limb is read
// from and written to HBM exactly once. With T = N / (32 C) threads per CTA every thread
// owns 32 residues and runs the butterflies of up to five consecutive stages in
// registers ("rounds"):
//   cross round (C > 1): the first log2(C) stages couple the C quarters of the limb; CTA c
//       loads the same 1/C^2 slice of every quarter, applies them, and stores quarter q into
//       CTA q's shared memory through distributed shared memory;
//   round A: stages with stride >= T   (thread holds p = tid + T*e,            e < 32)
//   round B: stages with stride 32..T/2 (thread holds p = T*g + lane + 32*e)
//   round C: the last five stages      (thread holds p = 32*rev(tid) + e,      e < 32)
// After round C thread tid holds outputs k = rev5(e)*T + tid, so the bit-reversal that
// the merged Cooley-Tukey form leaves (output position p holds A_bitrev(p)) becomes a
// coalesced store; with C > 1 the final quarter interleave goes through DSMEM.
// Shared memory is XOR-swizzled (p ^ ((p >> log2 T) & 31)) so every round and the
// bit-reversed store are free of bank conflicts.
// Arithmetic: Harvey's lazy butterflies with Shoup's precomputed-quotient multiplication;
// forward values live in [0, 4q), inverse values in [0, 2q), q < 2^30.
#include <cooperative_groups.h>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace fhe {
namespace {

struct NttArgs {
    uint32_t* data;
    int rows;   // n_limbs * batch
    int batch;
    const uint2* tw;    // [nmod][N]
    const uint2* twC;   // [nmod][C][31][T]
    const uint2* ninv;  // [nmod]
    LimbMap map;
};

template <int BITS>
__device__ __forceinline__ uint32_t rev_bits(uint32_t x) {
    return __brev(x) >> (32 - BITS);
}

template <int LOG_T>
__device__ __forceinline__ int swz(int p) {
    return p ^ ((p >> LOG_T) & 31);
}

// Forward Cooley-Tukey butterfly (Harvey): x, y in [0, 4q) -> [0, 4q).
__device__ __forceinline__ void ct_bfly(uint32_t& x, uint32_t& y, uint2 w, uint32_t q) {
    uint32_t x2 = csub(x, 2 * q);
    uint32_t t = mul_shoup_lazy(y, w.x, w.y, q);
    x = x2 + t;
    y = x2 - t + 2 * q;
}

// Inverse Gentleman-Sande butterfly (Harvey): x, y in [0, 2q) -> [0, 2q).
__device__ __forceinline__ void gs_bfly(uint32_t& x, uint32_t& y, uint2 w, uint32_t q) {
    uint32_t s = csub(x + y, 2 * q);
    uint32_t d = x - y + 2 * q;
    x = s;
    y = mul_shoup_lazy(d, w.x, w.y, q);
}

// Blocks per SM the register budget is sized for: at most 128 registers per thread.
template <int LOG_T>
constexpr int kMinBlocks = (1 << (14 - LOG_T)) / 32 > 0 ? (1 << (14 - LOG_T)) / 32 : 1;

__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n"
                 "barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

template <int LOG_T, int LOG_C>
__global__ void __launch_bounds__(1 << LOG_T, kMinBlocks<LOG_T>)
ntt_fwd_kernel(NttArgs a) {
    constexpr int T = 1 << LOG_T, C = 1 << LOG_C;
    constexpr int LOG_NC = LOG_T + 5, NC = 1 << LOG_NC;
    constexpr int N = NC * C;
    constexpr int RB = LOG_T - 5;
    extern __shared__ uint32_t sm[];
    const int tid = threadIdx.x;
    const int c = (C > 1) ? (int)blockIdx.x : 0;
    cg::cluster_group cluster = cg::this_cluster();

    for (int row = blockIdx.y; row < a.rows; row += gridDim.y) {
        const int limb = row / a.batch;
        const uint32_t q = a.map.q[limb];
        const int mod = a.map.mod[limb];
        const uint2* tw = a.tw + (size_t)mod * N;
        uint32_t* data = a.data + (size_t)row * N;
        uint32_t v[32];

        if constexpr (C > 1) {
            cluster_sync_all();  // peers resident; previous row's remote reads finished
            constexpr int PER = NC / C;  // elements of each quarter handled by this CTA
#pragma unroll
            for (int u = 0; u < PER / T; ++u) {
                const int jj = c * PER + u * T + tid;
                uint32_t x[C];
#pragma unroll
                for (int qq = 0; qq < C; ++qq) x[qq] = __ldg(&data[jj + qq * NC]);
#pragma unroll
                for (int s = 0; s < LOG_C; ++s) {
                    const int tq = C >> (s + 1);
#pragma unroll
                    for (int qq = 0; qq < C; ++qq) {
                        if ((qq / tq) % 2 == 0) {
                            uint2 w = __ldg(&tw[(1 << s) + qq / (2 * tq)]);
                            ct_bfly(x[qq], x[qq + tq], w, q);
                        }
                    }
                }
#pragma unroll
                for (int qq = 0; qq < C; ++qq) {
                    uint32_t* dst = cluster.map_shared_rank(sm, qq);
                    dst[swz<LOG_T>(jj)] = x[qq];
                }
            }
            cluster_sync_all();
#pragma unroll
            for (int e = 0; e < 32; ++e) v[e] = sm[swz<LOG_T>(tid + T * e)];
        } else {
#pragma unroll
            for (int e = 0; e < 32; ++e) v[e] = __ldg(&data[tid + T * e]);
        }

        // ---- round A: 5 stages, element e at p = tid + T*e
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const int half = 16 >> k;
#pragma unroll
            for (int e = 0; e < 32; ++e) {
                if ((e & half) == 0) {
                    uint2 w = __ldg(&tw[(1 << k) * (C + c) + (e >> (5 - k))]);
                    ct_bfly(v[e], v[e + half], w, q);
                }
            }
        }
#pragma unroll
        for (int e = 0; e < 32; ++e) sm[swz<LOG_T>(tid + T * e)] = v[e];
        __syncthreads();

        // ---- round B: RB stages on groups (g, lane): p = T*g + lane + 32*e, e < 2^RB
        if constexpr (RB > 0) {
            constexpr int GPT = 32 >> RB;  // groups per thread (= 1024 / T)
            constexpr int EG = 1 << RB;    // elements per group
            const int lane = tid & 31, w_ = tid >> 5;
#pragma unroll
            for (int gi = 0; gi < GPT; ++gi) {
                const int g = w_ * GPT + gi;
                uint32_t* vv = v + gi * EG;
#pragma unroll
                for (int e = 0; e < EG; ++e) vv[e] = sm[swz<LOG_T>(T * g + lane + 32 * e)];
#pragma unroll
                for (int k = 0; k < RB; ++k) {
                    const int half = EG >> (k + 1);
#pragma unroll
                    for (int e = 0; e < EG; ++e) {
                        if ((e & half) == 0) {
                            uint2 w = __ldg(&tw[(1 << k) * (32 * (C + c) + g) + (e >> (RB - k))]);
                            ct_bfly(vv[e], vv[e + half], w, q);
                        }
                    }
                }
            }
            __syncthreads();
#pragma unroll
            for (int gi = 0; gi < GPT; ++gi) {
                const int g = w_ * GPT + gi;
                uint32_t* vv = v + gi * EG;
#pragma unroll
                for (int e = 0; e < EG; ++e) sm[swz<LOG_T>(T * g + lane + 32 * e)] = vv[e];
            }
            __syncthreads();
        }

        // ---- round C: last 5 stages on 32 contiguous elements p = 32*gidx + e
        {
            const int gidx = rev_bits<LOG_T>(tid);
#pragma unroll
            for (int e = 0; e < 32; ++e) v[e] = sm[swz<LOG_T>(32 * gidx + e)];
            const uint2* twc = a.twC + (((size_t)mod * C + c) * 31) * T + tid;
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                const int half = 16 >> k;
#pragma unroll
                for (int e = 0; e < 32; ++e) {
                    if ((e & half) == 0) {
                        uint2 w = __ldg(&twc[(size_t)((1 << k) - 1 + (e >> (5 - k))) * T]);
                        ct_bfly(v[e], v[e + half], w, q);
                    }
                }
            }
#pragma unroll
            for (int e = 0; e < 32; ++e) v[e] = csub(csub(v[e], 2 * q), q);
        }

        if constexpr (C == 1) {
#pragma unroll
            for (int e = 0; e < 32; ++e) data[rev_bits<5>(e) * T + tid] = v[e];
            __syncthreads();  // sm is rewritten by the next row's round A
        } else {
            __syncthreads();  // every thread has read its round-C inputs
#pragma unroll
            for (int e = 0; e < 32; ++e) sm[swz<LOG_T>(rev_bits<5>(e) * T + tid)] = v[e];
            cluster_sync_all();
            // CTA c writes k in [c*NC, (c+1)*NC); k lives in CTA rev(k mod C) at k / C.
#pragma unroll 8
            for (int u = 0; u < 32; ++u) {
                const int k = c * NC + u * T + tid;
                const int own = rev_bits<LOG_C>(k & (C - 1));
                const uint32_t* src = cluster.map_shared_rank(sm, own);
                data[k] = src[swz<LOG_T>(k >> LOG_C)];
            }
        }
    }
    if constexpr (C > 1) cluster_sync_all();  // peers may still read this CTA's sm
}

template <int LOG_T, int LOG_C>
__global__ void __launch_bounds__(1 << LOG_T, kMinBlocks<LOG_T>)
ntt_inv_kernel(NttArgs a) {
    constexpr int T = 1 << LOG_T, C = 1 << LOG_C;
    constexpr int LOG_NC = LOG_T + 5, NC = 1 << LOG_NC;
    constexpr int N = NC * C;
    constexpr int RB = LOG_T - 5;
    extern __shared__ uint32_t sm[];
    const int tid = threadIdx.x;
    const int c = (C > 1) ? (int)blockIdx.x : 0;
    cg::cluster_group cluster = cg::this_cluster();

    for (int row = blockIdx.y; row < a.rows; row += gridDim.y) {
        const int limb = row / a.batch;
        const uint32_t q = a.map.q[limb];
        const int mod = a.map.mod[limb];
        const uint2* tw = a.tw + (size_t)mod * N;
        uint32_t* data = a.data + (size_t)row * N;
        uint32_t v[32];

        // ---- load in bit-reversed order: thread tid gets k_local = rev5(e)*T + tid
        if constexpr (C > 1) {
            cluster_sync_all();
#pragma unroll 8
            for (int u = 0; u < 32; ++u) {
                const int k = c * NC + u * T + tid;
                const int own = rev_bits<LOG_C>(k & (C - 1));
                uint32_t* dst = cluster.map_shared_rank(sm, own);
                dst[swz<LOG_T>(k >> LOG_C)] = __ldg(&data[k]);
            }
            cluster_sync_all();
#pragma unroll
            for (int e = 0; e < 32; ++e) v[e] = sm[swz<LOG_T>(rev_bits<5>(e) * T + tid)];
            __syncthreads();  // sm is rewritten below at round-C positions
        } else {
#pragma unroll
            for (int e = 0; e < 32; ++e) v[e] = __ldg(&data[rev_bits<5>(e) * T + tid]);
        }

        // ---- round C': first 5 GS stages (t = 1..16) on p = 32*gidx + e
        {
            const int gidx = rev_bits<LOG_T>(tid);
            const uint2* twc = a.twC + (((size_t)mod * C + c) * 31) * T + tid;
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                const int half = 1 << k;
                const int kf = 4 - k;  // the matching forward stage inside the round
#pragma unroll
                for (int e = 0; e < 32; ++e) {
                    if ((e & half) == 0) {
                        uint2 w = __ldg(&twc[(size_t)((1 << kf) - 1 + (e >> (5 - kf))) * T]);
                        gs_bfly(v[e], v[e + half], w, q);
                    }
                }
            }
#pragma unroll
            for (int e = 0; e < 32; ++e) sm[swz<LOG_T>(32 * gidx + e)] = v[e];
            __syncthreads();
        }

        // ---- round B'
        if constexpr (RB > 0) {
            constexpr int GPT = 32 >> RB;
            constexpr int EG = 1 << RB;
            const int lane = tid & 31, w_ = tid >> 5;
#pragma unroll
            for (int gi = 0; gi < GPT; ++gi) {
                const int g = w_ * GPT + gi;
                uint32_t* vv = v + gi * EG;
#pragma unroll
                for (int e = 0; e < EG; ++e) vv[e] = sm[swz<LOG_T>(T * g + lane + 32 * e)];
#pragma unroll
                for (int k = RB - 1; k >= 0; --k) {
                    const int half = EG >> (k + 1);
#pragma unroll
                    for (int e = 0; e < EG; ++e) {
                        if ((e & half) == 0) {
                            uint2 w = __ldg(&tw[(1 << k) * (32 * (C + c) + g) + (e >> (RB - k))]);
                            gs_bfly(vv[e], vv[e + half], w, q);
                        }
                    }
                }
            }
            __syncthreads();
#pragma unroll
            for (int gi = 0; gi < GPT; ++gi) {
                const int g = w_ * GPT + gi;
                uint32_t* vv = v + gi * EG;
#pragma unroll
                for (int e = 0; e < EG; ++e) sm[swz<LOG_T>(T * g + lane + 32 * e)] = vv[e];
            }
            __syncthreads();
        }

        // ---- round A'
#pragma unroll
        for (int e = 0; e < 32; ++e) v[e] = sm[swz<LOG_T>(tid + T * e)];
#pragma unroll
        for (int k = 4; k >= 0; --k) {
            const int half = 16 >> k;
#pragma unroll
            for (int e = 0; e < 32; ++e) {
                if ((e & half) == 0) {
                    uint2 w = __ldg(&tw[(1 << k) * (C + c) + (e >> (5 - k))]);
                    gs_bfly(v[e], v[e + half], w, q);
                }
            }
        }
        const uint2 ni = __ldg(&a.ninv[mod]);
        if constexpr (C == 1) {
#pragma unroll
            for (int e = 0; e < 32; ++e) data[tid + T * e] = mul_shoup(v[e], ni.x, ni.y, q);
            __syncthreads();
        } else {
            __syncthreads();
#pragma unroll
            for (int e = 0; e < 32; ++e) sm[swz<LOG_T>(tid + T * e)] = v[e];
            cluster_sync_all();
            constexpr int PER = NC / C;
#pragma unroll
            for (int u = 0; u < PER / T; ++u) {
                const int jj = c * PER + u * T + tid;
                uint32_t x[C];
#pragma unroll
                for (int qq = 0; qq < C; ++qq) {
                    const uint32_t* src = cluster.map_shared_rank(sm, qq);
                    x[qq] = src[swz<LOG_T>(jj)];
                }
#pragma unroll
                for (int s = LOG_C - 1; s >= 0; --s) {
                    const int tq = C >> (s + 1);
#pragma unroll
                    for (int qq = 0; qq < C; ++qq) {
                        if ((qq / tq) % 2 == 0) {
                            uint2 w = __ldg(&tw[(1 << s) + qq / (2 * tq)]);
                            gs_bfly(x[qq], x[qq + tq], w, q);
                        }
                    }
                }
#pragma unroll
                for (int qq = 0; qq < C; ++qq) data[jj + qq * NC] = mul_shoup(x[qq], ni.x, ni.y, q);
            }
        }
    }
    if constexpr (C > 1) cluster_sync_all();
}

template <int LOG_T, int LOG_C>
int launch(const fhe_ctx* ctx, const NttTables& t, bool inverse, uint32_t* d, int rows,
           int batch, const LimbMap& map, cudaStream_t stream) {
    constexpr int T = 1 << LOG_T, C = 1 << LOG_C;
    constexpr int smem = (T * 32) * 4;
    NttArgs args;
    args.data = d;
    args.rows = rows;
    args.batch = batch;
    args.tw = inverse ? t.inv : t.fwd;
    args.twC = inverse ? t.invC : t.fwdC;
    args.ninv = t.ninv;
    args.map = map;
    void (*kern)(NttArgs) = inverse ? ntt_inv_kernel<LOG_T, LOG_C> : ntt_fwd_kernel<LOG_T, LOG_C>;
    FHE_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    if (C > 1) FHE_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    // rows beyond the grid are looped over; size the grid to a few waves of the GPU
    int per_sm = (LOG_T >= 9) ? 2 : 4;
    int max_rows = ctx->num_sms * per_sm * 8 / C;
    if (max_rows < 1) max_rows = 1;
    int gy = rows < max_rows ? rows : max_rows;
    if (gy > 65535) gy = 65535;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C, gy, 1);
    cfg.blockDim = dim3(T, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    FHE_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, args));
    return FHE_OK;
}

uint32_t rev_h(uint32_t x, int bits) {
    uint32_t r = 0;
    for (int i = 0; i < bits; ++i) r |= ((x >> i) & 1u) << (bits - 1 - i);
    return r;
}

void ntt_shape(uint32_t logN, int* log_t, int* log_c) {
    *log_c = logN > 14 ? (int)logN - 14 : 0;
    *log_t = (int)logN - 5 - *log_c;
}

}  // namespace

int build_ntt_tables(fhe_ctx* ctx, uint32_t logN) {
    const int nmod = (int)ctx->mods.size();
    const uint32_t N = 1u << logN;
    int log_t, log_c;
    ntt_shape(logN, &log_t, &log_c);
    const int T = 1 << log_t, C = 1 << log_c;
    std::vector<uint2> fwd((size_t)nmod * N), inv((size_t)nmod * N);
    std::vector<uint2> fwdC((size_t)nmod * C * 31 * T), invC((size_t)nmod * C * 31 * T);
    std::vector<uint2> ninv(nmod);
    for (int m = 0; m < nmod; ++m) {
        const uint32_t q = ctx->mods[m];
        const uint32_t psi = root_2n(q, logN);
        const uint32_t psi_inv = invmod_h(psi, q);
        std::vector<uint32_t> pw(N), pwi(N);
        uint32_t a = 1, b = 1;
        for (uint32_t i = 0; i < N; ++i) {
            pw[i] = a;
            pwi[i] = b;
            a = mulmod_h(a, psi, q);
            b = mulmod_h(b, psi_inv, q);
        }
        for (uint32_t i = 0; i < N; ++i) {
            uint32_t r = rev_h(i, (int)logN);
            fwd[(size_t)m * N + i] = make_uint2(pw[r], shoup_h(pw[r], q));
            inv[(size_t)m * N + i] = make_uint2(pwi[r], shoup_h(pwi[r], q));
        }
        // last-round tables: thread tid of CTA c, entry (2^k - 1 + b) holds
        // tw[2^k * ((C + c) * T + rev(tid)) + b]
        for (int c = 0; c < C; ++c)
            for (int tid = 0; tid < T; ++tid) {
                uint32_t gidx = rev_h((uint32_t)tid, log_t);
                for (int k = 0; k < 5; ++k)
                    for (int bb = 0; bb < (1 << k); ++bb) {
                        size_t idx = (size_t)(1u << k) * ((uint32_t)(C + c) * T + gidx) + bb;
                        size_t dst = (((size_t)m * C + c) * 31 + ((1 << k) - 1 + bb)) * T + tid;
                        fwdC[dst] = fwd[(size_t)m * N + idx];
                        invC[dst] = inv[(size_t)m * N + idx];
                    }
            }
        uint32_t ni = invmod_h(N % q, q);
        ninv[m] = make_uint2(ni, shoup_h(ni, q));
    }
    NttTables& t = ctx->ntt[logN];
    int rc;
    if ((rc = dev_upload(ctx, &t.fwd, fwd))) return rc;
    if ((rc = dev_upload(ctx, &t.inv, inv))) return rc;
    if ((rc = dev_upload(ctx, &t.fwdC, fwdC))) return rc;
    if ((rc = dev_upload(ctx, &t.invC, invC))) return rc;
    if ((rc = dev_upload(ctx, &t.ninv, ninv))) return rc;
    return FHE_OK;
}

int ntt_u32(const fhe_ctx* ctx, uint32_t logN, bool inverse, uint32_t* d, int n_limbs, int batch,
            const LimbMap& map, cudaStream_t stream) {
    const NttTables& t = ctx->ntt[logN];
    if (!t.fwd) return set_error(FHE_EINVAL, "no NTT tables for this logN");
    const long long rows = (long long)n_limbs * batch;
    if (rows == 0) return FHE_OK;
    if (rows > (1LL << 30)) return set_error(FHE_EINVAL, "too many rows");
    switch (logN) {
        case 10: return launch<5, 0>(ctx, t, inverse, d, (int)rows, batch, map, stream);
        case 11: return launch<6, 0>(ctx, t, inverse, d, (int)rows, batch, map, stream);
        case 12: return launch<7, 0>(ctx, t, inverse, d, (int)rows, batch, map, stream);
        case 13: return launch<8, 0>(ctx, t, inverse, d, (int)rows, batch, map, stream);
        case 14: return launch<9, 0>(ctx, t, inverse, d, (int)rows, batch, map, stream);
        case 15: return launch<9, 1>(ctx, t, inverse, d, (int)rows, batch, map, stream);
        case 16: return launch<9, 2>(ctx, t, inverse, d, (int)rows, batch, map, stream);
        default: return set_error(FHE_EINVAL, "logN out of range");
    }
}

}  // namespace fhe

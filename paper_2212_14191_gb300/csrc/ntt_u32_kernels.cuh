// Kernels of the plain 32-bit negacyclic NTT / INTT on CUDA cores (the comparison path of Sec. IV-B;
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
// Shared memory uses a padded layout (PadLayout: p + p/32 + p/T) under which every round and
// the bit-reversed store are free of bank conflicts and every access is a per-thread base
// plus a compile-time offset (no per-access address arithmetic).
// Arithmetic: Harvey's lazy butterflies with Shoup's precomputed-quotient multiplication;
// forward values live in [0, 4q), inverse values in [0, 2q), q < 2^30.

#pragma once
#include "common.cuh"
#include "ptx.cuh"

#include <string.h>


namespace fhe {
namespace {

struct NttArgs {
    uint32_t* data;
    int rows;   // n_limbs * batch
    int batch;
    const uint2* tw;    // [nmod][N]
    const uint2* twC;   // [nmod][C][31][T]
    const uint2* ninv;  // [nmod]
    const uint2* ninv_w1;  // [nmod] N^-1 tw[1] (the single-CTA inverse's last stage, scaling folded in)
    int* status;        // device error word (FHE_ETIMEOUT on an expired wait)
    int contiguous;     // row order: 0 = interleaved across clusters, 1 = contiguous ranges
    const RowRef* rowtab;    // if set: row r is rowtab[r] (any buffer, any modulus) ...
    const uint32_t* mod_q;   // ... with modulus mod_q[rowtab[r].mod]; `data`/`map` unused
    LimbMap map;
};

// Data pointer, modulus and modulus index of a row.
template <int N>
__device__ __forceinline__ uint32_t* row_ref(const NttArgs& a, int row, uint32_t* q, int* mod) {
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

template <int N>
__device__ __forceinline__ uint32_t* row_ptr(const NttArgs& a, int row) {
    return a.rowtab ? a.rowtab[row].ptr : a.data + (size_t)row * N;
}

template <int BITS>
__device__ __forceinline__ uint32_t rev_bits(uint32_t x) {
    return __brev(x) >> (32 - BITS);
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

// First stages on canonical residues (below q), as loaded from a row: the forward's x needs no
// reduction below 2q and the inverse's x + y is already below 2q.
__device__ __forceinline__ void ct_bfly_first(uint32_t& x, uint32_t& y, uint2 w, uint32_t q) {
    uint32_t t = mul_shoup_lazy(y, w.x, w.y, q);
    uint32_t x0 = x;
    x = x0 + t;
    y = x0 - t + 2 * q;
}
__device__ __forceinline__ void gs_bfly_first(uint32_t& x, uint32_t& y, uint2 w, uint32_t q) {
    uint32_t s = x + y;
    uint32_t d = x - y + 2 * q;
    x = s;
    y = mul_shoup_lazy(d, w.x, w.y, q);
}

// Blocks per SM the register budget is sized for: at most 128 registers per thread; kernels
// built with OCC = 2 are capped at 64 registers so that twice as many CTAs share an SM.
template <int LOG_T>
constexpr int kMinBlocks = (1 << (14 - LOG_T)) / 32 > 0 ? (1 << (14 - LOG_T)) / 32 : 1;

// Shared memory (32-bit words) of a CTA: a working buffer holding its 32 * T residues in the
// padded layout and,
// with push exchange in a cluster, a receive buffer that peers store their outputs into.
// It is kept this small on purpose: the rest of the SM's 256 KB L1/shared array caches
// twiddle tables.
template <int LOG_T, int LOG_C, bool PUSH>
constexpr int kSmemWords = PadLayout<LOG_T>::kWords + ((LOG_C > 0 && PUSH) ? (32 << LOG_T) : 0);

// Round-C twiddles of one thread: its column (stride T) of the [31][T] last-round table,
// read from global memory through L1 or, with TWS, from a copy in this CTA's shared memory
// (after the working buffers) refreshed whenever the row's modulus changes. TWS kernels run
// their rows in contiguous ranges, so a CTA reloads its 31 * T * 8 bytes only when a range
// crosses a limb boundary. Every thread copies and reads only its own column, so a refresh
// needs no barrier: the thread's asynchronous copies complete at its `ready()`.
template <int LOG_T, bool TWS>
struct TwCol {
    const uint2* g;
    uint2* s;
    int have;
    __device__ __forceinline__ void refresh(const uint2* col, int mod) {
        g = col;
        if constexpr (TWS) {
            if (mod != have) {
#pragma unroll
                for (int j = 0; j < 31; ++j) ptx::cp_async8(s + (j << LOG_T), col + ((size_t)j << LOG_T));
                ptx::cp_async_commit();
                have = mod;
            }
        }
    }
    __device__ __forceinline__ void ready() const {
        if constexpr (TWS) ptx::cp_async_wait_all();
    }
    __device__ __forceinline__ uint2 operator[](int j) const {
        if constexpr (TWS)
            return s[j << LOG_T];
        else
            return __ldg(&g[(size_t)j << LOG_T]);
    }
};

template <int LOG_T, int LOG_C, bool PUSH, bool TWS>
constexpr int kSmemTotalWords = kSmemWords<LOG_T, LOG_C, PUSH> + (TWS ? (62 << LOG_T) : 0);

// Swizzle of the receive buffer: forward pushes arrive at stride C words per lane.
template <int LOG_C>
__device__ __forceinline__ int swo(int off) {
    return off ^ ((off >> 5) & ((1 << LOG_C) - 1));
}

// Rows handled by this cluster: interleaved (row = blockIdx.y + i * gridDim.y, so the
// clusters running at one time share a limb and its twiddle tables in L2) or one contiguous
// range (consecutive rows of a cluster share a limb, favouring L1).
struct RowIter {
    int row, end, step;
};
__device__ __forceinline__ RowIter row_iter(int rows, int contiguous) {
    if (contiguous) {
        const int per = (rows + gridDim.y - 1) / gridDim.y;
        const int b = min(rows, (int)blockIdx.y * per);
        return {b, min(rows, b + per), 1};
    }
    return {(int)blockIdx.y, rows, (int)gridDim.y};
}

// Ask the TMA unit to pull this CTA's share of a row into L2 ahead of its loads:
// forward with C > 1, the slice [c*PER, (c+1)*PER) of each of the C quarters; otherwise the
// CTA's contiguous range [c*NC, (c+1)*NC).
template <int LOG_T, int LOG_C, bool FWD>
__device__ __forceinline__ void prefetch_row(const uint32_t* data_row, int c) {
    constexpr int T = 1 << LOG_T, C = 1 << LOG_C;
    constexpr int NC = 32 * T;
    if (FWD && C > 1) {
        constexpr int PER = NC / C;
#pragma unroll
        for (int qq = 0; qq < C; ++qq) ptx::prefetch_l2(data_row + qq * NC + c * PER, PER * 4);
    } else {
        ptx::prefetch_l2(data_row + c * NC, NC * 4);
    }
}

template <int LOG_T, int LOG_C, bool PUSH, bool TWS, int OCC>
__global__ void __launch_bounds__(1 << LOG_T, kMinBlocks<LOG_T> * OCC)
ntt_fwd_kernel(const NttArgs a) {
    constexpr int T = 1 << LOG_T, C = 1 << LOG_C;
    constexpr int LOG_NC = LOG_T + 5, NC = 1 << LOG_NC;
    constexpr int N = NC * C;
    constexpr int RB = LOG_T - 5;
    extern __shared__ __align__(128) uint32_t work[];
    const uint32_t work_s = ptx::smem_u32(work);
    const int tid = threadIdx.x;
    const int c = (C > 1) ? (int)blockIdx.x : 0;
    using L = PadLayout<LOG_T>;
    static_assert(C == 1 || (T >> LOG_C) >= 32, "cluster exchange offsets need T / C >= 32");
    const int pA = L::pad(tid);                             // p = tid + T e
    const int pX = L::pad(c * (NC / C) + tid);              // p = c NC / C + tid + T u
    const int pK = L::pad((c * NC + tid) >> LOG_C);         // p = (c NC + u T + tid) / C
    const RowIter ri = row_iter(a.rows, a.contiguous);
    TwCol<LOG_T, TWS> twc{nullptr, reinterpret_cast<uint2*>(work + kSmemWords<LOG_T, LOG_C, PUSH>) + tid, -1};
    if constexpr (C > 1) ptx::cluster_sync();  // every peer is resident before the first push

    for (int row = ri.row; row < ri.end; row += ri.step) {
        uint32_t q;
        int mod;
        uint32_t* data = row_ref<N>(a, row, &q, &mod);
        const uint2* tw = a.tw + (size_t)mod * N;
        twc.refresh(a.twC + (((size_t)mod * C + c) * 31) * T + tid, mod);
        if (tid == 0 && row + ri.step < ri.end) prefetch_row<LOG_T, LOG_C, true>(row_ptr<N>(a, row + ri.step), c);
        uint32_t v[32];

        if constexpr (C > 1) {
            // push: peers finished reading their `work` before the previous row's second
            // barrier; pull: peers may still be reading this CTA's `work` (gather)
            if constexpr (!PUSH) {
                // only orders the peers' completed DSMEM reads before these writes
                __syncwarp();
                ptx::cluster_arrive_relaxed();
                ptx::cluster_wait();
            }
            constexpr int PER = NC / C;  // elements of each quarter handled by this CTA
            constexpr int U = PER / T;   // = 32 / C slices per thread
            // all 32 global loads first (v is free here), then the butterflies and pushes
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int qq = 0; qq < C; ++qq) v[u * C + qq] = __ldg(&data[c * PER + u * T + tid + qq * NC]);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                uint32_t* x = v + u * C;
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
                for (int qq = 0; qq < C; ++qq)
                    ptx::st_cluster(ptx::mapa(work_s + 4u * (pX + u * L::kSA), qq), x[qq]);
            }
            ptx::cluster_sync();
#pragma unroll
            for (int e = 0; e < 32; ++e) v[e] = work[pA + L::kSA * e];
        } else {
#pragma unroll
            for (int e = 0; e < 32; ++e) v[e] = __ldg(&data[tid + T * e]);
        }

        // ---- round A: 5 stages, element e at p = tid + T*e (with C = 1 the first stage takes the
        // row's canonical residues)
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const int half = 16 >> k;
#pragma unroll
            for (int e = 0; e < 32; ++e) {
                if ((e & half) == 0) {
                    uint2 w = __ldg(&tw[(1 << k) * (C + c) + (e >> (5 - k))]);
                    if (C == 1 && k == 0)
                        ct_bfly_first(v[e], v[e + half], w, q);
                    else
                        ct_bfly(v[e], v[e + half], w, q);
                }
            }
        }
#pragma unroll
        for (int e = 0; e < 32; ++e) work[pA + L::kSA * e] = v[e];
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
                for (int e = 0; e < EG; ++e) vv[e] = work[g * L::kSA + lane + 33 * e];
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
#pragma unroll
                for (int e = 0; e < EG; ++e) work[g * L::kSA + lane + 33 * e] = vv[e];
            }
            __syncthreads();
        }

        // ---- round C: last 5 stages on 32 contiguous elements p = 32*gidx + e
        {
            const int gidx = rev_bits<LOG_T>(tid);
            const int pC = L::pad(32 * gidx);
#pragma unroll
            for (int e = 0; e < 32; ++e) v[e] = work[pC + e];
            twc.ready();
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                const int half = 16 >> k;
#pragma unroll
                for (int e = 0; e < 32; ++e) {
                    if ((e & half) == 0) {
                        uint2 w = twc[(1 << k) - 1 + (e >> (5 - k))];
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
            __syncthreads();  // `work` is rewritten by the next row's round A
        } else if constexpr (!PUSH) {
            __syncthreads();  // every thread has read its round-C inputs
#pragma unroll
            for (int e = 0; e < 32; ++e) work[pA + L::kSA * rev_bits<5>(e)] = v[e];
            ptx::cluster_sync();
            // CTA c writes k in [c*NC, (c+1)*NC); k lives in CTA rev(k mod C) at k / C.
            // All 32 remote loads are issued before any store so their latencies overlap.
#pragma unroll
            for (int u = 0; u < 32; ++u) {
                const int k = c * NC + u * T + tid;
                const int own = rev_bits<LOG_C>(k & (C - 1));
                v[u] = ptx::ld_cluster(ptx::mapa(work_s + 4u * (pK + L::template offK<LOG_C>(u)), own));
            }
#pragma unroll
            for (int u = 0; u < 32; ++u) data[c * NC + u * T + tid] = v[u];
        } else {
            // output k = k_local * C + rev(c) goes to the CTA that stores [d*NC, (d+1)*NC)
            uint32_t* const recv = work + L::kWords;
            const uint32_t recv_s = work_s + 4u * L::kWords;
            const int rc = rev_bits<LOG_C>(c);
#pragma unroll
            for (int e = 0; e < 32; ++e) {
                const int k = (rev_bits<5>(e) * T + tid) * C + rc;
                ptx::st_cluster(ptx::mapa(recv_s + 4u * swo<LOG_C>(k & (NC - 1)), k >> LOG_NC), v[e]);
            }
            ptx::cluster_sync();
#pragma unroll
            for (int u = 0; u < 32; ++u) {
                const int off = u * T + tid;
                data[c * NC + off] = recv[swo<LOG_C>(off)];
            }
        }
    }
    if constexpr (C > 1) ptx::cluster_sync();
}

template <int LOG_T, int LOG_C, bool PUSH, bool TWS, int OCC>
__global__ void __launch_bounds__(1 << LOG_T, kMinBlocks<LOG_T> * OCC)
ntt_inv_kernel(const NttArgs a) {
    constexpr int T = 1 << LOG_T, C = 1 << LOG_C;
    constexpr int LOG_NC = LOG_T + 5, NC = 1 << LOG_NC;
    constexpr int N = NC * C;
    constexpr int RB = LOG_T - 5;
    extern __shared__ __align__(128) uint32_t work[];
    const uint32_t work_s = ptx::smem_u32(work);
    const int tid = threadIdx.x;
    const int c = (C > 1) ? (int)blockIdx.x : 0;
    using L = PadLayout<LOG_T>;
    static_assert(C == 1 || (T >> LOG_C) >= 32, "cluster exchange offsets need T / C >= 32");
    const int pA = L::pad(tid);                             // p = tid + T e
    const int pX = L::pad(c * (NC / C) + tid);              // p = c NC / C + tid + T u
    const int pK = L::pad((c * NC + tid) >> LOG_C);         // p = (c NC + u T + tid) / C
    const RowIter ri = row_iter(a.rows, a.contiguous);
    TwCol<LOG_T, TWS> twc{nullptr, reinterpret_cast<uint2*>(work + kSmemWords<LOG_T, LOG_C, PUSH>) + tid, -1};
    if constexpr (C > 1) ptx::cluster_sync();  // every peer is resident before the first push

    for (int row = ri.row; row < ri.end; row += ri.step) {
        uint32_t q;
        int mod;
        uint32_t* data = row_ref<N>(a, row, &q, &mod);
        const uint2* tw = a.tw + (size_t)mod * N;
        twc.refresh(a.twC + (((size_t)mod * C + c) * 31) * T + tid, mod);
        if (tid == 0 && row + ri.step < ri.end) prefetch_row<LOG_T, LOG_C, false>(row_ptr<N>(a, row + ri.step), c);
        uint32_t v[32];

        // ---- input in bit-reversed order: thread tid gets k_local = rev5(e)*T + tid
        if constexpr (C > 1) {
            // push: peers finished reading their `work` before the previous row's second
            // barrier; pull: peers may still be reading this CTA's `work` (cross stages)
            if constexpr (!PUSH) {
                __syncwarp();
                ptx::cluster_arrive_relaxed();
                ptx::cluster_wait();
            }
#pragma unroll
            for (int u = 0; u < 32; ++u) v[u] = __ldg(&data[c * NC + u * T + tid]);
#pragma unroll
            for (int u = 0; u < 32; ++u) {
                const int k = c * NC + u * T + tid;
                const int own = rev_bits<LOG_C>(k & (C - 1));
                ptx::st_cluster(ptx::mapa(work_s + 4u * (pK + L::template offK<LOG_C>(u)), own), v[u]);
            }
            ptx::cluster_sync();
#pragma unroll
            for (int e = 0; e < 32; ++e) v[e] = work[pA + L::kSA * rev_bits<5>(e)];
            __syncthreads();  // `work` is rewritten below
        } else {
#pragma unroll
            for (int e = 0; e < 32; ++e) v[e] = __ldg(&data[rev_bits<5>(e) * T + tid]);
        }

        // ---- round C': first 5 GS stages (t = 1..16) on p = 32*gidx + e
        {
            const int gidx = rev_bits<LOG_T>(tid);
            const int pC = L::pad(32 * gidx);
            twc.ready();
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                const int half = 1 << k;
                const int kf = 4 - k;  // the matching forward stage inside the round
#pragma unroll
                for (int e = 0; e < 32; ++e) {
                    if ((e & half) == 0) {
                        uint2 w = twc[(1 << kf) - 1 + (e >> (5 - kf))];
                        if (k == 0)
                            gs_bfly_first(v[e], v[e + half], w, q);  // the row's canonical residues
                        else
                            gs_bfly(v[e], v[e + half], w, q);
                    }
                }
            }
#pragma unroll
            for (int e = 0; e < 32; ++e) work[pC + e] = v[e];
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
                for (int e = 0; e < EG; ++e) vv[e] = work[g * L::kSA + lane + 33 * e];
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
#pragma unroll
                for (int e = 0; e < EG; ++e) work[g * L::kSA + lane + 33 * e] = vv[e];
            }
            __syncthreads();
        }

        // ---- round A'
#pragma unroll
        for (int e = 0; e < 32; ++e) v[e] = work[pA + L::kSA * e];
#pragma unroll
        for (int k = 4; k >= (C == 1 ? 1 : 0); --k) {
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
            // the last stage (pairs e, e + 16, twiddle tw[1]) with N^-1 folded in: (x + y) N^-1
            // and (x - y) (tw[1] N^-1), one Shoup product each, canonical
            const uint2 niw = __ldg(&a.ninv_w1[mod]);
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                const uint32_t x = v[e], y = v[e + 16];
                v[e] = mul_shoup(x + y, ni.x, ni.y, q);
                v[e + 16] = mul_shoup(x - y + 2 * q, niw.x, niw.y, q);
            }
#pragma unroll
            for (int e = 0; e < 32; ++e) data[tid + T * e] = v[e];
            __syncthreads();
        } else {
            constexpr int PER = NC / C;
            uint32_t* const recv = work + L::kWords;
            if constexpr (PUSH) {
                // quarter c's value at p goes to CTA p / PER, which runs the cross stages there
                const uint32_t recv_s = work_s + 4u * L::kWords;
#pragma unroll
                for (int e = 0; e < 32; ++e) {
                    const int p = tid + T * e;
                    ptx::st_cluster(ptx::mapa(recv_s + 4u * (c * PER + (p & (PER - 1))), p / PER), v[e]);
                }
            } else {
                // each thread rewrites exactly the positions it read in round A'
#pragma unroll
                for (int e = 0; e < 32; ++e) work[pA + L::kSA * e] = v[e];
            }
            ptx::cluster_sync();
            constexpr int U = PER / T;
            // all remote / local loads of the cross stages first (v is free here)
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int qq = 0; qq < C; ++qq) {
                    const int jl = u * T + tid;
                    if constexpr (PUSH) {
                        v[u * C + qq] = recv[qq * PER + jl];
                    } else {
                        v[u * C + qq] = ptx::ld_cluster(ptx::mapa(work_s + 4u * (pX + u * L::kSA), qq));
                    }
                }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int jl = u * T + tid;
                const int jj = c * PER + jl;
                uint32_t* x = v + u * C;
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
    if constexpr (C > 1) ptx::cluster_sync();
}

// Cross stages of the split forward for quarter CC of a row: thread tid loads position
// p = tid + T e of all C quarters, runs the first log2(C) Cooley-Tukey stages on them and
// keeps quarter CC. With CC a compile-time constant only the butterflies that feed it are
// computed (3 modmuls per position instead of 4 for C = 4); CC = -1 keeps quarter c_rt.
template <int LOG_T, int LOG_C, int CC>
__device__ __forceinline__ void split_cross(uint32_t (&v)[32], const uint32_t* data, const uint2* tw, uint32_t q,
                                            int tid, int c_rt = 0) {
    constexpr int T = 1 << LOG_T, C = 1 << LOG_C, NC = 32 * T;
#pragma unroll
    for (int e0 = 0; e0 < 32; e0 += 8) {
        uint32_t x[8][C];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int qq = 0; qq < C; ++qq) x[i][qq] = __ldg(&data[tid + T * (e0 + i) + qq * NC]);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
#pragma unroll
            for (int s = 0; s < LOG_C; ++s) {
                const int tq = C >> (s + 1);
#pragma unroll
                for (int qq = 0; qq < C; ++qq) {
                    if ((qq / tq) % 2 == 0) {
                        uint2 w = __ldg(&tw[(1 << s) + qq / (2 * tq)]);
                        ct_bfly(x[i][qq], x[i][qq + tq], w, q);
                    }
                }
            }
            if constexpr (CC >= 0) {
                v[e0 + i] = x[i][CC];
            } else {  // quarter chosen at run time
                uint32_t r = x[i][0];
#pragma unroll
                for (int qq = 1; qq < C; ++qq)
                    if (qq == c_rt) r = x[i][qq];
                v[e0 + i] = r;
            }
        }
    }
}

template <int LOG_T, int LOG_C>
__device__ __forceinline__ void split_cross_dispatch(int c, uint32_t (&v)[32], const uint32_t* data, const uint2* tw,
                                                     uint32_t q, int tid) {
    constexpr int C = 1 << LOG_C;
    static_assert(C <= 8, "split cross stages are specialised for clusters of up to 8 CTAs");
    switch (c) {
        case 0: split_cross<LOG_T, LOG_C, 0>(v, data, tw, q, tid); break;
        case 1: split_cross<LOG_T, LOG_C, 1 % C>(v, data, tw, q, tid); break;
        case 2: if constexpr (C > 2) split_cross<LOG_T, LOG_C, 2 % C>(v, data, tw, q, tid); break;
        case 3: if constexpr (C > 2) split_cross<LOG_T, LOG_C, 3 % C>(v, data, tw, q, tid); break;
        case 4: if constexpr (C > 4) split_cross<LOG_T, LOG_C, 4 % C>(v, data, tw, q, tid); break;
        case 5: if constexpr (C > 4) split_cross<LOG_T, LOG_C, 5 % C>(v, data, tw, q, tid); break;
        case 6: if constexpr (C > 4) split_cross<LOG_T, LOG_C, 6 % C>(v, data, tw, q, tid); break;
        default: if constexpr (C > 4) split_cross<LOG_T, LOG_C, 7 % C>(v, data, tw, q, tid); break;
    }
}

// Forward transform with independent quarters (exchange mode "split", C > 1): every CTA of
// the cluster reads its positions p in all C quarters of the row (the C reads of a position
// hit L2 after the first), runs the cross stages itself and keeps its own output quarter c,
// so no data moves between CTAs. The cluster only orders the in-place update: each CTA
// arrives on the cluster barrier once it has read the row and waits on it just before
// storing its outputs (k = k_local * C + rev(c)), so the barrier's latency hides behind the
// local stages.
template <int LOG_T, int LOG_C, bool TWS, int OCC>
__global__ void __launch_bounds__(1 << LOG_T, kMinBlocks<LOG_T> * OCC)
ntt_fwd_split_kernel(const NttArgs a) {
    constexpr int T = 1 << LOG_T, C = 1 << LOG_C;
    constexpr int LOG_NC = LOG_T + 5, NC = 1 << LOG_NC;
    constexpr int N = NC * C;
    constexpr int RB = LOG_T - 5;
    static_assert(C > 1, "split mode needs a cluster");
    extern __shared__ __align__(128) uint32_t work[];
    const int tid = threadIdx.x;
    const int c = (int)blockIdx.x;
    const int rc = rev_bits<LOG_C>(c);
    using L = PadLayout<LOG_T>;
    const int pA = L::pad(tid);
    const RowIter ri = row_iter(a.rows, a.contiguous);
    TwCol<LOG_T, TWS> twc{nullptr, reinterpret_cast<uint2*>(work + kSmemWords<LOG_T, LOG_C, false>) + tid, -1};

    for (int row = ri.row; row < ri.end; row += ri.step) {
        uint32_t q;
        int mod;
        uint32_t* data = row_ref<N>(a, row, &q, &mod);
        const uint2* tw = a.tw + (size_t)mod * N;
        twc.refresh(a.twC + (((size_t)mod * C + c) * 31) * T + tid, mod);
        if (tid == 0 && row + ri.step < ri.end)
            ptx::prefetch_l2(row_ptr<N>(a, row + ri.step) + c * NC, NC * 4);
        uint32_t v[32];

        // ---- cross stages for this CTA's quarter: specialised on c (only the butterflies that
        // feed quarter c) where registers allow, generic under the 64-register budget
        if constexpr (OCC == 1)
            split_cross_dispatch<LOG_T, LOG_C>(c, v, data, tw, q, tid);
        else
            split_cross<LOG_T, LOG_C, -1>(v, data, tw, q, tid, c);
        __syncwarp();
        ptx::cluster_arrive_relaxed();  // this CTA has read everything it needs from the row

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
        for (int e = 0; e < 32; ++e) work[pA + L::kSA * e] = v[e];
        __syncthreads();

        // ---- round B
        if constexpr (RB > 0) {
            constexpr int GPT = 32 >> RB;
            constexpr int EG = 1 << RB;
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
                    for (int e = 0; e < EG; ++e) {
                        if ((e & half) == 0) {
                            uint2 w = __ldg(&tw[(1 << k) * (32 * (C + c) + g) + (e >> (RB - k))]);
                            ct_bfly(vv[e], vv[e + half], w, q);
                        }
                    }
                }
#pragma unroll
                for (int e = 0; e < EG; ++e) work[g * L::kSA + lane + 33 * e] = vv[e];
            }
            __syncthreads();
        }

        // ---- round C
        {
            const int gidx = rev_bits<LOG_T>(tid);
            const int pC = L::pad(32 * gidx);
#pragma unroll
            for (int e = 0; e < 32; ++e) v[e] = work[pC + e];
            twc.ready();
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                const int half = 16 >> k;
#pragma unroll
                for (int e = 0; e < 32; ++e) {
                    if ((e & half) == 0) {
                        uint2 w = twc[(1 << k) - 1 + (e >> (5 - k))];
                        ct_bfly(v[e], v[e + half], w, q);
                    }
                }
            }
#pragma unroll
            for (int e = 0; e < 32; ++e) v[e] = csub(csub(v[e], 2 * q), q);
        }
        __syncwarp();
        ptx::cluster_wait();  // every CTA of the cluster has read the row: safe to overwrite it
#pragma unroll
        for (int e = 0; e < 32; ++e) data[(rev_bits<5>(e) * T + tid) * C + rc] = v[e];
        __syncthreads();  // `work` is rewritten by the next row's round A
    }
}

template <int LOG_T, int LOG_C, int EX, bool TWS, int OCC>
int launch(const fhe_ctx* ctx, const NttTables& t, int variant, bool inverse, uint32_t* d, int rows,
           int batch, const LimbMap& map, const RowRef* rowtab, cudaStream_t stream) {
    constexpr int T = 1 << LOG_T, C = 1 << LOG_C;
    constexpr bool PUSH = EX == 1;
    static_assert(!(PUSH && TWS), "push buffers and staged twiddles do not fit together");
    constexpr int smem = kSmemTotalWords<LOG_T, LOG_C, PUSH, TWS> * 4;
    NttArgs args;
    args.data = d;
    args.rows = rows;
    args.batch = batch;
    args.tw = inverse ? t.inv : t.fwd;
    args.twC = inverse ? t.invC[variant & 1] : t.fwdC[variant & 1];
    args.ninv = t.ninv;
    args.ninv_w1 = t.ninv_w1;
    args.status = ctx->d_status;
    args.contiguous = TWS ? 1 : 0;
    args.rowtab = rowtab;
    args.mod_q = ctx->d_mods;
    args.map = map;
    void (*kern)(NttArgs);
    if constexpr (EX == 2 && LOG_C > 0)
        kern = inverse ? ntt_inv_kernel<LOG_T, LOG_C, false, TWS, OCC> : ntt_fwd_split_kernel<LOG_T, LOG_C, TWS, OCC>;
    else
        kern = inverse ? ntt_inv_kernel<LOG_T, LOG_C, PUSH, TWS, OCC> : ntt_fwd_kernel<LOG_T, LOG_C, PUSH, TWS, OCC>;
    FHE_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    // give the rest of the L1/shared array to L1, which caches the (other) twiddle tables
    int carve = (int)((kMinBlocks<LOG_T> * OCC * (smem + 1024) * 100 + 228 * 1024 - 1) / (228 * 1024));
    FHE_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, carve > 100 ? 100 : carve));
    if (C > 1) FHE_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    cudaLaunchConfig_t cfg = {};
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
    // persistent: exactly one wave of clusters. Clusters must fit inside a GPC, so the number
    // that can be resident at once is asked from the occupancy calculator, not derived from
    // the SM count (a second, partial wave would double the run time).
    static int max_clusters[2] = {0, 0};
    int& mc = max_clusters[inverse ? 1 : 0];
    if (mc == 0) {
        cfg.gridDim = dim3(C, 1, 1);
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess || n < 1)
            n = ctx->num_sms * kMinBlocks<LOG_T> * OCC / C;
        mc = n < 1 ? 1 : n;
    }
    int gy = rows < mc ? rows : mc;
    if (gy > 65535) gy = 65535;
    cfg.gridDim = dim3(C, gy, 1);
    FHE_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, args));
    return FHE_OK;
}

// Launch of one plain-path variant for the shape (LT, LC); returns from the enclosing function.
#define FHE_NTT_CASE(LT, LC)                                                                          \
    if (log_t == LT && log_c == LC) {                                                                 \
        const int ex = LC > 0 ? ntt_variant_exchange(v) : 0;                                          \
        const bool tws = ntt_variant_tws(v), occ = ntt_variant_occ2(v);                               \
        if constexpr (LC > 0) {                                                                       \
            if (ex == 3) return ntt_u32_l2(ctx, logN, v & 1, inverse, d, rows, batch, map, rowtab, stream, scr); \
            if (ex == 1) return launch<LT, LC, 1, false, 1>(ctx, t, v, inverse, d, rows, batch, map, rowtab, stream); \
            if (ex == 2)                                                                              \
                return tws ? launch<LT, LC, 2, true, 1>(ctx, t, v, inverse, d, rows, batch, map, rowtab, stream) \
                     : occ ? launch<LT, LC, 2, false, 2>(ctx, t, v, inverse, d, rows, batch, map, rowtab, stream) \
                           : launch<LT, LC, 2, false, 1>(ctx, t, v, inverse, d, rows, batch, map, rowtab, stream); \
        }                                                                                             \
        return tws ? launch<LT, LC, 0, true, 1>(ctx, t, v, inverse, d, rows, batch, map, rowtab, stream) \
             : occ ? launch<LT, LC, 0, false, 2>(ctx, t, v, inverse, d, rows, batch, map, rowtab, stream) \
                   : launch<LT, LC, 0, false, 1>(ctx, t, v, inverse, d, rows, batch, map, rowtab, stream); \
    }

}  // namespace

// Launches for the shapes with clusters of 4 or more CTAs (ntt_u32_wide.cu).
int ntt_u32_launch_wide(const fhe_ctx* ctx, const NttTables& t, uint32_t logN, int log_t, int log_c, int v,
                        bool inverse, uint32_t* d, int rows, int batch, const LimbMap& map, const RowRef* rowtab,
                        cudaStream_t stream, NttScratch scr);

}  // namespace fhe

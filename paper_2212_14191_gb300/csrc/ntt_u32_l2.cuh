// Device code of the plain 32-bit NTT for N >= 2^15 in two passes through a scratch buffer:
// the local passes (a single-CTA transform of NC = 2^(LOG_T + 5) points per CTA) and the cross
// passes that combine the C = N / NC parts of a row. They are shared by the stand-alone
// launches of ntt_u32_l2.cu (see there for the decomposition) and by the persistent batch
// kernel of persist.cu, which also runs a local pass alone as the whole transform of N = NC
// points (C = 1).
#pragma once
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
    const uint2* ninv_w1;    // [nmod] N^-1 times tw[1] of the inverse tables (the last cross stage's twiddle)
    const uint2* tw_sub;     // decimation-in-time forward: tables of the NC-point ring degree
    const uint2* twC_sub;    // [nmod][1][31][T]
    const uint2* twist;      // [nmod][C-1][NC]
    const uint2* omega;      // [nmod][C/2]
    ptrdiff_t src_off;       // inverse, limb-map rows: read row r at data + r N + src_off (0: in place)
    int* cnt;                // per chunk row: local-pass CTAs finished (zeroed before each chunk)
    int fuse;                // 1: the last local-pass CTA of a row runs its cross pass
    LimbMap map;
    HmultTail tail;          // TAIL instantiations of the forward kernels only
};

// Row r of a TAIL transform: component c, polynomial p, output limb i, with i fastest, so that
// the rows in flight together share the last limb's row (c, p), which each of them reads
// whole; the row's modulus is entry c nout + i of the limb map.
struct TailRow {
    int c, i, p;
};
__device__ __forceinline__ TailRow tail_row(const L2Args& a, int r) {
    const int cp = r / a.tail.nout;
    return {cp / a.batch, r % a.tail.nout, cp % a.batch};
}
__device__ __forceinline__ void tail_mod(const L2Args& a, const TailRow& t, uint32_t* q, int* mod) {
    const int l = t.c * a.tail.nout + t.i;
    *q = a.map.q[l];
    *mod = a.map.mod[l];
}

// The C local-pass CTAs of a row each count themselves in cnt[i] once their scratch stores
// are visible (an acquire-release atomic); the one that completes the count runs the row's cross
// pass while the row's scratch is still in L2. Nothing waits: a CTA that is not last exits.
__device__ __forceinline__ bool last_of_row(const L2Args& a, int i, int C) {
    __shared__ int s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        // the barrier orders the CTA's scratch stores before this thread's release
        // (cumulative), so one acquire-release count publishes all of them and, for the last
        // CTA, makes the others' visible; the warps do not each wait for their own
        int old;
        asm volatile("atom.add.acq_rel.gpu.s32 %0, [%1], 1;" : "=r"(old) : "l"(&a.cnt[i]) : "memory");
        s_last = old == C - 1;
    }
    __syncthreads();
    return s_last != 0;
}

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
    if constexpr (BITS == 0)
        return 0;
    else
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
// The first stage of a transform whose inputs are canonical residues (below q), as the rows
// of every call are: the forward's x needs no reduction below 2q, the inverse's x + y is
// already below 2q. Outputs stay in the ranges of ct2 ([0, 4q)) and gs2 ([0, 2q)).
__device__ __forceinline__ void ct2_first(uint32_t& x, uint32_t& y, uint2 w, uint32_t q) {
    uint32_t t = mul_shoup_lazy(y, w.x, w.y, q);
    uint32_t x0 = x;
    x = x0 + t;
    y = x0 - t + 2 * q;
}
__device__ __forceinline__ void gs2_first(uint32_t& x, uint32_t& y, uint2 w, uint32_t q) {
    uint32_t s = x + y;
    uint32_t d = x - y + 2 * q;
    x = s;
    y = mul_shoup_lazy(d, w.x, w.y, q);
}

// ---- inverse cross pass: grid (blocks over NC/4 quad positions, chunk rows); 4 positions per
// thread; the last log2(C) Gentleman-Sande stages and the N^-1 scaling. The scaling rides on the
// last stage: its outputs are (x + y) N^-1 and (x - y) (w N^-1), one Shoup product each, where
// the stage and the scaling would take three (x + y < 4q and x - y + 2q < 4q are valid Shoup
// inputs, and the products come out canonical).
template <int LOG_NC, int LOG_C>
__device__ __forceinline__ void cross_inv_row(const L2Args& a, int i, int p0, int pstep) {
    constexpr int NC = 1 << LOG_NC, C = 1 << LOG_C, N = NC * C;
    uint32_t q;
    int mod;
    uint32_t* row = l2_row<N>(a, a.r0 + i, &q, &mod);
    const uint32_t* tmp = a.temp + (size_t)i * N;
    const uint2* tw = a.tw + (size_t)mod * N;
    const uint2 ni = __ldg(&a.ninv[mod]);
    const uint2 niw = __ldg(&a.ninv_w1[mod]);
    for (int p4 = p0; p4 < NC / 4; p4 += pstep) {
        uint4 x[C];
#pragma unroll
        for (int qq = 0; qq < C; ++qq) x[qq] = __ldcg(reinterpret_cast<const uint4*>(tmp + qq * NC) + p4);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint32_t y[C];
#pragma unroll
            for (int qq = 0; qq < C; ++qq) y[qq] = k == 0 ? x[qq].x : k == 1 ? x[qq].y : k == 2 ? x[qq].z : x[qq].w;
#pragma unroll
            for (int s = LOG_C - 1; s >= 1; --s) {
                const int tq = C >> (s + 1);
#pragma unroll
                for (int qq = 0; qq < C; ++qq)
                    if ((qq / tq) % 2 == 0) gs2(y[qq], y[qq + tq], __ldg(&tw[(1 << s) + qq / (2 * tq)]), q);
            }
            if constexpr (C > 1) {
                // the last stage (pairs qq, qq + C/2, all with twiddle tw[1]) and N^-1 at once
#pragma unroll
                for (int qq = 0; qq < C / 2; ++qq) {
                    const uint32_t u = y[qq], w = y[qq + C / 2];
                    y[qq] = mul_shoup(u + w, ni.x, ni.y, q);
                    y[qq + C / 2] = mul_shoup(u - w + 2 * q, niw.x, niw.y, q);
                }
            } else {
                y[0] = mul_shoup(y[0], ni.x, ni.y, q);
            }
#pragma unroll
            for (int qq = 0; qq < C; ++qq) {
                const uint32_t v = y[qq];
                if (k == 0) x[qq].x = v;
                else if (k == 1) x[qq].y = v;
                else if (k == 2) x[qq].z = v;
                else x[qq].w = v;
            }
        }
#pragma unroll
        for (int qq = 0; qq < C; ++qq) reinterpret_cast<uint4*>(row + qq * NC)[p4] = x[qq];
    }
}

// Row data loads of the local passes: the read-only path by default; through L2 (coherent with
// stores made earlier in the same kernel) when COH is set.
template <bool COH>
__device__ __forceinline__ uint32_t ld_row(const uint32_t* p) {
    if constexpr (COH)
        return __ldcg(p);
    else
        return __ldg(p);
}

// Loads of the fused HMULT tail's operands (read once each): streaming by default; through L2
// when COH is set, so that no L1 line of an earlier use of the same buffer can be hit.
template <bool COH, typename V>
__device__ __forceinline__ V ld_tail(const V* p) {
    if constexpr (COH)
        return __ldcg(p);
    else
        return __ldcs(p);
}

// Blocks per SM the register budget is sized for: 64 registers per thread, so twice the
// CTAs of the single-CTA kernels share an SM (measured 10 % faster at 2^15 and 2^16).
template <int LOG_T>
constexpr int kMinB = 2 * ((1 << (14 - LOG_T)) / 32 > 0 ? (1 << (14 - LOG_T)) / 32 : 1);

// ---- quarter pass, inverse: row (stride C, quarter c's bit-reversed share) -> GS stages -> scratch
// Row i of the chunk, quarter c, in a CTA of 2^LOG_T threads whose dynamic shared memory holds
// PadLayout<LOG_T>::kWords words. COH: the row is read through L2 (coherent with writes made
// earlier in the same kernel by other CTAs) instead of the read-only path. With C = 1
// (N = 2^(LOG_T + 5)) the transform ends here: N^-1 is applied and the row is written in place.
template <int LOG_T, int LOG_C, bool COH>
__device__ __forceinline__ void quarter_inv(const L2Args& a, int i, int c) {
    constexpr int T = 1 << LOG_T, C = 1 << LOG_C, NC = 32 * T, N = NC * C, RB = LOG_T - 5;
    extern __shared__ __align__(128) uint32_t work[];
    const int tid = threadIdx.x;
    const int rc = rbits<LOG_C>(c);
    using L = PadLayout<LOG_T>;
    const int pA = L::pad(tid);
    uint32_t q;
    int mod;
    const uint32_t* row = l2_row<N>(a, a.r0 + i, &q, &mod);
    const uint32_t* src = row + a.src_off;
    uint32_t* tmp = a.temp + (size_t)i * N + c * NC;
    const uint2* tw = a.tw + (size_t)mod * N;
    uint32_t v[32];
#pragma unroll
    for (int e = 0; e < 32; ++e) v[e] = ld_row<COH>(&src[(rbits<5>(e) * T + tid) * C + rc]);
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
                if ((e & half) == 0) {
                    const uint2 w = __ldg(&twc[(size_t)((1 << kf) - 1 + (e >> (5 - kf))) * T]);
                    if (k == 0)
                        gs2_first(v[e], v[e + half], w, q);
                    else
                        gs2(v[e], v[e + half], w, q);
                }
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
    if constexpr (C == 1) {
        const uint2 ni = __ldg(&a.ninv[mod]);
        uint32_t* out = const_cast<uint32_t*>(row);  // the in-place transform of this row ends here
#pragma unroll
        for (int e = 0; e < 32; ++e) out[tid + T * e] = mul_shoup(v[e], ni.x, ni.y, q);
    } else {
#pragma unroll
        for (int e = 0; e < 32; ++e) __stcg(&tmp[tid + T * e], v[e]);
        if (a.fuse && last_of_row(a, i, C)) cross_inv_row<LOG_T + 5, LOG_C>(a, i, tid, T);
    }
}

// ---- decimation-in-time forward (the two-pass forward): with n = C m + j and
// k = k' + NC t,
//   A_k = sum_j omega^(t j) psi^((2k'+1) j) B_j[k'],   B_j = NTT_NC(a[j + C m], psi^C),
// omega = psi^(2 NC) a C-th root of unity. psi^C is the NC-point root the library uses for
// that ring degree, so pass 1 is the single-CTA NC-point transform (its tables, natural-
// order output) of a decimated row; pass 2 twists and runs a C-point cyclic DFT, reading C
// contiguous streams and writing C contiguous streams. Pass 1 reads at stride C (the C CTAs
// of a row share every sector through L2), where the decimation-in-frequency order would
// store at stride C.
template <int LOG_NC, int LOG_C, bool TAIL, bool COH = false>
__device__ __forceinline__ void dit_cross_row(const L2Args& a, int i, int p0, int pstep) {
    constexpr int NC = 1 << LOG_NC, C = 1 << LOG_C, N = NC * C;
    uint32_t q;
    int mod;
    uint32_t* row = l2_row<N>(a, a.r0 + i, &q, &mod);
    // TAIL: out = ks' + d' - z'^ is stored instead of z'^
    const uint32_t* ksr = nullptr;
    const uint32_t* dr = nullptr;
    if constexpr (TAIL) {
        const TailRow t = tail_row(a, a.r0 + i);
        tail_mod(a, t, &q, &mod);
        ksr = a.tail.ks + (((size_t)t.c * a.tail.ext + t.i) * a.batch + t.p) * N;
        dr = a.tail.d + (((size_t)t.c * a.tail.nl + t.i) * a.batch + t.p) * N;
        row = a.tail.out + (((size_t)t.c * a.tail.nout + t.i) * a.batch + t.p) * N;
    }
    const uint32_t* tmp = a.temp + (size_t)i * N;
    const uint2* twist = a.twist + (size_t)mod * (C - 1) * NC;
    const uint2* om = a.omega + (size_t)mod * (C / 2);
    uint2 omv[C > 1 ? C / 2 : 1];
#pragma unroll
    for (int m = 0; m < C / 2; ++m) omv[m] = __ldg(&om[m]);
    for (int p4 = p0; p4 < NC / 4; p4 += pstep) {
        uint4 x[C];
#pragma unroll
        for (int jj = 0; jj < C; ++jj) x[jj] = __ldcg(reinterpret_cast<const uint4*>(tmp + jj * NC) + p4);
        // TAIL: ks and d of these outputs, loaded with the scratch so their HBM latency overlaps
        // (for C <= 4; with C = 8 they would not fit in the registers and load at the store)
        constexpr bool kHoist = TAIL && C <= 4;
        uint4 kv[kHoist ? C : 1], dv[kHoist ? C : 1];
        if constexpr (kHoist) {
#pragma unroll
            for (int t = 0; t < C; ++t) {
                kv[t] = ld_tail<COH>(reinterpret_cast<const uint4*>(ksr + t * NC) + p4);
                dv[t] = ld_tail<COH>(reinterpret_cast<const uint4*>(dr + t * NC) + p4);
            }
        }
        uint4 tw2[C > 1 ? 2 * (C - 1) : 1];  // four twist pairs of every j >= 1: two uint4 each
#pragma unroll
        for (int jj = 1; jj < C; ++jj) {
            const uint4* tp = reinterpret_cast<const uint4*>(twist + (size_t)(jj - 1) * NC + 4 * p4);
            tw2[2 * (jj - 1)] = __ldg(tp);
            tw2[2 * (jj - 1) + 1] = __ldg(tp + 1);
        }
        uint4 o[C];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint32_t y[C];
#pragma unroll
            for (int jj = 0; jj < C; ++jj) y[jj] = k == 0 ? x[jj].x : k == 1 ? x[jj].y : k == 2 ? x[jj].z : x[jj].w;
            y[0] = csub(y[0], 2 * q);  // the local pass stores [0, 4q)
#pragma unroll
            for (int jj = 1; jj < C; ++jj) {
                const uint4 t4 = tw2[2 * (jj - 1) + (k >> 1)];
                const uint2 w = (k & 1) ? make_uint2(t4.z, t4.w) : make_uint2(t4.x, t4.y);
                y[jj] = mul_shoup_lazy(y[jj], w.x, w.y, q);  // [0, 2q)
            }
            // C-point cyclic DFT, radix-2 decimation in frequency: position p ends up holding
            // output t = rev(p); values stay in [0, 2q)
#pragma unroll
            for (int s = 0; s < LOG_C; ++s) {
                const int h = C >> (s + 1);
#pragma unroll
                for (int b = 0; b < C; b += 2 * h)
#pragma unroll
                    for (int jj = 0; jj < h; ++jj) {
                        const int m = jj << s;  // omega^m
                        if (m == 0) {
                            const uint32_t su = csub(y[b + jj] + y[b + jj + h], 2 * q);
                            const uint32_t di = csub(y[b + jj] - y[b + jj + h] + 2 * q, 2 * q);
                            y[b + jj] = su;
                            y[b + jj + h] = di;
                        } else {
                            gs2(y[b + jj], y[b + jj + h], omv[m], q);
                        }
                    }
            }
#pragma unroll
            for (int p = 0; p < C; ++p) {
                const int t = rbits<LOG_C>(p);
                const uint32_t val = csub(y[p], q);
                if (k == 0) o[t].x = val;
                else if (k == 1) o[t].y = val;
                else if (k == 2) o[t].z = val;
                else o[t].w = val;
            }
        }
        if constexpr (TAIL) {
#pragma unroll
            for (int t = 0; t < C; ++t) {
                uint4 kt, dt;
                if constexpr (kHoist) {
                    kt = kv[t];
                    dt = dv[t];
                } else {
                    kt = ld_tail<COH>(reinterpret_cast<const uint4*>(ksr + t * NC) + p4);
                    dt = ld_tail<COH>(reinterpret_cast<const uint4*>(dr + t * NC) + p4);
                }
                uint4 r;
                r.x = csub(csub(kt.x + dt.x, q) + q - o[t].x, q);
                r.y = csub(csub(kt.y + dt.y, q) + q - o[t].y, q);
                r.z = csub(csub(kt.z + dt.z, q) + q - o[t].z, q);
                r.w = csub(csub(kt.w + dt.w, q) + q - o[t].w, q);
                __stcs(reinterpret_cast<uint4*>(row + t * NC) + p4, r);
            }
        } else {
#pragma unroll
            for (int t = 0; t < C; ++t) reinterpret_cast<uint4*>(row + t * NC)[p4] = o[t];
        }
    }
}

// Local pass of row i, sub-transform j (see quarter_inv for the shared memory and COH). With
// C = 1 and no tail the transform ends here and the row is written in place, in natural order.
// LAST (TAIL only): the tail has the relinearised last limb's term (the HMULT's RESCALE tail);
// false: z' = y' (the ModDown combine of key switching, a.tail.last null).
template <int LOG_T, int LOG_C, bool TAIL, bool COH, bool LAST = true>
__device__ __forceinline__ void dit_local(const L2Args& a, int i, int j) {
    constexpr int T = 1 << LOG_T, C = 1 << LOG_C, NC = 32 * T, N = NC * C, RB = LOG_T - 5;
    extern __shared__ __align__(128) uint32_t work[];
    const int tid = threadIdx.x;
    using L = PadLayout<LOG_T>;
    const int pA = L::pad(tid);
    uint32_t q;
    int mod;
    uint32_t* row = l2_row<N>(a, a.r0 + i, &q, &mod);
    uint32_t* tmp = a.temp + (size_t)i * N + (size_t)j * NC;
    TailRow t{};
    if constexpr (TAIL) {
        t = tail_row(a, a.r0 + i);
        tail_mod(a, t, &q, &mod);
    }
    const uint2* tw = a.tw_sub + (size_t)mod * NC;
    uint32_t v[32];
    if constexpr (TAIL) {
        // z' = y' + [last]_q q_l^-1 (last centred: values above (q_l - 1) / 2 stand for last - q_l),
        // or z' = y' without a last limb (the ModDown combine of key switching)
        const uint32_t* yr = a.tail.y + (((size_t)t.c * a.tail.nl + t.i) * a.batch + t.p) * N;
        const uint32_t* lr = LAST ? a.tail.last + ((size_t)t.c * a.batch + t.p) * N : nullptr;
        const uint2 qlinv = LAST ? __ldg(&a.tail.qlinv[t.i]) : make_uint2(0, 0);
        if (tid == 0 && a.fuse) {
            // the row's cross pass, run by the last of its C local passes, reads all of the
            // row's ks and d: each local pass brings its own part of them into L2 meanwhile
            const size_t part = (size_t)j * NC;
            ptx::prefetch_l2(a.tail.ks + (((size_t)t.c * a.tail.ext + t.i) * a.batch + t.p) * N + part, NC * 4);
            ptx::prefetch_l2(a.tail.d + (((size_t)t.c * a.tail.nl + t.i) * a.batch + t.p) * N + part, NC * 4);
        }
        // The Shoup product takes any 32-bit word, so the centred last limb needs no reduction
        // first: x = last + (q - q_l mod q) stands for last - q_l (x < 2^31). The first
        // butterfly stage pairs e with e + 16 and takes x-side inputs below 2q and y-side
        // inputs of any size, so only e < 16 is brought from [0, 3q) below 2q.
        if constexpr (LAST) {
            const uint32_t half = (a.tail.ql - 1) / 2, lift = q - a.tail.ql % q;
#pragma unroll
            for (int e = 0; e < 32; ++e) {
                const size_t idx = (size_t)(tid + T * e) * C + j;
                const uint32_t lv = ld_tail<COH>(&lr[idx]), yv = ld_tail<COH>(&yr[idx]);
                const uint32_t x = lv > half ? lv + lift : lv;
                const uint32_t z = yv + mul_shoup_lazy(x, qlinv.x, qlinv.y, q);
                v[e] = e < 16 ? csub(z, q) : z;
            }
        } else {
#pragma unroll
            for (int e = 0; e < 32; ++e) v[e] = ld_tail<COH>(&yr[(size_t)(tid + T * e) * C + j]);
        }
    } else {
#pragma unroll
        for (int e = 0; e < 32; ++e) v[e] = ld_row<COH>(&row[(size_t)(tid + T * e) * C + j]);
    }
    // round A: stages 0..4 of the NC-point transform
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const int half = 16 >> k;
#pragma unroll
        for (int e = 0; e < 32; ++e)
            if ((e & half) == 0) {
                const uint2 w = __ldg(&tw[(1 << k) + (e >> (5 - k))]);
                if (k == 0)
                    ct2_first(v[e], v[e + half], w, q);
                else
                    ct2(v[e], v[e + half], w, q);
            }
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
                        ct2(vv[e], vv[e + half], __ldg(&tw[(1 << k) * (32 + g) + (e >> (RB - k))]), q);
            }
#pragma unroll
            for (int e = 0; e < EG; ++e) work[g * L::kSA + lane + 33 * e] = vv[e];
        }
        __syncthreads();
    }
    // round C: last five stages, per-thread twiddle columns of the single-CTA shape
    {
        const int gidx = rbits<LOG_T>(tid);
        const int pC = L::pad(32 * gidx);
#pragma unroll
        for (int e = 0; e < 32; ++e) v[e] = work[pC + e];
        const uint2* twc = a.twC_sub + ((size_t)mod * 31) * T + tid;
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const int half = 16 >> k;
#pragma unroll
            for (int e = 0; e < 32; ++e)
                if ((e & half) == 0) ct2(v[e], v[e + half], __ldg(&twc[(size_t)((1 << k) - 1 + (e >> (5 - k))) * T]), q);
        }
    }
    // natural order: thread tid holds k' = rev5(e) T + tid
    if constexpr (C == 1 && !TAIL) {
#pragma unroll
        for (int e = 0; e < 32; ++e) row[rbits<5>(e) * T + tid] = csub(csub(v[e], 2 * q), q);
    } else {
        // stored as they are, in [0, 4q): the cross pass's twists (lazy Shoup products, any
        // 32-bit input) bring streams j >= 1 below 2q and it reduces stream 0 itself, after
        // which its DFT keeps [0, 2q)
#pragma unroll
        for (int e = 0; e < 32; ++e) __stcg(&tmp[rbits<5>(e) * T + tid], v[e]);
        if (a.fuse && last_of_row(a, i, C)) dit_cross_row<LOG_T + 5, LOG_C, TAIL, COH>(a, i, tid, T);
    }
}

}  // namespace
}  // namespace fhe

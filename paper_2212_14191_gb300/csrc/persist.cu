// Operation-level batching (Sec. IV-D) in one persistent launch: every NTT / INTT / HMULT of a
// batch plan at N >= 2^14 runs as tiles of a single kernel whose CTAs pop work from a device
// queue, so operations of uneven ring degree and level overlap on the GPU instead of running
// group after group.
//
// Tiles. A tile is one piece of one pipeline stage:
//   NTT      one local pass of the two-pass transform (row, part) in the 512-thread, 2^14-point
//            shape of ntt_u32_l2.cuh; the last of a row's C = N / 2^14 parts runs the row's
//            cross pass; with C = 1 (N = 2^14) the local pass is the whole transform;
//   TENSOR, CONV, IP, RELIN_LAST, LAST_FIX
//            16384 residues of one limb (of every destination limb for CONV) of the HMULT
//            stages of ckks_kernels.cuh.
// An HMULT runs the stages of the fused pipeline of ckks.cu (hmult_fused): tensor product,
// INTT of d2, per slice Conv + NTT, inner product, per component INTT of the P limbs and the
// ModDown Conv, the last limb's relinearisation and INTT, and the forward NTT with the fused
// RESCALE tail that writes the output.
//
// Dependencies. Each stage counts its completed tiles in a device counter; a tile lists up to
// two (counter, target) pairs that must be reached before it starts. Thread 0 of the CTA spins
// on them with a bounded wait: past the limit it records FHE_ETIMEOUT in the context's status
// word and raises an abort flag, after which every remaining tile is skipped (and still
// counted), so the kernel always finishes. Tiles are queued in an order in which every
// dependency points to an earlier tile, and a CTA takes its next ticket only once its current
// tile may start, so the earliest unfinished tile is always running: the queue cannot
// deadlock, whatever the number of resident CTAs.
//
// Memory. HMULTs run in S scratch slots; the HMULT after another in the same slot waits for its
// predecessor's last stage, which bounds the scratch. Data written inside the kernel is read
// through L2 (ld.global.cg), never through the read-only or L1 path.
#include <algorithm>
#include <vector>

#include "ckks_kernels.cuh"
#include "ntt_u32_l2.cuh"
#include "persist.h"

namespace fhe {
namespace {

constexpr int kLogPT = 9;
constexpr int kPT = 1 << kLogPT;           // threads per CTA
constexpr size_t kChunk4 = 4096;           // 16-byte words per elementwise tile (16384 residues)
// Conv tiles are shorter: each converts 4096 coefficients into every destination limb (up to
// 64), so with the 16384 of the other stages one tile would run for far longer than any other
// and hold up the transforms that wait for it.
constexpr size_t kConvChunk2 = 2048;       // 8-byte words per Conv tile
constexpr uint32_t kNoDep = 0xffffffffu;
constexpr size_t kAlign = 256;

enum : uint16_t { PK_NTT = 0, PK_TENSOR, PK_CONV, PK_IP, PK_RELIN_LAST, PK_LAST_FIX, PK_NOP };
// PK_NTT sub-kind: bits 0-1 log2(C), bit 2 inverse, bit 3 fused HMULT tail
constexpr uint16_t kSubInv = 4, kSubTail = 8;

struct PTile {
    uint16_t kind, sub;
    uint32_t desc;          // index into the kind's argument table
    uint32_t x, y;          // NTT: row, part; others: limb (component), chunk
    uint32_t dep[2], need[2];
    uint32_t done;          // counter incremented once the tile has completed (kNoDep: none)
    uint32_t pad;
};

// Device tables hold each argument block padded to a multiple of 16 bytes, so that a tile can
// copy its block into shared memory with 16-byte loads.
template <typename T>
struct alignas(16) Slot {
    T v;
};

struct PParams {
    const PTile* tiles;
    int ntiles;
    unsigned* ctr;          // [0] queue head, [1] abort flag, then stage counters
    const Slot<L2Args>* ntt;
    const Slot<TensorArgs>* ten;
    const Slot<ConvArgs>* conv;
    const Slot<IpArgs>* ip;
    const Slot<LastArgs>* last;
    int* status;
    long long wait_cycles;
};

// Argument block of the running tile, copied into shared memory at the tile's start.
union alignas(16) TileArgs {
    L2Args ntt;
    TensorArgs ten;
    ConvArgs conv;
    IpArgs ip;
    LastArgs last;
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned ld_relaxed(const unsigned* p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Thread 0: wait until ctr[idx] >= need, within the cycle limit. False if the limit passed
// (then FHE_ETIMEOUT is recorded and the abort flag raised) or the run was aborted meanwhile.
__device__ bool wait_counter(const PParams& p, uint32_t idx, uint32_t need) {
    const long long t0 = clock64();
    for (;;) {
        if (ld_acquire(&p.ctr[idx]) >= need) return true;
        if (ld_relaxed(&p.ctr[1])) return false;
        if (clock64() - t0 > p.wait_cycles) {
            atomicCAS(p.status, 0, FHE_ETIMEOUT);
            atomicExch(&p.ctr[1], 1u);
            return false;
        }
        __nanosleep(128);
    }
}

template <typename T>
__device__ __forceinline__ void copy_args(const Slot<T>* src, TileArgs* dst) {
    static_assert(sizeof(Slot<T>) % 16 == 0 && sizeof(Slot<T>) <= sizeof(TileArgs), "argument block size");
    constexpr int kWords = (int)(sizeof(Slot<T>) / 16);
    for (int k = threadIdx.x; k < kWords; k += kPT)
        reinterpret_cast<uint4*>(dst)[k] = __ldg(reinterpret_cast<const uint4*>(src) + k);
}

template <int LC>
__device__ __forceinline__ void run_ntt(const L2Args& a, uint16_t sub, int row, int part) {
    if (sub & kSubInv)
        quarter_inv<kLogPT, LC, true>(a, row, part);
    else if (sub & kSubTail)
        dit_local<kLogPT, LC, true, true>(a, row, part);
    else
        dit_local<kLogPT, LC, false, true>(a, row, part);
}

template <int NS>
__device__ __forceinline__ void run_conv_ns(const ConvArgs& c, const uint32_t* s_hat, size_t n0, size_t n1) {
    conv_range<NS, true, 2>(c, s_hat, n0 + threadIdx.x, n1, kPT);
}

__device__ __forceinline__ void run_conv(const ConvArgs& c, uint32_t* work, uint32_t chunk) {
    conv_load_hat(c, c.nsrc, work);
    __syncthreads();
    const size_t L2 = c.L4 * 2, n0 = (size_t)chunk * kConvChunk2, n1 = min(L2, n0 + kConvChunk2);
    switch (c.nsrc) {
        case 1: run_conv_ns<1>(c, work, n0, n1); break;
        case 2: run_conv_ns<2>(c, work, n0, n1); break;
        case 3: run_conv_ns<3>(c, work, n0, n1); break;
        case 4: run_conv_ns<4>(c, work, n0, n1); break;
        case 5: run_conv_ns<5>(c, work, n0, n1); break;
        case 6: run_conv_ns<6>(c, work, n0, n1); break;
        case 7: run_conv_ns<7>(c, work, n0, n1); break;
        case 8: run_conv_ns<8>(c, work, n0, n1); break;
        case 9: run_conv_ns<9>(c, work, n0, n1); break;
        case 10: run_conv_ns<10>(c, work, n0, n1); break;
        case 11: run_conv_ns<11>(c, work, n0, n1); break;
        case 12: run_conv_ns<12>(c, work, n0, n1); break;
        case 13: run_conv_ns<13>(c, work, n0, n1); break;
        case 14: run_conv_ns<14>(c, work, n0, n1); break;
        default: run_conv_ns<15>(c, work, n0, n1); break;
    }
}

__device__ __forceinline__ void chunk_range(size_t L4, uint32_t chunk, size_t* i0, size_t* i1) {
    *i0 = (size_t)chunk * kChunk4 + threadIdx.x;
    *i1 = min(L4, (size_t)(chunk + 1) * kChunk4);
}

__device__ void run_tile(const PParams& p, const PTile& t, TileArgs* sa, uint32_t* work) {
    size_t i0, i1;
    switch (t.kind) {
        case PK_NTT: {
            copy_args(&p.ntt[t.desc], sa);
            __syncthreads();
            const int lc = t.sub & 3;
            if (lc == 0)
                run_ntt<0>(sa->ntt, t.sub, t.x, t.y);
            else if (lc == 1)
                run_ntt<1>(sa->ntt, t.sub, t.x, t.y);
            else
                run_ntt<2>(sa->ntt, t.sub, t.x, t.y);
            break;
        }
        case PK_TENSOR:
            copy_args(&p.ten[t.desc], sa);
            __syncthreads();
            chunk_range(sa->ten.L4, t.y, &i0, &i1);
            tensor_range(sa->ten, t.x, i0, i1, kPT);
            break;
        case PK_CONV:
            copy_args(&p.conv[t.desc], sa);
            __syncthreads();
            run_conv(sa->conv, work, t.y);
            break;
        case PK_IP:
            copy_args(&p.ip[t.desc], sa);
            __syncthreads();
            chunk_range(sa->ip.L4, t.y, &i0, &i1);
            // the slice loop unrolled where it fits without spilling (1 to 4 slices)
            switch (sa->ip.dnum) {
                case 1: ip_range<true, 1>(sa->ip, t.x, i0, i1, kPT); break;
                case 2: ip_range<true, 2>(sa->ip, t.x, i0, i1, kPT); break;
                case 3: ip_range<true, 3>(sa->ip, t.x, i0, i1, kPT); break;
                case 4: ip_range<true, 4>(sa->ip, t.x, i0, i1, kPT); break;
                default: ip_range<true>(sa->ip, t.x, i0, i1, kPT); break;
            }
            break;
        case PK_RELIN_LAST:
            copy_args(&p.last[t.desc], sa);
            __syncthreads();
            chunk_range(sa->last.L4, t.y, &i0, &i1);
            relin_last_range<true>(sa->last, t.x, i0, i1, kPT);
            break;
        case PK_LAST_FIX:
            copy_args(&p.last[t.desc], sa);
            __syncthreads();
            chunk_range(sa->last.L4, t.y, &i0, &i1);
            last_fix_range<true>(sa->last, t.x, i0, i1, kPT);
            break;
        default:
            break;
    }
}

__global__ void __launch_bounds__(kPT, 2) k_persist(const PParams p) {
    extern __shared__ __align__(128) uint32_t work[];
    __shared__ TileArgs s_args;
    __shared__ int s_next, s_skip;
    if (threadIdx.x == 0) s_next = (int)atomicAdd(&p.ctr[0], 1u);
    __syncthreads();
    int t = s_next;
    while (t < p.ntiles) {
        const PTile tile = p.tiles[t];
        if (threadIdx.x == 0) {
            bool ok = ld_relaxed(&p.ctr[1]) == 0;
            for (int d = 0; d < 2 && ok; ++d)
                if (tile.dep[d] != kNoDep) ok = wait_counter(p, tile.dep[d], tile.need[d]);
            s_skip = ok ? 0 : 1;
            // the next ticket is taken only now that this tile may start (see the file comment)
            s_next = (int)atomicAdd(&p.ctr[0], 1u);
        }
        __syncthreads();
        if (!s_skip) run_tile(p, tile, &s_args, work);
        const int next = s_next;
        __syncthreads();  // the tile's stores are done, shared memory may be reused
        // one release increment publishes the CTA's stores (cumulative through the barrier) to the
        // tiles that wait on this counter with acquire loads
        if (threadIdx.x == 0 && tile.done != kNoDep)
            asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&p.ctr[tile.done]) : "memory");
        t = next;
    }
}

// ------------------------------------------------------------------ host planning

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

int log_c_of(uint32_t logN) { return (int)logN - (kLogPT + 5); }

struct HmInst {
    int op;
    uint32_t logN;
    int nl, B, dnum, ext, C;
    size_t N, limb, L4, nch, nconv;  // residues per limb (B N), 16-byte words, elementwise and Conv tiles per limb
    int nd[16];                     // destination limbs of slice j's ModUp Conv
    size_t rows_t0, rows_t1;        // rows of the two shared NTT temporaries
    size_t bytes;                   // scratch of one instance
    int slot;
};

size_t hm_limbs(int nl, int K, int dnum) {
    const size_t ext = (size_t)nl + K;
    return 3 * (size_t)nl + (size_t)nl + (size_t)dnum * ext + 2 * ext + 2 * (size_t)nl;
}

}  // namespace

struct PersistPlan {
    const fhe_ctx* ctx = nullptr;
    std::vector<fhe_op> ops;
    std::vector<int> ntt_ops;             // indices into ops
    std::vector<HmInst> hm;
    int slots = 0;
    size_t slot_bytes = 0;
    // scratch layout
    size_t ctr_words = 0, ntt_temp_off = 0, slot_off = 0, scratch_bytes = 0;
    // host tables (rebuilt when the scratch buffer changes) and their device copies
    std::vector<PTile> tiles;
    std::vector<L2Args> ntt;
    std::vector<TensorArgs> ten;
    std::vector<ConvArgs> conv;
    std::vector<IpArgs> ip;
    std::vector<LastArgs> last;
    std::vector<RowRef> rows;
    PTile* d_tiles = nullptr;
    Slot<L2Args>* d_ntt = nullptr;
    Slot<TensorArgs>* d_ten = nullptr;
    Slot<ConvArgs>* d_conv = nullptr;
    Slot<IpArgs>* d_ip = nullptr;
    Slot<LastArgs>* d_last = nullptr;
    RowRef* d_rows = nullptr;
    void* bound = nullptr;
    int grid = 0;
    long long wait_cycles = 0;
};

namespace {

// Counter allocator and tile emitter used while building the tables.
struct Builder {
    PersistPlan& P;
    uint8_t* base;  // scratch base (nullptr while sizing)
    uint32_t nctr = 2;
    size_t rowcnt_words = 0;  // per-row completion counters of the NTT stages, after the stage counters
    std::vector<std::pair<L2Args*, size_t>> cnt_fix;  // (stage, word offset of its row counters)
    explicit Builder(PersistPlan& p, uint8_t* b) : P(p), base(b) {}
    uint32_t counter() { return nctr++; }
    void tile(uint16_t kind, uint16_t sub, uint32_t desc, uint32_t x, uint32_t y, uint32_t d0, uint32_t n0,
              uint32_t d1, uint32_t n1, uint32_t done) {
        P.tiles.push_back(PTile{kind, sub, desc, x, y, {d0, d1}, {n0, n1}, done, 0});
    }
};

// An NTT stage over `rows` rows (limb-map mode when rowtab is null: row r is limb r / batch of
// data), with its scratch rows at `temp`; an inverse in limb-map mode reads its rows from src
// instead when given. Returns its descriptor index.
uint32_t ntt_stage(Builder& b, uint32_t logN, bool inverse, uint32_t* data, int batch, const LimbMap* map,
                   const RowRef* rowtab, size_t rows, uint32_t* temp, const HmultTail* tail,
                   const uint32_t* src = nullptr) {
    const fhe_ctx* ctx = b.P.ctx;
    const NttTables& t = ctx->ntt[logN];
    const NttTables& ts = ctx->ntt[kLogPT + 5];
    L2Args a;
    memset(&a, 0, sizeof(a));
    a.data = data;
    a.batch = batch;
    a.rowtab = rowtab;
    a.mod_q = ctx->d_mods;
    a.temp = temp;
    a.r0 = 0;
    a.nrows = (int)rows;
    a.tw = inverse ? t.inv : t.fwd;
    a.twC = inverse ? t.invC[0] : t.fwdC[0];
    a.ninv = t.ninv;
    a.ninv_w1 = t.ninv_w1;
    a.tw_sub = ts.fwd;
    a.twC_sub = ts.fwdC[0];
    a.twist = t.dit_twist[0];
    a.omega = t.dit_omega[0];
    a.fuse = 1;
    if (map) a.map = *map;
    if (tail) a.tail = *tail;
    if (src) a.src_off = src - data;
    b.cnt_fix.push_back({nullptr, b.rowcnt_words});
    b.rowcnt_words += rows;
    b.P.ntt.push_back(a);
    return (uint32_t)(b.P.ntt.size() - 1);
}

void ntt_tiles(Builder& b, uint32_t desc, uint16_t sub, size_t rows, int C, uint32_t d0, uint32_t n0, uint32_t done) {
    for (size_t r = 0; r < rows; ++r)
        for (int j = 0; j < C; ++j) b.tile(PK_NTT, sub, desc, (uint32_t)r, (uint32_t)j, d0, n0, kNoDep, 0, done);
}

ConvArgs conv_args(const fhe_ctx* ctx, const ConvTable& ct, const uint32_t* src, int nsrc, const int* src_mod,
                   uint32_t* dst, int ndst, const int* dst_mod, size_t limb, const uint2* s1, const uint2* s2,
                   int scale_lt) {
    ConvArgs ca;
    memset(&ca, 0, sizeof(ca));
    ca.src = src;
    ca.src_stride = limb;
    ca.nsrc = nsrc;
    for (int i = 0; i < nsrc; ++i) {
        ca.src_q[i] = ctx->mods[src_mod[i]];
        ca.hat_inv[i] = ct.hat_inv_h[i];
    }
    ca.hat_mod = ct.hat_mod;
    ca.nmod = (int)ctx->mods.size();
    ca.dst = dst;
    ca.dst_stride = limb;
    ca.ndst = ndst;
    for (int t = 0; t < ndst; ++t) ca.dst_mod[t] = (uint8_t)dst_mod[t];
    ca.dm = modvec(ctx, dst_mod, ndst);
    ca.L4 = limb / 4;
    ca.s1 = s1;
    ca.s2 = s2;
    ca.scale_lt = scale_lt;
    return ca;
}

// Stage tiles of one HMULT instance at scratch `sb`, stage by stage into per-stage lists so that
// the caller can interleave the instances of a wave. stage[k] collects stage k's tiles.
struct HmStages {
    std::vector<std::vector<PTile>> st;
    uint32_t c_tail = 0, n_tail = 0;
};

void hm_build(Builder& b, const HmInst& h, uint8_t* sb, uint32_t pred_ctr, uint32_t pred_need, HmStages* out) {
    const fhe_ctx* ctx = b.P.ctx;
    const fhe_op& o = b.P.ops[h.op];
    const int nl = h.nl, K = ctx->np, ext = h.ext, alpha = ctx->alpha, nq = ctx->nq, B = h.B, C = h.C;
    const size_t limb = h.limb, L4 = h.L4, N = h.N;
    uint32_t* s = (uint32_t*)sb;
    uint32_t* dd = s;                                 // (2, nl)
    uint32_t* d2 = dd + 2 * (size_t)nl * limb;        // (nl)
    uint32_t* ksx = d2 + (size_t)nl * limb;           // d2c (nl), then ModUp digits (dnum, ext)
    uint32_t* digits = ksx + (size_t)nl * limb;
    uint32_t* ks = digits + (size_t)h.dnum * ext * limb;
    uint32_t* y = ks + 2 * (size_t)ext * limb;
    uint32_t* last = ksx;                             // reuses d2c once the ModUp is complete
    uint32_t* tmp = y + 2 * (size_t)nl * limb;        // NTT temporaries
    uint32_t* t0 = tmp;
    uint32_t* t1 = t0 + h.rows_t0 * N;
    uint32_t* tlast = t1 + h.rows_t1 * N;             // (2 B rows) for the last limb's INTT
    uint32_t* tj[16];
    {
        uint32_t* q = tlast + 2 * (size_t)B * N;
        for (int j = 0; j < h.dnum; ++j) {
            tj[j] = j == 0 ? t0 : j == 1 ? t1 : q;
            if (j >= 2) q += (size_t)h.nd[j] * B * N;
        }
    }
    out->st.assign(10, {});
    const size_t mark0 = b.P.tiles.size();
    auto take = [&](int stage, size_t from) {
        out->st[stage].insert(out->st[stage].end(), b.P.tiles.begin() + from, b.P.tiles.end());
        b.P.tiles.resize(from);
    };
    const uint2* qlinv = ctx->ql_inv + (size_t)(nl - 1) * nq;
    int qidx[kMaxLimbs];
    for (int i = 0; i < nl; ++i) qidx[i] = i;
    // stage 0: tensor product (the first tiles wait for the slot's previous instance)
    const uint32_t c_ten = b.counter();
    b.P.ten.push_back(TensorArgs{o.a, o.b, dd, dd + (size_t)nl * limb, d2, nullptr, L4, (size_t)nl * L4,
                                 modvec(ctx, qidx, nl), qlinv, nl - 1});
    const uint32_t ten_desc = (uint32_t)(b.P.ten.size() - 1);
    for (int l = 0; l < nl; ++l)
        for (size_t c = 0; c < h.nch; ++c)
            b.tile(PK_TENSOR, 0, ten_desc, l, (uint32_t)c, pred_ctr, pred_need, kNoDep, 0, c_ten);
    const uint32_t n_ten = (uint32_t)(nl * h.nch);
    take(0, mark0);
    // stage 1: INTT of d2 into d2c (the local passes read d2, the cross passes write d2c)
    const uint32_t c_intt = b.counter();
    {
        LimbMap lm = contiguous_map(ctx, 0, nl);
        const uint32_t d = ntt_stage(b, h.logN, true, ksx, B, &lm, nullptr, (size_t)nl * B, t0, nullptr, d2);
        const size_t m = b.P.tiles.size();
        ntt_tiles(b, d, (uint16_t)(log_c_of(h.logN) | kSubInv), (size_t)nl * B, C, c_ten, n_ten, c_intt);
        take(1, m);
    }
    const uint32_t n_intt = (uint32_t)((size_t)nl * B * C);
    // stages 2, 3: per slice, Conv Q_j -> (Q_l \ Q_j) u P and the NTT of the converted limbs
    const uint32_t c_modup = b.counter();
    uint32_t n_modup = 0;
    for (int j = 0; j < h.dnum; ++j) {
        const int lo = j * alpha, hi = std::min(nl, (j + 1) * alpha);
        const ConvTable& ct = ctx->modup[j][hi - lo - 1];
        int smod[16], dmod[kMaxLimbs], nd = 0;
        for (int i = lo; i < hi; ++i) smod[i - lo] = i;
        for (int t = 0; t < nl; ++t)
            if (t < lo || t >= hi) dmod[nd++] = t;
        for (int k = 0; k < K; ++k) dmod[nd++] = nq + k;
        uint32_t* dst = digits + (size_t)j * ext * limb;
        b.P.conv.push_back(conv_args(ctx, ct, ksx + (size_t)lo * limb, hi - lo, smod, dst, nd, dmod, limb, nullptr,
                                     nullptr, 0));
        const uint32_t cd = (uint32_t)(b.P.conv.size() - 1);
        const uint32_t c_conv = b.counter();
        size_t m = b.P.tiles.size();
        for (size_t c = 0; c < h.nconv; ++c) b.tile(PK_CONV, 0, cd, 0, (uint32_t)c, c_intt, n_intt, kNoDep, 0, c_conv);
        take(2, m);
        LimbMap lm;
        memset(&lm, 0, sizeof(lm));
        for (int t = 0; t < nd; ++t) {
            lm.mod[t] = (uint8_t)dmod[t];
            lm.q[t] = ctx->mods[dmod[t]];
        }
        const uint32_t d = ntt_stage(b, h.logN, false, dst, B, &lm, nullptr, (size_t)nd * B, tj[j], nullptr);
        m = b.P.tiles.size();
        ntt_tiles(b, d, (uint16_t)log_c_of(h.logN), (size_t)nd * B, C, c_conv, (uint32_t)h.nconv, c_modup);
        take(3, m);
        n_modup += (uint32_t)((size_t)nd * B * C);
    }
    // stage 4: inner product with the key over all slices
    const uint32_t c_ip = b.counter();
    {
        int ext_mod[kMaxLimbs];
        for (int t = 0; t < ext; ++t) ext_mod[t] = t < nl ? t : nq + (t - nl);
        IpArgs ia;
        memset(&ia, 0, sizeof(ia));
        ia.d2 = d2;
        ia.tmp = digits;
        ia.evk = o.evk;
        ia.ks = ks;
        ia.nl = nl;
        ia.alpha = alpha;
        ia.dnum = h.dnum;
        ia.ext = ext;
        ia.nq = nq;
        ia.nmod = (int)ctx->mods.size();
        ia.L4 = L4;
        ia.N4 = N / 4;
        ia.m = modvec(ctx, ext_mod, ext);
        ip_set_post(ctx, ia, nl, ext, nl - 1, true);
        b.P.ip.push_back(ia);
        const size_t m = b.P.tiles.size();
        for (int t = 0; t < ext; ++t)
            for (size_t c = 0; c < h.nch; ++c)
                b.tile(PK_IP, 0, (uint32_t)(b.P.ip.size() - 1), t, (uint32_t)c, c_modup, n_modup, kNoDep, 0, c_ip);
        take(4, m);
    }
    const uint32_t n_ip = (uint32_t)(ext * h.nch);
    // stage 5: INTT of each component's P limbs; the last limb's relinearisation
    const uint32_t c_relin = b.counter();
    uint32_t c_pintt[2];
    {
        const LimbMap pm = contiguous_map(ctx, nq, K);
        for (int c = 0; c < 2; ++c) {
            c_pintt[c] = b.counter();
            const uint32_t d = ntt_stage(b, h.logN, true, ks + ((size_t)c * ext + nl) * limb, B, &pm, nullptr,
                                         (size_t)K * B, c == 0 ? t0 : t1, nullptr);
            const size_t m = b.P.tiles.size();
            ntt_tiles(b, d, (uint16_t)(log_c_of(h.logN) | kSubInv), (size_t)K * B, C, c_ip, n_ip, c_pintt[c]);
            take(5, m);
        }
        b.P.last.push_back(LastArgs{dd, ks, y, last, ctx->p_inv_h[nl - 1], ctx->mods[nl - 1], nl, ext, L4});
        const size_t m = b.P.tiles.size();
        for (int c = 0; c < 2; ++c)
            for (size_t ch = 0; ch < h.nch; ++ch)
                b.tile(PK_RELIN_LAST, 0, (uint32_t)(b.P.last.size() - 1), c, (uint32_t)ch, c_ip, n_ip, kNoDep, 0,
                       c_relin);
        take(5, m);
    }
    const uint32_t last_desc = (uint32_t)(b.P.last.size() - 1);
    const uint32_t n_relin = (uint32_t)(2 * h.nch);
    // stage 6: ModDown Conv P -> Q of each component (scaled for the fused tail); the last
    // limb's INTT
    const uint32_t c_md = b.counter(), c_lintt = b.counter();
    {
        int smod[16], dmod[kMaxLimbs];
        for (int k = 0; k < K; ++k) smod[k] = nq + k;
        for (int t = 0; t < nl; ++t) dmod[t] = t;
        for (int c = 0; c < 2; ++c) {
            b.P.conv.push_back(conv_args(ctx, ctx->moddown, ks + ((size_t)c * ext + nl) * limb, K, smod,
                                         y + (size_t)c * nl * limb, nl, dmod, limb, ctx->p_inv, qlinv, nl - 1));
            const size_t m = b.P.tiles.size();
            for (size_t ch = 0; ch < h.nconv; ++ch)
                b.tile(PK_CONV, 0, (uint32_t)(b.P.conv.size() - 1), 0, (uint32_t)ch, c_pintt[c],
                       (uint32_t)((size_t)K * B * C), kNoDep, 0, c_md);
            take(6, m);
        }
        LimbMap lm;
        memset(&lm, 0, sizeof(lm));
        lm.mod[0] = lm.mod[1] = (uint8_t)(nl - 1);
        lm.q[0] = lm.q[1] = ctx->mods[nl - 1];
        const uint32_t d = ntt_stage(b, h.logN, true, last, B, &lm, nullptr, 2 * (size_t)B, tlast, nullptr);
        const size_t m = b.P.tiles.size();
        ntt_tiles(b, d, (uint16_t)(log_c_of(h.logN) | kSubInv), 2 * (size_t)B, C, c_relin, n_relin, c_lintt);
        take(6, m);
    }
    // stage 7: last = INTT(u) - y_l P^-1
    const uint32_t c_fix = b.counter();
    {
        const size_t m = b.P.tiles.size();
        for (int c = 0; c < 2; ++c)
            for (size_t ch = 0; ch < h.nch; ++ch)
                b.tile(PK_LAST_FIX, 0, last_desc, c, (uint32_t)ch, c_lintt, (uint32_t)(2 * (size_t)B * C), c_md,
                       (uint32_t)(2 * h.nconv), c_fix);
        take(7, m);
    }
    // stage 8: forward NTT of z' with the fused RESCALE tail, writing the output
    const uint32_t c_tail = b.counter();
    {
        const int nout = nl - 1;
        LimbMap qm2;
        memset(&qm2, 0, sizeof(qm2));
        for (int c = 0; c < 2; ++c)
            for (int i = 0; i < nout; ++i) {
                qm2.mod[c * nout + i] = (uint8_t)i;
                qm2.q[c * nout + i] = ctx->mods[i];
            }
        HmultTail tl;
        tl.y = y;
        tl.last = last;
        tl.ks = ks;
        tl.d = dd;
        tl.out = o.out;
        tl.qlinv = qlinv;
        tl.ql = ctx->mods[nl - 1];
        tl.nl = nl;
        tl.nout = nout;
        tl.ext = ext;
        const size_t rows = 2 * (size_t)nout * B;
        const uint32_t d = ntt_stage(b, h.logN, false, o.out, B, &qm2, nullptr, rows, t0, &tl);
        const size_t m = b.P.tiles.size();
        ntt_tiles(b, d, (uint16_t)(log_c_of(h.logN) | kSubTail), rows, C, c_fix, (uint32_t)(2 * h.nch), c_tail);
        take(8, m);
        out->c_tail = c_tail;
        out->n_tail = (uint32_t)(rows * C);
    }
}

size_t hm_bytes(const fhe_ctx* ctx, HmInst& h) {
    const int K = ctx->np;
    h.rows_t0 = (size_t)h.B * std::max({(size_t)h.nl, (size_t)h.nd[0], (size_t)K, 2 * (size_t)(h.nl - 1)});
    h.rows_t1 = (size_t)h.B * std::max((size_t)K, h.dnum > 1 ? (size_t)h.nd[1] : 0);
    size_t extra_rows = 2 * (size_t)h.B;
    for (int j = 2; j < h.dnum; ++j) extra_rows += (size_t)h.nd[j] * h.B;
    const size_t words = hm_limbs(h.nl, K, h.dnum) * h.limb + (h.rows_t0 + h.rows_t1 + extra_rows) * h.N;
    return align_up(words * 4);
}

// Builds every table for scratch base `base` (nullptr: sizing only).
int build_tables(PersistPlan& P, uint8_t* base) {
    P.tiles.clear();
    P.ntt.clear();
    P.ten.clear();
    P.conv.clear();
    P.ip.clear();
    P.last.clear();
    P.rows.clear();
    Builder b(P, base);
    // standalone NTT operations: one stage per (logN, direction); row tables with absolute pointers
    std::vector<std::vector<PTile>> ntt_part;
    size_t temp_off = 0;
    std::vector<std::pair<uint32_t, int>> keys;
    for (int i : P.ntt_ops) {
        const fhe_op& o = P.ops[i];
        const std::pair<uint32_t, int> k{o.logN, o.kind == FHE_OPK_NTT_INV ? 1 : 0};
        if (std::find(keys.begin(), keys.end(), k) == keys.end()) keys.push_back(k);
    }
    std::vector<PTile> ntt_tiles_all;
    for (const auto& k : keys) {
        const size_t r0 = P.rows.size();
        for (int i : P.ntt_ops) {
            const fhe_op& o = P.ops[i];
            if (o.logN != k.first || (o.kind == FHE_OPK_NTT_INV ? 1 : 0) != k.second) continue;
            const size_t N = (size_t)1 << o.logN;
            for (int l = 0; l < o.n_limbs; ++l)
                for (int bb = 0; bb < o.batch; ++bb)
                    P.rows.push_back(RowRef{o.data + ((size_t)l * o.batch + bb) * N, (uint32_t)(o.first_limb + l), 0});
        }
        const size_t nrows = P.rows.size() - r0;
        const size_t N = (size_t)1 << k.first;
        uint32_t* temp = base ? (uint32_t*)(base + P.ntt_temp_off + temp_off) : nullptr;
        temp_off += align_up(nrows * N * 4);
        // the row table's device address is known once d_rows exists (bind); sizing passes null
        const RowRef* rt = P.d_rows ? P.d_rows + r0 : reinterpret_cast<const RowRef*>(16);
        const uint32_t d = ntt_stage(b, k.first, k.second != 0, nullptr, 1, nullptr, rt, nrows, temp, nullptr);
        const int C = 1 << log_c_of(k.first);
        const size_t m = P.tiles.size();
        ntt_tiles(b, d, (uint16_t)(log_c_of(k.first) | (k.second ? kSubInv : 0)), nrows, C, kNoDep, 0, kNoDep);
        ntt_tiles_all.insert(ntt_tiles_all.end(), P.tiles.begin() + m, P.tiles.end());
        P.tiles.resize(m);
    }
    const size_t ntt_temp_bytes = temp_off;
    // HMULT instances in waves of P.slots, stage by stage
    std::vector<PTile> order;
    const int nw = P.hm.empty() ? 1 : (int)((P.hm.size() + P.slots - 1) / P.slots);
    std::vector<uint32_t> slot_ctr(P.slots, kNoDep), slot_need(P.slots, 0);
    size_t ntt_next = 0;
    for (int w = 0; w < nw; ++w) {
        std::vector<HmStages> st;
        for (size_t k = (size_t)w * P.slots; k < P.hm.size() && k < (size_t)(w + 1) * P.slots; ++k) {
            const HmInst& h = P.hm[k];
            // while sizing (no base yet) the instance tables are built against offset 0
            uint8_t* sb = (base ? base : (uint8_t*)kAlign) + P.slot_off + (size_t)h.slot * P.slot_bytes;
            HmStages hs;
            hm_build(b, h, sb, slot_ctr[h.slot], slot_ctr[h.slot] == kNoDep ? 0 : slot_need[h.slot], &hs);
            slot_ctr[h.slot] = hs.c_tail;
            slot_need[h.slot] = hs.n_tail;
            st.push_back(std::move(hs));
        }
        for (int s = 0; s < 10; ++s) {
            for (auto& hs : st)
                if (s < (int)hs.st.size()) order.insert(order.end(), hs.st[s].begin(), hs.st[s].end());
            if (s == 0) {  // this wave's share of the stand-alone NTT tiles fills the pipeline's start
                const size_t share = (ntt_tiles_all.size() - ntt_next + (nw - w) - 1) / (nw - w);
                order.insert(order.end(), ntt_tiles_all.begin() + ntt_next, ntt_tiles_all.begin() + ntt_next + share);
                ntt_next += share;
            }
        }
    }
    P.tiles = std::move(order);
    // row-counter offsets of the NTT stages (after the stage counters)
    P.ctr_words = b.nctr + b.rowcnt_words;
    for (size_t s = 0; s < P.ntt.size(); ++s) {
        const size_t off = b.nctr + b.cnt_fix[s].second;
        P.ntt[s].cnt = base ? reinterpret_cast<int*>(base) + off : nullptr;
    }
    if (!base) {
        P.ntt_temp_off = align_up(P.ctr_words * 4);
        P.slot_off = P.ntt_temp_off + align_up(ntt_temp_bytes);
        P.scratch_bytes = P.slot_off + (size_t)P.slots * P.slot_bytes;
    }
    return FHE_OK;
}

template <typename T>
int upload_vec(T** d, const std::vector<T>& h, cudaStream_t st) {
    if (h.empty()) return FHE_OK;
    FHE_CUDA_TRY(cudaMemcpyAsync(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, st));
    return FHE_OK;
}
template <typename T>
int upload_vec(Slot<T>** d, const std::vector<T>& h, cudaStream_t st) {
    if (h.empty()) return FHE_OK;
    std::vector<Slot<T>> padded(h.size());
    for (size_t i = 0; i < h.size(); ++i) padded[i].v = h[i];
    FHE_CUDA_TRY(cudaMemcpyAsync(*d, padded.data(), padded.size() * sizeof(Slot<T>), cudaMemcpyHostToDevice, st));
    FHE_CUDA_TRY(cudaStreamSynchronize(st));  // `padded` is freed on return
    return FHE_OK;
}
template <typename T>
int alloc_vec(T** d, size_t n) {
    *d = nullptr;
    if (n == 0) return FHE_OK;
    cudaError_t e = cudaMalloc((void**)d, n * sizeof(T));
    if (e != cudaSuccess) return set_error(FHE_ENOMEM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
    return FHE_OK;
}

}  // namespace

int persist_create(const fhe_ctx* ctx, const fhe_op* ops, int n, const std::vector<int>& idx, size_t slot_budget,
                   PersistPlan** out) {
    *out = nullptr;
    PersistPlan* P = new PersistPlan();
    P->ctx = ctx;
    P->ops.assign(ops, ops + n);
    for (int i : idx) {
        const fhe_op& o = ops[i];
        if (o.batch == 0) continue;
        if (o.kind == FHE_OPK_HMULT) {
            HmInst h;
            memset(&h, 0, sizeof(h));
            h.op = i;
            h.logN = o.logN;
            h.nl = o.n_limbs;
            h.B = o.batch;
            h.dnum = (o.n_limbs + ctx->alpha - 1) / ctx->alpha;
            h.ext = o.n_limbs + ctx->np;
            h.C = 1 << log_c_of(o.logN);
            h.N = (size_t)1 << o.logN;
            h.limb = h.N * h.B;
            h.L4 = h.limb / 4;
            h.nch = (h.L4 + kChunk4 - 1) / kChunk4;
            h.nconv = (2 * h.L4 + kConvChunk2 - 1) / kConvChunk2;
            for (int j = 0; j < h.dnum; ++j)
                h.nd[j] = h.ext - (std::min(h.nl, (j + 1) * ctx->alpha) - j * ctx->alpha);
            h.bytes = hm_bytes(ctx, h);
            P->hm.push_back(h);
        } else {
            P->ntt_ops.push_back(i);
        }
    }
    // largest instances first; slots sized for the largest, as many as the budget allows
    std::stable_sort(P->hm.begin(), P->hm.end(), [](const HmInst& a, const HmInst& b) { return a.bytes > b.bytes; });
    P->slot_bytes = P->hm.empty() ? 0 : P->hm[0].bytes;
    if (!P->hm.empty()) {
        size_t s = std::max<size_t>(1, slot_budget / P->slot_bytes);
        P->slots = (int)std::min<size_t>(s, P->hm.size());
        for (size_t k = 0; k < P->hm.size(); ++k) P->hm[k].slot = (int)(k % P->slots);
    }
    int rc = build_tables(*P, nullptr);  // sizes and tile order only
    if (rc == FHE_OK && P->tiles.size() > (size_t)INT32_MAX) rc = set_error(FHE_EINVAL, "too many tiles");
    if (rc == FHE_OK) rc = alloc_vec(&P->d_tiles, P->tiles.size());
    if (rc == FHE_OK) rc = alloc_vec(&P->d_ntt, P->ntt.size());
    if (rc == FHE_OK) rc = alloc_vec(&P->d_ten, P->ten.size());
    if (rc == FHE_OK) rc = alloc_vec(&P->d_conv, P->conv.size());
    if (rc == FHE_OK) rc = alloc_vec(&P->d_ip, P->ip.size());
    if (rc == FHE_OK) rc = alloc_vec(&P->d_last, P->last.size());
    if (rc == FHE_OK) rc = alloc_vec(&P->d_rows, P->rows.size());
    if (rc == FHE_OK) {
        const size_t smem = PadLayout<kLogPT>::kWords * 4;
        cudaError_t e = cudaFuncSetAttribute(k_persist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int per_sm = 0;
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_persist, kPT, smem);
        if (e != cudaSuccess) rc = cuda_error(e, "k_persist occupancy");
        P->grid = std::max(1, per_sm) * ctx->num_sms;
    }
    // about two seconds at the maximum SM clock
    P->wait_cycles = 4000000000LL;
    if (rc != FHE_OK) {
        persist_destroy(P);
        return rc;
    }
    *out = P;
    return FHE_OK;
}

size_t persist_scratch_bytes(const PersistPlan* P) { return P ? P->scratch_bytes : 0; }
size_t persist_tiles(const PersistPlan* P) { return P ? P->tiles.size() : 0; }

int persist_run(PersistPlan* P, void* scratch, cudaStream_t st) {
    if (!P || P->tiles.empty()) return FHE_OK;
    if (P->bound != scratch) {
        // tables hold absolute scratch addresses: rebuild and upload them for this buffer (not
        // allowed while the stream is being captured; runs on another buffer must be complete)
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        FHE_CUDA_TRY(cudaStreamIsCapturing(st, &cs));
        if (cs != cudaStreamCaptureStatusNone)
            return set_error(FHE_EINVAL, "batch plan: first run on a new scratch buffer inside a stream capture");
        FHE_CUDA_TRY(cudaStreamSynchronize(st));
        int rc = build_tables(*P, (uint8_t*)scratch);
        if (rc) return rc;
        if ((rc = upload_vec(&P->d_tiles, P->tiles, st)) || (rc = upload_vec(&P->d_ntt, P->ntt, st)) ||
            (rc = upload_vec(&P->d_ten, P->ten, st)) || (rc = upload_vec(&P->d_conv, P->conv, st)) ||
            (rc = upload_vec(&P->d_ip, P->ip, st)) || (rc = upload_vec(&P->d_last, P->last, st)) ||
            (rc = upload_vec(&P->d_rows, P->rows, st)))
            return rc;
        FHE_CUDA_TRY(cudaStreamSynchronize(st));
        P->bound = scratch;
    }
    FHE_CUDA_TRY(cudaMemsetAsync(scratch, 0, P->ctr_words * 4, st));
    PParams p;
    p.tiles = P->d_tiles;
    p.ntiles = (int)P->tiles.size();
    p.ctr = (unsigned*)scratch;
    p.ntt = P->d_ntt;
    p.ten = P->d_ten;
    p.conv = P->d_conv;
    p.ip = P->d_ip;
    p.last = P->d_last;
    p.status = P->ctx->d_status;
    p.wait_cycles = P->wait_cycles;
    const size_t smem = PadLayout<kLogPT>::kWords * 4;
    const int grid = std::min<int>(P->grid, p.ntiles);
    k_persist<<<grid, kPT, smem, st>>>(p);
    FHE_CUDA_TRY(cudaGetLastError());
    return FHE_OK;
}

void persist_destroy(PersistPlan* P) {
    if (!P) return;
    cudaFree(P->d_tiles);
    cudaFree(P->d_ntt);
    cudaFree(P->d_ten);
    cudaFree(P->d_conv);
    cudaFree(P->d_ip);
    cudaFree(P->d_last);
    cudaFree(P->d_rows);
    delete P;
}

// Self-test of the queue's bounded wait: one tile whose dependency counter nothing increments.
int persist_selftest_timeout(const fhe_ctx* ctx, long long limit_cycles, cudaStream_t st) {
    PTile t{PK_NOP, 0, 0, 0, 0, {2, kNoDep}, {1, 0}, kNoDep, 0};
    void* mem = nullptr;
    FHE_CUDA_TRY(cudaMalloc(&mem, 256));
    PTile* d_t = (PTile*)((uint8_t*)mem + 64);
    FHE_CUDA_TRY(cudaMemsetAsync(mem, 0, 64, st));
    FHE_CUDA_TRY(cudaMemcpyAsync(d_t, &t, sizeof(t), cudaMemcpyHostToDevice, st));
    PParams p;
    memset(&p, 0, sizeof(p));
    p.tiles = d_t;
    p.ntiles = 1;
    p.ctr = (unsigned*)mem;
    p.status = ctx->d_status;
    p.wait_cycles = limit_cycles;
    const size_t smem = PadLayout<kLogPT>::kWords * 4;
    FHE_CUDA_TRY(cudaFuncSetAttribute(k_persist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_persist<<<1, kPT, smem, st>>>(p);
    FHE_CUDA_TRY(cudaGetLastError());
    const cudaError_t e = cudaStreamSynchronize(st);  // the host copy of the tile is on this stack frame
    cudaFree(mem);
    if (e != cudaSuccess) return cuda_error(e, "cudaStreamSynchronize");
    return FHE_OK;
}

}  // namespace fhe

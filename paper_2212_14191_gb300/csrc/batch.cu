// Operation-level batching (Sec. IV-D) of many independent NTT / INTT / HMULT operations of
// uneven ring degree and level, submitted as one plan and replayed as one CUDA graph launch.
//
// Operations at N >= 2^14 go through the persistent engine of persist.cu: one launch whose CTAs
// pop the tiles of every operation's stages from a device queue. The grouped form below is used
// for smaller ring degrees (and for every operation when a plan asks for it): every limb
// transform of one ring degree and direction becomes one row of a single row-table NTT launch
// (rows may live in any buffer); HMULTs of the same (N, limbs, key) are gathered into one
// (2, L, B, N) batch, run through the batched HMULT pipeline and scattered back. Gathers and
// scatters are one copy kernel each, driven by a device table of segments.
#include <algorithm>
#include <map>
#include <tuple>

#include "common.cuh"
#include "persist.h"

namespace fhe {
namespace {

struct Seg {
    uint64_t src;  // absolute address, or offset from the scratch base when (flags & 1)
    uint64_t dst;  // absolute address, or offset from the scratch base when (flags & 2)
    uint64_t n4;   // 16-byte words
    uint64_t flags;
};

__global__ void k_segcopy(const Seg* __restrict__ segs, uint8_t* base) {
    const Seg s = segs[blockIdx.y];
    const uint4* src = reinterpret_cast<const uint4*>((s.flags & 1) ? base + s.src : reinterpret_cast<uint8_t*>(s.src));
    uint4* dst = reinterpret_cast<uint4*>((s.flags & 2) ? base + s.dst : reinterpret_cast<uint8_t*>(s.dst));
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < s.n4; i += (uint64_t)gridDim.x * blockDim.x)
        dst[i] = __ldg(src + i);
}

struct NttGroup {
    uint32_t logN;
    bool inverse;
    int nrows;
    RowRef* d_rows;
};

struct HmGroup {
    uint32_t logN;
    int nl, btot;
    const uint32_t* evk;
    Seg* d_in;
    int nin;
    Seg* d_out;
    int nout;
    uint64_t max_seg4;
    size_t a_off, b_off, o_off, s_off, s_bytes;
};

}  // namespace
}  // namespace fhe

struct fhe_batch {
    const fhe_ctx* ctx = nullptr;
    std::vector<fhe::NttGroup> ntt;
    std::vector<fhe::HmGroup> hm;
    size_t scratch_bytes = 0;
    std::vector<void*> allocs;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    fhe::PersistPlan* persist = nullptr;  // operations at N >= 2^14 (persistent mode)
    int n_ops = 0;
    int n_launch = 0;  // kernels launched per run (excluding those inside library calls' counts)
};

using namespace fhe;

namespace {

template <typename T>
int upload(fhe_batch* b, T** p, const std::vector<T>& h) {
    void* v = nullptr;
    if (h.empty()) {
        *p = nullptr;
        return FHE_OK;
    }
    cudaError_t e = cudaMalloc(&v, h.size() * sizeof(T));
    if (e != cudaSuccess) return set_error(FHE_ENOMEM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
    b->allocs.push_back(v);
    e = cudaMemcpy(v, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_error(e, "cudaMemcpy");
    *p = (T*)v;
    return FHE_OK;
}

bool al16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

int run_batch(const fhe_batch* b, void* scratch, cudaStream_t st) {
    const fhe_ctx* ctx = b->ctx;
    int rc;
    uint8_t* base = (uint8_t*)scratch;
    // the NTT groups run first and use the start of the scratch for their two-pass chunks
    for (const NttGroup& g : b->ntt) {
        NttScratch ns;
        ns.bytes = ntt_region_bytes(g.logN, (size_t)g.nrows);
        if (ns.bytes) ns.p = (uint32_t*)base;
        if ((rc = ntt_u32_rows(ctx, g.logN, g.inverse, g.d_rows, g.nrows, st, ns))) return rc;
    }
    for (const HmGroup& g : b->hm) {
        const unsigned gx = (unsigned)std::min<uint64_t>((g.max_seg4 + 255) / 256, 1024);
        k_segcopy<<<dim3(gx, g.nin), 256, 0, st>>>(g.d_in, base);
        FHE_CUDA_TRY(cudaGetLastError());
        if ((rc = fhe_hmult(ctx, g.logN, g.nl, g.btot, (const uint32_t*)(base + g.a_off), (const uint32_t*)(base + g.b_off),
                            g.evk, (uint32_t*)(base + g.o_off), base + g.s_off, g.s_bytes, st)))
            return rc;
        k_segcopy<<<dim3(gx, g.nout), 256, 0, st>>>(g.d_out, base);
        FHE_CUDA_TRY(cudaGetLastError());
    }
    // the persistent engine runs after the grouped operations and reuses the same scratch
    if (b->persist) return persist_run(b->persist, scratch, st);
    return FHE_OK;
}

}  // namespace

extern "C" {

int fhe_batch_create(const fhe_ctx* ctx, const fhe_op* ops, int n, fhe_batch** out) {
    return fhe_batch_create_ex(ctx, ops, n, FHE_BATCH_PERSISTENT, 0, out);
}

int fhe_batch_create_ex(const fhe_ctx* ctx, const fhe_op* ops, int n, int mode, size_t slot_bytes, fhe_batch** out) {
    FHE_CHECK(out != nullptr, "out is NULL");
    *out = nullptr;
    FHE_CHECK(ctx != nullptr, "ctx is NULL");
    FHE_CHECK(n >= 0 && (n == 0 || ops != nullptr), "bad op list");
    FHE_CHECK(mode == FHE_BATCH_PERSISTENT || mode == FHE_BATCH_GROUPED, "unknown batch mode");
    std::vector<int> persistent;  // operations for the persistent engine
    const int nmod = (int)ctx->mods.size();
    std::map<std::pair<uint32_t, int>, std::vector<RowRef>> rows;  // (logN, inverse) -> rows
    std::map<std::tuple<uint32_t, int, const uint32_t*>, std::vector<int>> hm;  // (logN, nl, evk) -> ops
    for (int i = 0; i < n; ++i) {
        const fhe_op& o = ops[i];
        FHE_CHECK(o.logN >= FHE_LOGN_MIN && o.logN <= ctx->logN_max, "op: logN out of range");
        FHE_CHECK(o.batch >= 0, "op: batch < 0");
        const size_t N = (size_t)1 << o.logN;
        const bool pers = mode == FHE_BATCH_PERSISTENT && o.logN >= 14;
        if (o.kind == FHE_OPK_NTT_FWD || o.kind == FHE_OPK_NTT_INV) {
            FHE_CHECK(o.n_limbs >= 1 && o.first_limb >= 0 && o.first_limb + o.n_limbs <= nmod, "op: limb range");
            FHE_CHECK(o.batch == 0 || (o.data && al16(o.data)), "op: data NULL or misaligned");
            if (pers) {
                persistent.push_back(i);
                continue;
            }
            auto& v = rows[{o.logN, o.kind == FHE_OPK_NTT_INV ? 1 : 0}];
            for (int l = 0; l < o.n_limbs; ++l)
                for (int bb = 0; bb < o.batch; ++bb)
                    v.push_back(RowRef{o.data + ((size_t)l * o.batch + bb) * N, (uint32_t)(o.first_limb + l), 0});
        } else if (o.kind == FHE_OPK_HMULT) {
            FHE_CHECK(ctx->np > 0, "op: HMULT needs special primes");
            FHE_CHECK(o.n_limbs >= 2 && o.n_limbs <= ctx->nq, "op: HMULT n_limbs out of [2, nq]");
            FHE_CHECK(o.batch == 0 || (o.a && o.b && o.evk && o.out && al16(o.a) && al16(o.b) && al16(o.out)),
                      "op: HMULT pointer NULL or misaligned");
            if (pers)
                persistent.push_back(i);
            else if (o.batch > 0)
                hm[std::make_tuple(o.logN, o.n_limbs, o.evk)].push_back(i);
        } else {
            return set_error(FHE_EINVAL, "op: unknown kind");
        }
    }
    fhe_batch* b = new fhe_batch();
    b->ctx = ctx;
    b->n_ops = n;
    int rc = FHE_OK;
    for (auto& kv : rows) {
        NttGroup g;
        g.logN = kv.first.first;
        g.inverse = kv.first.second != 0;
        g.nrows = (int)kv.second.size();
        if ((rc = upload(b, &g.d_rows, kv.second))) break;
        b->scratch_bytes = std::max(b->scratch_bytes, ntt_region_bytes(g.logN, (size_t)g.nrows));
        b->ntt.push_back(g);
        b->n_launch += 1;
    }
    for (auto it = hm.begin(); rc == FHE_OK && it != hm.end(); ++it) {
        HmGroup g;
        g.logN = std::get<0>(it->first);
        g.nl = std::get<1>(it->first);
        g.evk = std::get<2>(it->first);
        const size_t N = (size_t)1 << g.logN;
        int btot = 0;
        for (int i : it->second) btot += ops[i].batch;
        g.btot = btot;
        const size_t limb = (size_t)btot * N * 4;  // bytes of one limb of the gathered batch
        g.a_off = 0;
        g.b_off = g.a_off + 2 * (size_t)g.nl * limb;
        g.o_off = g.b_off + 2 * (size_t)g.nl * limb;
        g.s_off = g.o_off + 2 * (size_t)(g.nl - 1) * limb;
        g.s_bytes = fhe_scratch_bytes(ctx, FHE_OP_HMULT, g.logN, g.nl, btot);
        b->scratch_bytes = std::max(b->scratch_bytes, g.s_off + g.s_bytes);
        std::vector<Seg> in, outs;
        g.max_seg4 = 0;
        int bo = 0;
        for (int i : it->second) {
            const fhe_op& o = ops[i];
            const uint64_t n4 = (uint64_t)o.batch * N / 4;
            g.max_seg4 = std::max(g.max_seg4, n4);
            for (int c = 0; c < 2; ++c)
                for (int l = 0; l < g.nl; ++l) {
                    const size_t src_el = ((size_t)c * g.nl + l) * o.batch * N;
                    const size_t dst_b = (((size_t)c * g.nl + l) * btot + bo) * N * 4;
                    in.push_back(Seg{(uint64_t)(uintptr_t)(o.a + src_el), g.a_off + dst_b, n4, 2});
                    in.push_back(Seg{(uint64_t)(uintptr_t)(o.b + src_el), g.b_off + dst_b, n4, 2});
                    if (l < g.nl - 1) {
                        const size_t osrc_b = (((size_t)c * (g.nl - 1) + l) * btot + bo) * N * 4;
                        const size_t odst_el = ((size_t)c * (g.nl - 1) + l) * o.batch * N;
                        outs.push_back(Seg{g.o_off + osrc_b, (uint64_t)(uintptr_t)(o.out + odst_el), n4, 1});
                    }
                }
            bo += o.batch;
        }
        g.nin = (int)in.size();
        g.nout = (int)outs.size();
        if (g.nin > 65535 || g.nout > 65535) {
            rc = set_error(FHE_EINVAL, "too many HMULT segments in one group");
            break;
        }
        if ((rc = upload(b, &g.d_in, in))) break;
        if ((rc = upload(b, &g.d_out, outs))) break;
        b->hm.push_back(g);
    }
    if (rc == FHE_OK && !persistent.empty()) {
        const size_t budget = slot_bytes ? slot_bytes : ((size_t)8 << 30);
        rc = persist_create(ctx, ops, n, persistent, budget, &b->persist);
        if (rc == FHE_OK) {
            b->scratch_bytes = std::max(b->scratch_bytes, persist_scratch_bytes(b->persist));
            b->n_launch += 2;
        }
    }
    if (rc != FHE_OK) {
        fhe_batch_destroy(b);
        return rc;
    }
    if (b->scratch_bytes == 0) b->scratch_bytes = 16;
    *out = b;
    return FHE_OK;
}

size_t fhe_batch_scratch_bytes(const fhe_batch* b) { return b ? b->scratch_bytes : 0; }

int fhe_batch_run(const fhe_batch* b, void* scratch, size_t scratch_bytes, void* stream) {
    FHE_CHECK(b != nullptr, "batch is NULL");
    FHE_CHECK(scratch != nullptr && al16(scratch), "scratch NULL or misaligned");
    if (scratch_bytes < b->scratch_bytes) return set_error(FHE_ENOMEM, "scratch too small");
    return run_batch(b, scratch, (cudaStream_t)stream);
}

int fhe_batch_capture(fhe_batch* b, void* scratch, size_t scratch_bytes) {
    FHE_CHECK(b != nullptr, "batch is NULL");
    FHE_CHECK(scratch != nullptr && al16(scratch), "scratch NULL or misaligned");
    if (scratch_bytes < b->scratch_bytes) return set_error(FHE_ENOMEM, "scratch too small");
    cudaStream_t st;
    FHE_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    // one eager run first: per-kernel attributes and occupancy are set up outside the capture
    int rc = run_batch(b, scratch, st);
    if (rc == FHE_OK) {
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = cuda_error(e, "cudaStreamSynchronize");
    }
    if (rc == FHE_OK) {
        cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) rc = cuda_error(e, "cudaStreamBeginCapture");
        if (rc == FHE_OK) {
            rc = run_batch(b, scratch, st);
            cudaGraph_t g = nullptr;
            e = cudaStreamEndCapture(st, &g);
            if (rc == FHE_OK && e != cudaSuccess) rc = cuda_error(e, "cudaStreamEndCapture");
            if (rc == FHE_OK) {
                if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
                if (b->graph) cudaGraphDestroy(b->graph);
                b->graph = g;
                e = cudaGraphInstantiate(&b->graph_exec, g, 0);
                if (e != cudaSuccess) rc = cuda_error(e, "cudaGraphInstantiate");
            } else if (g) {
                cudaGraphDestroy(g);
            }
        }
    }
    cudaStreamDestroy(st);
    return rc;
}

int fhe_batch_launch(const fhe_batch* b, void* stream) {
    FHE_CHECK(b != nullptr && b->graph_exec != nullptr, "batch has no captured graph");
    FHE_CUDA_TRY(cudaGraphLaunch(b->graph_exec, (cudaStream_t)stream));
    return FHE_OK;
}

int fhe_batch_destroy(fhe_batch* b) {
    if (!b) return FHE_OK;
    if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (void* v : b->allocs) cudaFree(v);
    persist_destroy(b->persist);
    delete b;
    return FHE_OK;
}

int fhe_selftest_queue_timeout(const fhe_ctx* ctx, long long limit_cycles, void* stream) {
    FHE_CHECK(ctx != nullptr, "ctx is NULL");
    FHE_CHECK(limit_cycles > 0 && limit_cycles <= 4000000000LL, "limit_cycles out of (0, 4e9]");
    return persist_selftest_timeout(ctx, limit_cycles, (cudaStream_t)stream);
}

}  // extern "C"

// Plain 32-bit negacyclic NTT / INTT on CUDA cores: tables, kernel variants and dispatch for
// the single-CTA shapes and clusters of two (the kernels are in ntt_u32_kernels.cuh; the
// shapes with clusters of four or more CTAs are instantiated in ntt_u32_wide.cu so that the
// two halves compile in parallel).
#include "ntt_u32_kernels.cuh"

namespace fhe {

namespace {
uint32_t rev_h(uint32_t x, int bits) {
    uint32_t r = 0;
    for (int i = 0; i < bits; ++i) r |= ((x >> i) & 1u) << (bits - 1 - i);
    return r;
}
}  // namespace

// Variant bit 0 selects the shape: CTAs of up to 512 threads (one limb of N <= 2^14 per CTA),
// or CTAs of half the size in clusters twice as large (two CTAs share an SM). variant >> 1
// selects how a cluster shares a limb: 0 = peers read each other's buffers (pull, one
// buffer, three barriers per row), 1 = peers store into a receive buffer (push, two
// buffers, two barriers), 2 = forward transforms read all quarters themselves (split, no
// data exchange, one barrier; inverse transforms then use pull), 3 = no cluster: two passes
// through an L2-resident scratch (ntt_u32_l2.cu). Bit 3 stages each thread's last-round
// twiddles in shared memory (pull and split exchange, and single-CTA shapes; rows then run
// in contiguous ranges per cluster). Bit 4 caps the kernel at 64 registers per thread so
// that twice as many CTAs share an SM (pull and split exchange, and single-CTA shapes,
// without bit 3). The forward and the inverse transform of a ring degree each have their
// own variant.
int ntt_variant_exchange(int variant) { return (variant >> 1) & 3; }
bool ntt_variant_tws(int variant) { return ((variant >> 3) & 1) != 0; }
bool ntt_variant_occ2(int variant) { return ((variant >> 4) & 1) != 0; }

bool ntt_variant_shape(uint32_t logN, int variant, int* log_t, int* log_c) {
    if (logN < FHE_LOGN_MIN || logN > FHE_LOGN_MAX || variant < 0 || variant >= kNttVariants) return false;
    int lt = logN >= 14 ? 9 : (int)logN - 5;
    if ((variant & 1) == 1) {
        if (logN <= 11) return false;
        lt -= 1;
    }
    *log_t = lt;
    *log_c = (int)logN - 5 - lt;
    if (*log_c == 0 && ntt_variant_exchange(variant) != 0) return false;  // no cluster to share
    if (ntt_variant_exchange(variant) == 3 && logN < 15) return false;    // two-pass kernels: N >= 2^15
    if (ntt_variant_tws(variant) && (ntt_variant_exchange(variant) & 1)) return false;  // push / two-pass
    if (ntt_variant_occ2(variant) && (ntt_variant_tws(variant) || (ntt_variant_exchange(variant) & 1)))
        return false;  // shared memory of twice the CTAs does not fit; two-pass kernels have one shape
    return true;
}

int build_ntt_tables(fhe_ctx* ctx, uint32_t logN) {
    const int nmod = (int)ctx->mods.size();
    const uint32_t N = 1u << logN;
    std::vector<uint2> fwd((size_t)nmod * N), inv((size_t)nmod * N);
    std::vector<uint2> ninv(nmod), ninv_w1(nmod);
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
        uint32_t ni = invmod_h(N % q, q);
        ninv[m] = make_uint2(ni, shoup_h(ni, q));
        const uint32_t niw = mulmod_h(ni, inv[(size_t)m * N + 1].x, q);
        ninv_w1[m] = make_uint2(niw, shoup_h(niw, q));
    }
    NttTables& t = ctx->ntt[logN];
    int rc;
    // last-round tables per shape: thread tid of CTA c, entry (2^k - 1 + b) holds
    // tw[2^k * ((C + c) * T + rev(tid)) + b]
    for (int v = 0; v < 2; ++v) {
        int log_t, log_c;
        if (!ntt_variant_shape(logN, v, &log_t, &log_c)) continue;
        const int T = 1 << log_t, C = 1 << log_c;
        std::vector<uint2> fwdC((size_t)nmod * C * 31 * T), invC((size_t)nmod * C * 31 * T);
        for (int m = 0; m < nmod; ++m)
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
        if ((rc = dev_upload(ctx, &t.fwdC[v], fwdC))) return rc;
        if ((rc = dev_upload(ctx, &t.invC[v], invC))) return rc;
    }
    if ((rc = dev_upload(ctx, &t.fwd, fwd))) return rc;
    if ((rc = dev_upload(ctx, &t.inv, inv))) return rc;
    if ((rc = dev_upload(ctx, &t.ninv, ninv))) return rc;
    if ((rc = dev_upload(ctx, &t.ninv_w1, ninv_w1))) return rc;
    // two-pass decimation-in-time forward: twists and C-th roots of unity per shape
    for (int v = 0; v < 2 && logN >= 15; ++v) {
        int log_t, log_c;
        if (!ntt_variant_shape(logN, v, &log_t, &log_c)) continue;
        const uint32_t C = 1u << log_c, NC = N >> log_c;
        std::vector<uint2> twist((size_t)nmod * (C - 1) * NC), omega((size_t)nmod * (C / 2));
        for (int m = 0; m < nmod; ++m) {
            const uint32_t q = ctx->mods[m];
            const uint32_t psi = root_2n(q, logN);
            const uint32_t psi2 = mulmod_h(psi, psi, q);
            uint32_t base = psi;  // psi^(2k'+1)
            for (uint32_t k = 0; k < NC; ++k) {
                uint32_t w = base;
                for (uint32_t j = 1; j < C; ++j) {
                    twist[((size_t)m * (C - 1) + (j - 1)) * NC + k] = make_uint2(w, shoup_h(w, q));
                    w = mulmod_h(w, base, q);
                }
                base = mulmod_h(base, psi2, q);
            }
            const uint32_t om = powmod_h(psi, 2ull * NC, q);
            uint32_t w = 1;
            for (uint32_t j = 0; j < C / 2; ++j) {
                omega[(size_t)m * (C / 2) + j] = make_uint2(w, shoup_h(w, q));
                w = mulmod_h(w, om, q);
            }
        }
        if ((rc = dev_upload(ctx, &t.dit_twist[v], twist))) return rc;
        if ((rc = dev_upload(ctx, &t.dit_omega[v], omega))) return rc;
    }
    return FHE_OK;
}

namespace {
int ntt_u32_dispatch(const fhe_ctx* ctx, uint32_t logN, bool inverse, uint32_t* d, long long rows, int batch,
                     const LimbMap& map, const RowRef* rowtab, cudaStream_t stream, NttScratch scr);
}

int ntt_u32(const fhe_ctx* ctx, uint32_t logN, bool inverse, uint32_t* d, int n_limbs, int batch,
            const LimbMap& map, cudaStream_t stream, NttScratch scr) {
    return ntt_u32_dispatch(ctx, logN, inverse, d, (long long)n_limbs * batch, batch, map, nullptr, stream, scr);
}

int ntt_u32_rows(const fhe_ctx* ctx, uint32_t logN, bool inverse, const RowRef* d_rows, int nrows,
                 cudaStream_t stream, NttScratch scr) {
    LimbMap unused;
    memset(&unused, 0, sizeof(unused));
    return ntt_u32_dispatch(ctx, logN, inverse, nullptr, nrows, 1, unused, d_rows, stream, scr);
}

namespace {
int ntt_u32_dispatch(const fhe_ctx* ctx, uint32_t logN, bool inverse, uint32_t* d, long long rows_ll, int batch,
                     const LimbMap& map, const RowRef* rowtab, cudaStream_t stream, NttScratch scr) {
    const NttTables& t = ctx->ntt[logN];
    if (!t.fwd) return set_error(FHE_EINVAL, "no NTT tables for this logN");
    if (rows_ll == 0) return FHE_OK;
    if (rows_ll > (1LL << 30)) return set_error(FHE_EINVAL, "too many rows");
    const int rows = (int)rows_ll;
    const int v = ctx->plain_variant[inverse ? 1 : 0][logN];
    int log_t, log_c;
    if (!ntt_variant_shape(logN, v, &log_t, &log_c)) return set_error(FHE_EINVAL, "logN out of range");
    if (log_c >= 2)
        return ntt_u32_launch_wide(ctx, t, logN, log_t, log_c, v, inverse, d, rows, batch, map, rowtab, stream, scr);
    FHE_NTT_CASE(5, 0)
    FHE_NTT_CASE(6, 0)
    FHE_NTT_CASE(7, 0)
    FHE_NTT_CASE(8, 0)
    FHE_NTT_CASE(9, 0)
    FHE_NTT_CASE(9, 1)
    FHE_NTT_CASE(6, 1)
    FHE_NTT_CASE(7, 1)
    FHE_NTT_CASE(8, 1)
    return set_error(FHE_EINVAL, "no kernel for this NTT shape");
}
}  // namespace

}  // namespace fhe

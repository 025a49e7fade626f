// Context creation, moduli validation, host-side table generation and the NTT entry points.
#include <string.h>

#include <algorithm>
#include <string>

#include "common.cuh"

namespace fhe {

namespace {
thread_local int g_last_code = FHE_OK;
thread_local std::string g_last_msg;
}  // namespace

int set_error(int code, const std::string& msg) {
    g_last_code = code;
    g_last_msg = msg;
    return code;
}

int cuda_error(cudaError_t e, const char* where) {
    return set_error(FHE_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

uint32_t powmod_h(uint32_t b, uint64_t e, uint32_t q) {
    uint64_t r = 1 % q, x = b % q;
    while (e) {
        if (e & 1) r = r * x % q;
        x = x * x % q;
        e >>= 1;
    }
    return (uint32_t)r;
}

// Deterministic Miller-Rabin with bases 2, 3, 5, 7 (exact below 3,215,031,751).
bool is_prime_u32(uint32_t n) {
    if (n < 2) return false;
    const uint32_t small[] = {2, 3, 5, 7, 11, 13};
    for (uint32_t p : small)
        if (n % p == 0) return n == p;
    uint32_t d = n - 1;
    int s = 0;
    while ((d & 1) == 0) {
        d >>= 1;
        ++s;
    }
    const uint32_t bases[] = {2, 3, 5, 7};
    for (uint32_t a : bases) {
        uint64_t x = powmod_h(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int r = 1; r < s; ++r) {
            x = x * x % n;
            if (x == n - 1) {
                comp = false;
                break;
            }
        }
        if (comp) return false;
    }
    return true;
}

// psi = x^((q-1)/2N) for the smallest quadratic non-residue x: psi^N = -1, order 2N.
uint32_t root_2n(uint32_t q, uint32_t logN) {
    uint32_t x = 2;
    while (powmod_h(x, (q - 1) / 2, q) != q - 1) ++x;
    return powmod_h(x, (q - 1) >> (logN + 1), q);
}

LimbMap contiguous_map(const fhe_ctx* ctx, int first, int n) {
    LimbMap m;
    memset(&m, 0, sizeof(m));
    for (int l = 0; l < n; ++l) {
        m.mod[l] = (uint8_t)(first + l);
        m.q[l] = ctx->mods[first + l];
    }
    return m;
}

int ntt_any(const fhe_ctx* ctx, int path, uint32_t logN, bool inverse, uint32_t* d, int n_limbs,
            int batch, const LimbMap& map, cudaStream_t stream, NttScratch scr) {
    if (path == FHE_NTT_DEFAULT) path = ctx->ntt_variant[inverse ? 1 : 0][logN] >= kNttVariants ? FHE_NTT_TC : FHE_NTT_U32;
    if (path == FHE_NTT_TC) return ntt_tc(ctx, logN, inverse, d, n_limbs, batch, map, stream, scr);
    return ntt_u32(ctx, logN, inverse, d, n_limbs, batch, map, stream, scr);
}

size_t ntt_region_bytes(uint32_t logN, size_t rows) {
    // from 2^15 the two-pass kernels; from 2^12 to 2^14 the one-CTA-per-row shape of the same
    // kernels that carries the fused HMULT tail and ModDown combine
    if (logN < 12 || rows == 0) return 0;
    const size_t b = rows * (((size_t)4 << logN) + 4);  // residues and a completion counter per row
    return b < kNttTempBytes ? b : kNttTempBytes;
}

size_t op_region_bytes(const fhe_ctx* ctx, uint32_t logN, size_t rows) {
    size_t b = ntt_region_bytes(logN, rows);
    const bool tc = ctx->ntt_variant[0][logN] >= kNttVariants || ctx->ntt_variant[1][logN] >= kNttVariants;
    if (tc && rows > 0) {
        // the tensor-core path's digit planes: 8 bytes per residue of a chunk of rows
        const size_t tc = std::min(rows * ((size_t)8 << logN), kTcPlaneBytes);
        b = std::max(b, tc);
    }
    return b;
}

static int build_conv(fhe_ctx* ctx, const std::vector<int>& src, ConvTable* out) {
    const int nmod = (int)ctx->mods.size();
    const int ns = (int)src.size();
    std::vector<uint2> hat_inv(ns);
    std::vector<uint32_t> hat_mod((size_t)ns * nmod);
    for (int i = 0; i < ns; ++i) {
        const uint32_t bi = ctx->mods[src[i]];
        uint32_t prod_i = 1;  // (B / b_i) mod b_i
        for (int k = 0; k < ns; ++k)
            if (k != i) prod_i = mulmod_h(prod_i, ctx->mods[src[k]] % bi, bi);
        uint32_t inv = invmod_h(prod_i, bi);
        hat_inv[i] = make_uint2(inv, shoup_h(inv, bi));
        for (int t = 0; t < nmod; ++t) {
            const uint32_t mt = ctx->mods[t];
            uint32_t pr = 1;  // (B / b_i) mod t
            for (int k = 0; k < ns; ++k)
                if (k != i) pr = mulmod_h(pr, ctx->mods[src[k]] % mt, mt);
            hat_mod[(size_t)i * nmod + t] = pr;
        }
    }
    // tensor-core Conv operand: for destination modulus t and digit k, row K' = 4 i + j holds
    // the k-th balanced base-256 digit of [(B / b_i) 256^j]_t as fp16 (64 entries, zero padded)
    std::vector<uint16_t> bdig((size_t)nmod * 4 * kConvKPad, 0);
    for (int t = 0; t < nmod; ++t) {
        const uint32_t mt = ctx->mods[t];
        for (int i = 0; i < ns; ++i)
            for (int j = 0; j < 4; ++j) {
                const uint32_t w = mulmod_h(hat_mod[(size_t)i * nmod + t], powmod_h(256 % mt, j, mt), mt);
                const uint32_t y = w + 0x80808080u;  // w < 2^30: bytes of y minus 128 are the digits
                for (int k = 0; k < 4; ++k)
                    bdig[((size_t)t * 4 + k) * kConvKPad + 4 * i + j] =
                        f16_bits_of_small_int((int)((y >> (8 * k)) & 0xFF) - 128);
            }
    }
    out->nsrc = ns;
    out->hat_inv_h = hat_inv;
    int rc;
    if ((rc = dev_upload(ctx, &out->hat_inv, hat_inv))) return rc;
    if ((rc = dev_upload(ctx, &out->hat_mod, hat_mod))) return rc;
    if ((rc = dev_upload(ctx, &out->bdig, bdig))) return rc;
    return FHE_OK;
}

static int build_ckks_tables(fhe_ctx* ctx) {
    const int nq = ctx->nq, np = ctx->np, a = ctx->alpha;
    int rc;
    ctx->dnum = (nq + a - 1) / a;
    ctx->modup.assign(ctx->dnum, {});
    for (int j = 0; j < ctx->dnum; ++j) {
        const int lo = j * a, hi = std::min(nq, (j + 1) * a);
        ctx->modup[j].resize(hi - lo);
        for (int e = lo + 1; e <= hi; ++e) {
            std::vector<int> src;
            for (int i = lo; i < e; ++i) src.push_back(i);
            if ((rc = build_conv(ctx, src, &ctx->modup[j][e - lo - 1]))) return rc;
        }
    }
    std::vector<int> psrc;
    for (int k = 0; k < np; ++k) psrc.push_back(nq + k);
    if ((rc = build_conv(ctx, psrc, &ctx->moddown))) return rc;
    std::vector<uint2> pinv(nq), qlinv((size_t)nq * nq);
    for (int i = 0; i < nq; ++i) {
        const uint32_t qi = ctx->mods[i];
        uint32_t pm = 1;
        for (int k = 0; k < np; ++k) pm = mulmod_h(pm, ctx->mods[nq + k] % qi, qi);
        uint32_t inv = invmod_h(pm, qi);
        pinv[i] = make_uint2(inv, shoup_h(inv, qi));
    }
    for (int l = 0; l < nq; ++l)
        for (int i = 0; i < nq; ++i) {
            const uint32_t qi = ctx->mods[i];
            uint32_t inv = (i == l) ? 0 : invmod_h(ctx->mods[l] % qi, qi);
            qlinv[(size_t)l * nq + i] = make_uint2(inv, shoup_h(inv, qi));
        }
    ctx->p_inv_h = pinv;
    if ((rc = dev_upload(ctx, &ctx->p_inv, pinv))) return rc;
    if ((rc = dev_upload(ctx, &ctx->ql_inv, qlinv))) return rc;
    return FHE_OK;
}

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

static int check_ntt_args(const fhe_ctx* ctx, int path, uint32_t logN, const uint32_t* d,
                          int first_limb, int n_limbs, int batch) {
    FHE_CHECK(ctx != nullptr, "ctx is NULL");
    FHE_CHECK(logN >= FHE_LOGN_MIN && logN <= ctx->logN_max, "logN out of [10, logN_max]");
    FHE_CHECK(path == FHE_NTT_DEFAULT || path == FHE_NTT_U32 || path == FHE_NTT_TC, "bad path");
    FHE_CHECK(n_limbs >= 1 && first_limb >= 0 && first_limb + n_limbs <= (int)ctx->mods.size(),
              "limb range outside the context's moduli");
    FHE_CHECK(batch >= 0, "batch < 0");
    FHE_CHECK(batch == 0 || (d != nullptr && aligned16(d)), "data pointer NULL or not 16-byte aligned");
    return FHE_OK;
}

namespace {
// A choice id the library accepts at logN: a plain-path variant with a kernel shape there, or
// one of the two tensor-core tile widths.
bool choice_valid(uint32_t logN, int v) {
    int lt, lc;
    return v == kTcVariant64 || v == kTcVariant32 || ntt_variant_shape(logN, v, &lt, &lc);
}
void set_choice(fhe_ctx* ctx, uint32_t logN, int dir, int v) {
    ctx->ntt_variant[dir][logN] = v;
    if (v < kNttVariants)
        ctx->plain_variant[dir][logN] = v;
    else
        ctx->tc_nt[dir][logN] = v == kTcVariant64 ? 64 : 32;
}
}  // namespace

}  // namespace fhe

using namespace fhe;

extern "C" {

int fhe_last_error(char* buf, size_t n) {
    if (buf && n) {
        size_t k = std::min(n - 1, g_last_msg.size());
        memcpy(buf, g_last_msg.data(), k);
        buf[k] = 0;
    }
    return g_last_code;
}

int fhe_gen_primes(uint32_t logN_max, int bits, int count, uint32_t* out) {
    FHE_CHECK(out != nullptr || count == 0, "out is NULL");
    FHE_CHECK(logN_max >= FHE_LOGN_MIN && logN_max <= FHE_LOGN_MAX, "logN_max out of [10, 16]");
    FHE_CHECK(bits >= 20 && bits <= 31, "bits out of [20, 31]");
    FHE_CHECK(count >= 0, "count < 0");
    const uint64_t step = 1ull << (logN_max + 1);
    uint64_t qv = (((1ull << bits) - 1) / step) * step + 1;
    int k = 0;
    while (k < count) {
        if (qv <= (1ull << (bits - 1))) return set_error(FHE_EINVAL, "not enough primes");
        if (is_prime_u32((uint32_t)qv)) out[k++] = (uint32_t)qv;
        qv -= step;
    }
    return FHE_OK;
}

int fhe_ctx_create(uint32_t logN_max, const uint32_t* q, int nq, const uint32_t* p, int np,
                   int alpha, int default_path, fhe_ctx** out) {
    FHE_CHECK(out != nullptr, "out is NULL");
    *out = nullptr;
    FHE_CHECK(logN_max >= FHE_LOGN_MIN && logN_max <= FHE_LOGN_MAX, "logN_max out of [10, 16]");
    FHE_CHECK(q != nullptr && nq >= 1, "need at least one ciphertext prime");
    FHE_CHECK(np >= 0 && np <= 15 && (np == 0 || p != nullptr), "np out of [0, 15]");
    FHE_CHECK(nq + np <= FHE_MAX_MODULI, "more than 64 moduli");
    FHE_CHECK(alpha >= 1 && alpha <= 15, "alpha out of [1, 15]");
    FHE_CHECK(default_path == FHE_NTT_U32 || default_path == FHE_NTT_TC, "bad default_path");
    std::vector<uint32_t> mods(q, q + nq);
    mods.insert(mods.end(), p, p + np);
    for (size_t i = 0; i < mods.size(); ++i) {
        const uint32_t m = mods[i];
        FHE_CHECK(m < (1u << 30), "modulus >= 2^30");
        FHE_CHECK(((uint64_t)m - 1) % (1ull << (logN_max + 1)) == 0, "modulus != 1 mod 2N");
        FHE_CHECK(is_prime_u32(m), "modulus is not prime");
        for (size_t k = 0; k < i; ++k) FHE_CHECK(mods[k] != m, "moduli not distinct");
    }
    if (np > 0) {
        // P > every slice product Q_j (Sec. II-B); compare in log2 with a safety margin of
        // one bit and exactly when close.
        double logP = 0;
        for (int k = 0; k < np; ++k) logP += log2((double)p[k]);
        for (int j = 0; j * alpha < nq; ++j) {
            double lq = 0;
            for (int i = j * alpha; i < std::min(nq, (j + 1) * alpha); ++i) lq += log2((double)q[i]);
            FHE_CHECK(logP > lq + 1e-9, "special-prime product P is not larger than a slice product Q_j");
        }
    }
    fhe_ctx* ctx = new fhe_ctx();
    ctx->logN_max = logN_max;
    ctx->nq = nq;
    ctx->np = np;
    ctx->alpha = alpha;
    ctx->default_path = default_path;
    ctx->mods = mods;
    // default plain-path variants (forward, inverse): the fastest measured on GB300 for 44
    // limbs x (2^22 / N) polynomials; fhe_autotune_ntt re-measures them for the caller's batch
    static const int kDefaultVariant[3][2] = {
        {16, 8},  // 2^14: single CTA at 64 registers / single CTA with staged twiddles
        {7, 7},   // 2^15: two-pass, 256 threads, both directions
        {6, 6},   // 2^16: two-pass (decimation-in-time forward), 512 threads, both directions
    };
    for (int l = 14; l <= 16; ++l) {
        ctx->plain_variant[0][l] = kDefaultVariant[l - 14][0];
        ctx->plain_variant[1][l] = kDefaultVariant[l - 14][1];
    }
    // FHE_NTT_DEFAULT starts on the context's default path; fhe_ntt_set_variant and
    // fhe_autotune_ntt may move a ring degree and direction to the other one
    for (int dir = 0; dir < 2; ++dir)
        for (int l = 0; l <= FHE_LOGN_MAX; ++l) {
            ctx->tc_nt[dir][l] = 64;
            ctx->ntt_variant[dir][l] = default_path == FHE_NTT_TC ? kTcVariant64 : ctx->plain_variant[dir][l];
        }
    int rc = FHE_OK;
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device);
    if (e != cudaSuccess) rc = cuda_error(e, "cudaGetDevice");
    if (rc == FHE_OK) {
        rc = dev_alloc(ctx, &ctx->d_status, 1);
        if (rc == FHE_OK) {
            cudaError_t ce = cudaMemset(ctx->d_status, 0, sizeof(int));
            if (ce != cudaSuccess) rc = cuda_error(ce, "cudaMemset");
        }
    }
    if (rc == FHE_OK) rc = dev_upload(ctx, &ctx->d_mods, ctx->mods);
    if (rc == FHE_OK && logN_max >= 15) rc = dev_alloc(ctx, &ctx->ntt_temp, kNttTempBytes / 4);
    for (uint32_t lg = FHE_LOGN_MIN; rc == FHE_OK && lg <= logN_max; ++lg) rc = build_ntt_tables(ctx, lg);
    if (rc == FHE_OK && np > 0) rc = build_ckks_tables(ctx);
    if (rc == FHE_OK && default_path == FHE_NTT_TC) {
        for (uint32_t lg = FHE_LOGN_MIN; rc == FHE_OK && lg <= logN_max; ++lg) rc = build_tc_tables(ctx, lg);
    }
    if (rc != FHE_OK) {
        fhe_ctx_destroy(ctx);
        return rc;
    }
    *out = ctx;
    return FHE_OK;
}

int fhe_ctx_destroy(fhe_ctx* ctx) {
    if (!ctx) return FHE_OK;
    for (void* v : ctx->allocations) cudaFree(v);
    delete ctx;
    return FHE_OK;
}

int fhe_ntt_fwd(const fhe_ctx* ctx, int path, uint32_t logN, uint32_t* d, int first_limb,
                int n_limbs, int batch, void* stream) {
    int rc = check_ntt_args(ctx, path, logN, d, first_limb, n_limbs, batch);
    if (rc) return rc;
    if (batch == 0) return FHE_OK;
    return ntt_any(ctx, path, logN, false, d, n_limbs, batch, contiguous_map(ctx, first_limb, n_limbs),
                   (cudaStream_t)stream);
}

int fhe_ntt_inv(const fhe_ctx* ctx, int path, uint32_t logN, uint32_t* d, int first_limb,
                int n_limbs, int batch, void* stream) {
    int rc = check_ntt_args(ctx, path, logN, d, first_limb, n_limbs, batch);
    if (rc) return rc;
    if (batch == 0) return FHE_OK;
    return ntt_any(ctx, path, logN, true, d, n_limbs, batch, contiguous_map(ctx, first_limb, n_limbs),
                   (cudaStream_t)stream);
}

int fhe_device_status(const fhe_ctx* ctx, int clear) {
    FHE_CHECK(ctx != nullptr, "ctx is NULL");
    int v = 0;
    FHE_CUDA_TRY(cudaMemcpy(&v, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (clear && v) FHE_CUDA_TRY(cudaMemset(ctx->d_status, 0, sizeof(int)));
    if (v == FHE_ETIMEOUT) return set_error(FHE_ETIMEOUT, "a bounded device-side wait expired");
    if (v) return set_error(v, "device reported an error");
    return FHE_OK;
}

int fhe_ntt_variant_count(const fhe_ctx* ctx, uint32_t logN) {
    if (!ctx || logN < FHE_LOGN_MIN || logN > ctx->logN_max) return -1;
    return kNttChoices;
}


int fhe_ntt_get_variant(const fhe_ctx* ctx, uint32_t logN, int inverse) {
    if (!ctx || logN < FHE_LOGN_MIN || logN > ctx->logN_max) return -1;
    return ctx->ntt_variant[inverse ? 1 : 0][logN];
}

int fhe_ntt_set_variant(fhe_ctx* ctx, uint32_t logN, int fwd_variant, int inv_variant) {
    FHE_CHECK(ctx != nullptr, "ctx is NULL");
    FHE_CHECK(logN >= FHE_LOGN_MIN && logN <= ctx->logN_max, "logN out of [10, logN_max]");
    FHE_CHECK(choice_valid(logN, fwd_variant), "no such forward NTT variant for this logN");
    FHE_CHECK(choice_valid(logN, inv_variant), "no such inverse NTT variant for this logN");
    set_choice(ctx, logN, 0, fwd_variant);
    set_choice(ctx, logN, 1, inv_variant);
    return FHE_OK;
}

int fhe_conv_set_path(fhe_ctx* ctx, int path) {
    FHE_CHECK(ctx != nullptr, "ctx is NULL");
    FHE_CHECK(path == FHE_CONV_CUDA || path == FHE_CONV_TC, "path must be FHE_CONV_CUDA or FHE_CONV_TC");
    ctx->conv_path = path;
    return FHE_OK;
}

int fhe_conv_get_path(const fhe_ctx* ctx) { return ctx ? ctx->conv_path : -1; }

int fhe_autotune_ntt(fhe_ctx* ctx, uint32_t logN, uint32_t* d, int n_limbs, int batch, int reps,
                     float* ms_out, void* stream) {
    int rc = check_ntt_args(ctx, FHE_NTT_U32, logN, d, 0, n_limbs, batch);
    if (rc) return rc;
    FHE_CHECK(batch >= 1 && reps >= 1, "batch and reps must be >= 1");
    cudaStream_t st = (cudaStream_t)stream;
    const LimbMap map = contiguous_map(ctx, 0, n_limbs);
    int keep[3][2];
    for (int dir = 0; dir < 2; ++dir) {
        keep[0][dir] = ctx->ntt_variant[dir][logN];
        keep[1][dir] = ctx->plain_variant[dir][logN];
        keep[2][dir] = ctx->tc_nt[dir][logN];
    }
    // per direction: the fastest choice overall, the fastest plain-path variant and the
    // fastest tensor-core tile width (the latter two serve explicit FHE_NTT_U32 / _TC calls)
    int best[2] = {keep[0][0], keep[0][1]}, best_plain[2] = {keep[1][0], keep[1][1]};
    int best_tc[2] = {keep[2][0] == 32 ? kTcVariant32 : kTcVariant64, keep[2][1] == 32 ? kTcVariant32 : kTcVariant64};
    float best_ms[2] = {-1.0f, -1.0f}, best_plain_ms[2] = {-1.0f, -1.0f}, best_tc_ms[2] = {-1.0f, -1.0f};
    const int count = fhe_ntt_variant_count(ctx, logN);
    cudaEvent_t ev[3];
    for (int i = 0; i < 3; ++i) FHE_CUDA_TRY(cudaEventCreate(&ev[i]));
    for (int v = 0; v < count && rc == FHE_OK; ++v) {
        if (!choice_valid(logN, v)) {
            if (ms_out) ms_out[v] = ms_out[count + v] = -1.0f;
            continue;
        }
        set_choice(ctx, logN, 0, v);
        set_choice(ctx, logN, 1, v);
        float sum[2] = {0.0f, 0.0f};
        // one untimed round trip, then `reps` timed ones (forward and inverse timed apart)
        for (int r = 0; r <= reps && rc == FHE_OK; ++r) {
            cudaEventRecord(ev[0], st);
            rc = ntt_any(ctx, FHE_NTT_DEFAULT, logN, false, d, n_limbs, batch, map, st);
            cudaEventRecord(ev[1], st);
            if (rc == FHE_OK) rc = ntt_any(ctx, FHE_NTT_DEFAULT, logN, true, d, n_limbs, batch, map, st);
            cudaEventRecord(ev[2], st);
            cudaError_t ce = cudaEventSynchronize(ev[2]);
            if (rc == FHE_OK && ce != cudaSuccess) rc = cuda_error(ce, "cudaEventSynchronize");
            if (rc != FHE_OK || r == 0) continue;
            float f = 0, i = 0;
            cudaEventElapsedTime(&f, ev[0], ev[1]);
            cudaEventElapsedTime(&i, ev[1], ev[2]);
            sum[0] += f;
            sum[1] += i;
        }
        if (rc != FHE_OK) break;
        for (int dir = 0; dir < 2; ++dir) {
            const float ms = sum[dir] / reps;
            if (ms_out) ms_out[dir * count + v] = ms;
            if (best_ms[dir] < 0 || ms < best_ms[dir]) {
                best_ms[dir] = ms;
                best[dir] = v;
            }
            float& bk = v < kNttVariants ? best_plain_ms[dir] : best_tc_ms[dir];
            if (bk < 0 || ms < bk) {
                bk = ms;
                (v < kNttVariants ? best_plain : best_tc)[dir] = v;
            }
        }
    }
    for (int i = 0; i < 3; ++i) cudaEventDestroy(ev[i]);
    for (int dir = 0; dir < 2; ++dir) {
        if (rc == FHE_OK) {
            set_choice(ctx, logN, dir, best_plain[dir]);
            set_choice(ctx, logN, dir, best_tc[dir]);
            set_choice(ctx, logN, dir, best[dir]);
        } else {
            ctx->ntt_variant[dir][logN] = keep[0][dir];
            ctx->plain_variant[dir][logN] = keep[1][dir];
            ctx->tc_nt[dir][logN] = keep[2][dir];
        }
    }
    return rc;
}

}  // extern "C"

// Internal declarations shared by the libfhe translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/fhe.h"

namespace fhe {

// ---------------------------------------------------------------- errors

int set_error(int code, const std::string& msg);
int cuda_error(cudaError_t e, const char* where);

#define FHE_CUDA_TRY(expr)                                  \
    do {                                                    \
        cudaError_t _e = (expr);                            \
        if (_e != cudaSuccess) return cuda_error(_e, #expr); \
    } while (0)

#define FHE_CHECK(cond, msg)                                \
    do {                                                    \
        if (!(cond)) return set_error(FHE_EINVAL, (msg));   \
    } while (0)

// ---------------------------------------------------------------- host modular arithmetic

static inline uint32_t mulmod_h(uint32_t a, uint32_t b, uint32_t q) {
    return (uint32_t)((uint64_t)a * b % q);
}
uint32_t powmod_h(uint32_t b, uint64_t e, uint32_t q);
static inline uint32_t invmod_h(uint32_t a, uint32_t q) { return powmod_h(a, (uint64_t)q - 2, q); }
// Shoup's precomputed quotient floor(w * 2^32 / q) for multiplications by the constant w < q.
static inline uint32_t shoup_h(uint32_t w, uint32_t q) {
    return (uint32_t)(((uint64_t)w << 32) / q);
}
bool is_prime_u32(uint32_t n);
uint32_t root_2n(uint32_t q, uint32_t logN);  // primitive 2N-th root from the smallest non-residue

// ---------------------------------------------------------------- context

// Plain-path kernel shapes per ring degree: threads per CTA T = 2^log_t and CTAs per
// cluster C = 2^log_c with 32 * T * C = N (see ntt_u32.cu).
constexpr int kNttVariants = 32;
// Choice ids beyond the plain-path variants (fhe_ntt_set_variant, fhe_autotune_ntt): the
// tensor-core path with output tiles of 64 or of 32 columns (NT).
constexpr int kTcVariant64 = FHE_NTT_VARIANT_TC64, kTcVariant32 = FHE_NTT_VARIANT_TC32;
static_assert(kTcVariant64 == kNttVariants && kTcVariant32 == kNttVariants + 1, "choice ids follow the plain variants");
constexpr int kNttChoices = kNttVariants + 2;
#ifndef FHE_NTT_CHUNK_MIB
#define FHE_NTT_CHUNK_MIB 1024
#endif
// scratch of the two-pass NTT, one chunk of rows at a time. Large chunks pay: each chunk is
// two launches, and on GB300 a 1 GiB chunk (the whole 44 x 64 batch at 2^16 in one chunk)
// measured 1.68 ms per forward + inverse against 1.97 ms with 64 MiB chunks; the scratch
// spills from L2 either way.
constexpr size_t kNttTempBytes = (size_t)FHE_NTT_CHUNK_MIB << 20;
bool ntt_variant_shape(uint32_t logN, int variant, int* log_t, int* log_c);
int ntt_variant_exchange(int variant);
bool ntt_variant_tws(int variant);
bool ntt_variant_occ2(int variant);

// Plain-path NTT tables for one ring degree N = 2^logN (device memory).
struct NttTables {
    uint2* fwd = nullptr;   // [nmod][N]  (psi^bitrev(i), shoup)
    uint2* inv = nullptr;   // [nmod][N]  (psi^-bitrev(i), shoup)
    uint2* fwdC[2] = {};  // per shape: [nmod][C][31][T] last-round twiddles, per-thread order
    uint2* invC[2] = {};
    uint2* ninv = nullptr;  // [nmod] (N^-1 mod q, shoup)
    uint2* ninv_w1 = nullptr;  // [nmod] (N^-1 inv[1] mod q, shoup): the two-pass inverse's last stage
    // decimation-in-time two-pass forward (N >= 2^15), per shape with C = N / NC sub-NTTs of
    // NC points: twist[nmod][C-1][NC] = psi^((2k'+1) j) for j = 1..C-1, and omega[nmod][C/2] =
    // (psi^(2 NC))^m, the C-th roots of unity of the C-point DFT (all with Shoup quotients)
    uint2* dit_twist[2] = {};
    uint2* dit_omega[2] = {};
};

// Tensor-core path tables for one ring degree (device memory); see ntt_tc.cu. Built on the
// first tensor-core call at that degree.
struct TcTables {
    uint16_t* mat[4] = {};     // digit planes (fp16) of W1 fwd, W3 fwd, W3 inv, W1 inv: [nmod][4][cols][4K]
    uint2* tw_fwd = nullptr;   // [nmod][N1][N2] (psi^((2k1+1) n2), shoup)
    uint2* tw_inv = nullptr;   // [nmod][N2][N1] (N^-1 psi^(-(2k1+1) n2), shoup)
    CUtensorMap map_b[4];      // TMA maps over mat[kind], box of min(64, cols) rows (NT = 64 tiles)
    CUtensorMap map_b32[4];    // the same with a box of 32 rows (NT = 32 tiles)
    CUtensorMap map_a[2];      // TMA maps over the plane buffer, inner extent 4*N1 / 4*N2
    int n1 = 0, n2 = 0;
    bool built = false;
};

// Basis-conversion constants (Conv of Sec. IV-A) for one source basis.
// Reduction length of the tensor-core Conv operand rows: 4 digits x at most 15 source limbs,
// padded to the 64 fp16 of one 128-byte shared-memory row.
constexpr int kConvKPad = 64;

struct ConvTable {
    // src: hat_inv[i] = [(B/b_i)^-1]_{b_i} with Shoup quotient; dst: hat_mod[i][t] = [B/b_i]_t
    uint2* hat_inv = nullptr;   // [nsrc]
    uint32_t* hat_mod = nullptr; // [nsrc][nmod]  indexed by destination modulus index
    uint16_t* bdig = nullptr;   // [nmod][4][kConvKPad] fp16 digits of [hat_mod[i][t] 256^j]_t (tensor-core Conv)
    std::vector<uint2> hat_inv_h; // host copy of hat_inv (passed to kernels by value)
    int nsrc = 0;
};

}  // namespace fhe

struct fhe_ctx {
    uint32_t logN_max = 0;
    int nq = 0, np = 0, alpha = 0, default_path = FHE_NTT_U32;
    int dnum = 0;
    std::vector<uint32_t> mods;  // q_0.., p_0..
    fhe::NttTables ntt[FHE_LOGN_MAX + 1];
    // per direction (0 fwd, 1 inv) and logN: the choice FHE_NTT_DEFAULT runs (a plain-path
    // variant id, or kTcVariant64 / kTcVariant32), the plain-path variant of FHE_NTT_U32 calls
    // and the tensor-core tile width of FHE_NTT_TC calls
    int ntt_variant[2][FHE_LOGN_MAX + 1] = {};
    int plain_variant[2][FHE_LOGN_MAX + 1] = {};
    int tc_nt[2][FHE_LOGN_MAX + 1] = {};
    int conv_path = FHE_CONV_CUDA;              // basis-conversion kernel (fhe_conv_set_path)
    fhe::TcTables tc[FHE_LOGN_MAX + 1];
    // conv tables: modup[j][e] for slice j ending (exclusive) at limb e; moddown from P
    std::vector<std::vector<fhe::ConvTable>> modup;
    fhe::ConvTable moddown;
    uint2* p_inv = nullptr;        // [nq]  ([P^-1]_{q_i}, shoup)
    std::vector<uint2> p_inv_h;    // host copy of p_inv
    uint2* ql_inv = nullptr;       // [nq][nq]  row l: ([q_l^-1]_{q_i}, shoup)
    std::vector<void*> allocations;
    int device = 0;
    int num_sms = 0;
    int* d_status = nullptr;  // device error word written by kernels (FHE_ETIMEOUT, ...)
    void* tc_planes = nullptr;  // tensor-core digit planes of fhe_ntt_fwd / fhe_ntt_inv (kTcPlaneBytes)
    uint32_t* ntt_temp = nullptr;  // two-pass plain NTT scratch (kNttTempBytes, stays in L2)
    uint32_t* d_mods = nullptr;  // device copy of `mods`
};

namespace fhe {

// Per-limb modulus mapping passed by value to kernels.
// Up to 128 limbs per launch (two ciphertext components of 64 limbs each).
constexpr int kMaxLimbs = 2 * FHE_MAX_MODULI;
struct LimbMap {
    uint32_t q[kMaxLimbs];
    uint8_t mod[kMaxLimbs];
};

// One row of a row-table NTT launch: a polynomial limb anywhere in device memory.
struct RowRef {
    uint32_t* ptr;
    uint32_t mod;  // modulus index into the context's moduli
    uint32_t pad;
};

// Device scratch of the two-pass plain NTT for one call: `bytes` (a multiple of N * 4 is
// used) at `p`. p == nullptr selects the context's own scratch, which calls on different
// streams must not use at the same time; library operations that take a caller scratch pass
// a region of it instead (ntt_region_bytes).
struct NttScratch {
    uint32_t* p = nullptr;
    size_t bytes = 0;
};
// Bytes of that region for NTT calls of up to `rows` rows at 2^logN (0 below 2^12).
size_t ntt_region_bytes(uint32_t logN, size_t rows);
// Digit-plane buffer of the tensor-core NTT between its two GEMMs: the context's own buffer
// (fhe_ntt_fwd / fhe_ntt_inv), and the most an operation's scratch region provides for it.
// 256 MiB holds the planes of 8 limbs x 64 polynomials at N = 2^16. Smaller buffers were
// measured on a GB300 (64 and 128 MiB): every chunk costs two more launches and their tails,
// and the planes still did not stay in L2 between the two GEMMs.
#ifndef FHE_TC_PLANE_MIB
#define FHE_TC_PLANE_MIB 256
#endif
constexpr size_t kTcPlaneBytes = (size_t)FHE_TC_PLANE_MIB << 20;
// The NTT region of a CKKS operation's scratch for NTT calls of up to `rows` rows on this
// context: the two-pass region, and on a tensor-core context room for its digit planes.
size_t op_region_bytes(const fhe_ctx* ctx, uint32_t logN, size_t rows);

// Plain-path NTT over rows listed in a device table (operation-level batching of rows
// that live in different buffers).
int ntt_u32_rows(const fhe_ctx* ctx, uint32_t logN, bool inverse, const RowRef* d_rows, int nrows,
                 cudaStream_t stream, NttScratch scr = NttScratch());

// Plain-path NTT for N >= 2^15 in two passes through a scratch buffer (ntt_u32_l2.cu).
int ntt_u32_l2(const fhe_ctx* ctx, uint32_t logN, int shape, bool inverse, uint32_t* d, int rows, int batch,
               const LimbMap& map, const RowRef* rowtab, cudaStream_t st, NttScratch scr);

// The HMULT + RESCALE tail (ckks.cu) fused into the forward two-pass NTT of z. Row r of the
// transform is limb (c, i) = (r / batch / nout, r / batch % nout) of polynomial p = r % batch.
// The local pass loads z'_i = y'_i + [last]_q_i q_l^-1 (last taken centred in (-q_l/2, q_l/2])
// instead of a stored z', and the cross pass stores out_i = ks'_i + d'_i - z'^_i instead of
// z'^: the two HBM passes that would build z' and combine z'^ disappear. y', ks', d' are the
// ModDown conversion, key-switching output and tensor product already multiplied by
// P^-1 q_l^-1, P^-1 q_l^-1 and q_l^-1 (limbs i < l).
struct HmultTail {
    const uint32_t* y;     // (2, nl, batch, N): y', coefficient domain
    const uint32_t* last;  // (2, batch, N): the relinearised last limb, coefficient domain, [0, q_l);
                           // null: no last-limb term (z' = y', the ModDown combine of key switching)
    const uint32_t* ks;    // (2, ext, batch, N): ks', NTT domain
    const uint32_t* d;     // (2, nl, batch, N): d0', d1', NTT domain
    uint32_t* out;         // (2, nout, batch, N)
    const uint2* qlinv;    // [i] q_l^-1 mod q_i (value, Shoup quotient)
    uint32_t ql;
    int nl, nout, ext;
};
// True when the inverse NTT of this ring degree runs the two-pass plain kernels, which can read
// their input from another buffer than the one they write.
bool ntt_inv_out_of_place(const fhe_ctx* ctx, uint32_t logN);
// Inverse NTT of src (n_limbs x batch rows, NTT domain, limb moduli from map) into dst: read
// directly by the two-pass kernels where ntt_inv_out_of_place holds, else copied into dst and
// transformed there. src is left unchanged either way.
int ntt_inv_from(const fhe_ctx* ctx, uint32_t logN, uint32_t* dst, const uint32_t* src, int n_limbs, int batch,
                 const LimbMap& map, cudaStream_t st, NttScratch scr);
// True when the forward NTT of this ring degree runs the two-pass plain kernels (the only ones
// with the fused tail); the tail then runs as one call to ntt_u32_l2_tail.
bool ntt_tail_fusable(const fhe_ctx* ctx, int path, uint32_t logN);
int ntt_u32_l2_tail(const fhe_ctx* ctx, uint32_t logN, int rows, int batch, const LimbMap& map, cudaStream_t st,
                    NttScratch scr, const HmultTail& tail);

// Plain-path batched NTT over `n_limbs` limbs whose moduli are map.mod[l].
int ntt_u32(const fhe_ctx* ctx, uint32_t logN, bool inverse, uint32_t* d, int n_limbs,
            int batch, const LimbMap& map, cudaStream_t stream, NttScratch scr = NttScratch());
// Tensor-core path; its digit planes go to scr (at least 8 N bytes) when given, else to the
// context's own buffer.
int ntt_tc(const fhe_ctx* ctx, uint32_t logN, bool inverse, uint32_t* d, int n_limbs,
           int batch, const LimbMap& map, cudaStream_t stream, NttScratch scr = NttScratch());
int build_tc_tables(fhe_ctx* ctx, uint32_t logN);
int build_ntt_tables(fhe_ctx* ctx, uint32_t logN);

// Basis conversion (Conv of Sec. IV-A) on the tensor cores (conv_tc.cu): for every
// coefficient n and destination t, dst_t[n] = sum_i [x_i[n] (B/b_i)^-1]_{b_i} [B/b_i]_t mod q_t,
// as one exact fp16 GEMM per 128 coefficients (K' = 4 nsrc data digits, N = 4 ndst constant
// digits, fp32 accumulation in TMEM) and a shift-and-add reconstruction.
struct TcConvArgs {
    const uint32_t* src;
    size_t src_stride;         // elements between source limbs
    int nsrc;                  // 1..15
    uint32_t src_q[16];
    uint2 hat_inv[16];         // [(B/b_i)^-1]_{b_i} (value, Shoup quotient)
    const uint16_t* bdig;      // ConvTable::bdig
    uint32_t* dst;
    size_t dst_stride;
    int ndst;                  // 1..64
    uint8_t dst_mod[64];       // modulus index of destination t
    uint32_t dst_q[64];
    uint2 dst_c16[64];         // [2^16]_{q_t} (value, Shoup quotient)
    uint2 dst_one[64];         // 1 with its Shoup quotient floor(2^32 / q_t): a reduction mod q_t
    uint32_t dst_off[64];      // the least multiple of q_t that is >= 2^29
    size_t ncoef;              // coefficients per limb (batch x N)
};
int launch_conv_tc(const fhe_ctx* ctx, const TcConvArgs& a, cudaStream_t st);

// Dispatch on path.
int ntt_any(const fhe_ctx* ctx, int path, uint32_t logN, bool inverse, uint32_t* d, int n_limbs,
            int batch, const LimbMap& map, cudaStream_t stream, NttScratch scr = NttScratch());

LimbMap contiguous_map(const fhe_ctx* ctx, int first, int n);

template <typename T>
int dev_alloc(fhe_ctx* ctx, T** p, size_t count) {
    void* v = nullptr;
    cudaError_t e = cudaMalloc(&v, count * sizeof(T) + 16);
    if (e != cudaSuccess) {
        set_error(FHE_ENOMEM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
        return FHE_ENOMEM;
    }
    ctx->allocations.push_back(v);
    *p = (T*)v;
    return FHE_OK;
}

template <typename T>
int dev_upload(fhe_ctx* ctx, T** p, const std::vector<T>& h) {
    int rc = dev_alloc(ctx, p, h.size());
    if (rc) return rc;
    FHE_CUDA_TRY(cudaMemcpy(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
    return FHE_OK;
}

// ---------------------------------------------------------------- device helpers

// Shared-memory layout of a CTA's 32 * T residues in the plain NTT kernels: position p lives
// at word pad(p) = p + p / 32 + p / T (the last term only for T > 32). The map is strictly
// increasing, every access pattern of the kernels' rounds touches 32 distinct banks per warp
// under it, and for tid < T each pattern is a per-thread base plus a compile-time offset:
//   p = tid + T e           -> pad(tid) + kSA e
//   p = T g + lane + 32 e   -> kSA g + lane + 33 e          (e < T / 32)
//   p = 32 g + e            -> pad(32 g) + e                (e < 32)
//   p = (c 32T + tid) / C + u T / C -> pad(p at u = 0) + offK(u)   (T / C >= 32)
// Round C reads p = 32 rev(tid) + e; within a warp rev(tid) = rev5(lane) 2^(log T - 5) + r,
// so its bank is (rev5(lane) (2^(log T - 5) + 1) + r + e) mod 32: an odd multiple of a
// permutation of the lanes.
template <int LOG_T>
struct PadLayout {
    static constexpr int T = 1 << LOG_T;
    static constexpr int kHi = LOG_T > 5 ? 1 : 0;
    static constexpr int kSA = T + T / 32 + kHi;
    static constexpr int kWords = 33 * T + 32;
    __host__ __device__ static constexpr int pad(int p) { return p + (p >> 5) + (kHi ? (p >> LOG_T) : 0); }
    template <int LOG_C>
    __host__ __device__ static constexpr int offK(int u) {
        return u * ((T >> LOG_C) + (T >> (LOG_C + 5))) + kHi * (u >> LOG_C);
    }
};

// Shoup multiplication by a constant, lazy: for any x < 2^32 returns x*w mod q in [0, 2q).
__device__ __forceinline__ uint32_t mul_shoup_lazy(uint32_t x, uint32_t w, uint32_t wq, uint32_t q) {
    uint32_t qt = __umulhi(x, wq);
    return x * w - qt * q;
}
// [0, 2m) -> [0, m) for m = q or 2q; relies on unsigned wrap-around.
__device__ __forceinline__ uint32_t csub(uint32_t x, uint32_t m) { return min(x, x - m); }

__device__ __forceinline__ uint32_t mul_shoup(uint32_t x, uint32_t w, uint32_t wq, uint32_t q) {
    return csub(mul_shoup_lazy(x, w, wq, q), q);
}

// Four balanced base-256 digits of v < 2^30 as fp16: v = sum_j (b_j - 128) 256^j where b_j are
// the bytes of v + 0x80808080 (no wrap-around since v < 2^30). The half with bits 0x64bb is
// exactly 1024 + bb, so one byte permute per pair of digits and one f16x2 subtraction of
// 1152 give the digits exactly (every integer of magnitude <= 2048 is exact in fp16).
__device__ __forceinline__ uint2 split_f16x4(uint32_t v) {
    const uint32_t y = v + 0x80808080u;
    const uint32_t lo = __byte_perm(y, 0x64u, 0x4140), hi = __byte_perm(y, 0x64u, 0x4342);
    uint2 r;
    asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(r.x) : "r"(lo), "r"(0x64806480u));
    asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(r.y) : "r"(hi), "r"(0x64806480u));
    return r;
}

// fp16 bit pattern of a small integer (exact for |e| <= 2048; host side).
inline uint16_t f16_bits_of_small_int(int e) {
    if (e == 0) return 0;
    const uint16_t sign = e < 0 ? 0x8000 : 0;
    const uint32_t a = (uint32_t)(e < 0 ? -e : e);
    int ex = 0;
    while ((a >> (ex + 1)) != 0) ++ex;  // 2^ex <= a < 2^(ex+1)
    const uint32_t mant = (a << (10 - ex)) & 0x3FFu;
    return (uint16_t)(sign | ((ex + 15) << 10) | mant);
}

// 64-bit Barrett: x mod q for any x < 2^64, with mu = floor(2^64 / q) (q < 2^31).
__device__ __forceinline__ uint32_t reduce_u64(uint64_t x, uint64_t mu, uint32_t q) {
    uint64_t qt = __umul64hi(x, mu);
    uint64_t r = x - qt * (uint64_t)q;  // in [0, 3q)
    uint32_t r32 = (uint32_t)r;
    r32 = csub(r32, 2 * q);
    return csub(r32, q);
}

__device__ __forceinline__ uint32_t mulmod(uint32_t a, uint32_t b, uint32_t q, uint64_t mu) {
    return reduce_u64((uint64_t)a * b, mu, q);
}

}  // namespace fhe

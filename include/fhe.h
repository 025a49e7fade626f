/*
 * fhe.h -- C ABI of libfhe: batched negacyclic NTT/INTT and CKKS HMULT on one
 * NVIDIA GB300 (sm_103a), after TensorFHE (arXiv 2212.14191).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Residues are uint32 values in canonical form [0, q) for the limb's prime q.
 * - Polynomial data use the limb-major (L, B, N) layout of Sec. IV-D: limb l of
 *   polynomial b starts at element (l * B + b) * N and holds N coefficients
 *   (coefficient domain) or N NTT values (NTT domain, natural order k = 0..N-1).
 * - A ciphertext batch is (2, L, B, N): component c (c = 0, 1) first. The pair
 *   decrypts as c0 + c1 * s; both components are stored in the NTT domain.
 * - "Modulus index" t numbers the context's moduli: q_0..q_{nq-1} are t = 0..nq-1
 *   and the special primes p_0..p_{np-1} are t = nq..nq+np-1.
 * - Device pointers are caller-owned, must be 16-byte aligned and must stay valid
 *   until the work queued on `stream` has finished. Host pointers are read (or
 *   written) before the call returns unless stated otherwise.
 * - Every call is asynchronous on the given CUDA stream (cudaStream_t passed as
 *   void*; NULL is the legacy default stream) and returns a status code. Nothing
 *   throws across the ABI. fhe_last_error() gives a message for the calling
 *   thread's most recent failure.
 * - Inputs are not checked for being below q (an input >= q gives an unspecified
 *   but in-bounds result); every other argument is validated before any launch.
 */
#ifndef FHE_H
#define FHE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define FHE_OK 0
#define FHE_EINVAL 1   /* malformed call: range, null/misaligned pointer, bad moduli */
#define FHE_ENOMEM 2   /* scratch too small, or a library allocation failed */
#define FHE_ECUDA 3    /* a CUDA launch or runtime call failed (message has the CUDA error) */
#define FHE_ETIMEOUT 4 /* a bounded device-side wait expired */

/* NTT implementations (Sec. IV-B/IV-C). FHE_NTT_DEFAULT picks the context's default. */
#define FHE_NTT_DEFAULT 0
#define FHE_NTT_U32 1 /* 32-bit integer butterflies on CUDA cores (Shoup/Harvey arithmetic) */
#define FHE_NTT_TC 2  /* four-step NTT, 8-bit segments on tcgen05 tensor cores */

#define FHE_LOGN_MIN 10
#define FHE_LOGN_MAX 16
#define FHE_MAX_MODULI 64

typedef struct fhe_ctx fhe_ctx;

/*
 * fhe_gen_primes -- the `count` largest primes q < 2^bits with q = 1 mod 2^(logN_max+1),
 * in descending order, written to host array out[count].
 * Sec. II-A only asks for a prime with a primitive N-th (here 2N-th) root of unity; this
 * helper fixes one deterministic choice. bits in [20, 31], logN_max in [10, 16].
 * Returns FHE_EINVAL when fewer than `count` such primes exist above 2^(bits-1).
 */
int fhe_gen_primes(uint32_t logN_max, int bits, int count, uint32_t* out);

/*
 * fhe_ctx_create -- validate the moduli and build every per-modulus table on the device.
 *   logN_max : tables are built for every N = 2^logN, FHE_LOGN_MIN <= logN <= logN_max.
 *   q[nq]    : ciphertext primes q_0..q_{nq-1} (host array), the RNS limbs of Sec. II-B.
 *   p[np]    : special primes p_0..p_{np-1} of generalized key switching (Sec. II-B); np may
 *              be 0 (then HMULT and key switching are unavailable).
 *   alpha    : primes per key-switching slice Q_j (Sec. II-B: alpha = (L+1)/dnum); the last
 *              slice may be short. Requires prod(p) > every slice product (checked).
 *   default_path : FHE_NTT_U32 or FHE_NTT_TC, used by FHE_NTT_DEFAULT and by the HMULT pipeline.
 * Every prime must be distinct, prime, < 2^30 and = 1 mod 2^(logN_max+1); nq + np <= 64;
 * 1 <= alpha <= 15; np <= 15. The context owns its device tables.
 * Concurrency: the CKKS operations (fhe_keyswitch .. fhe_hadd) take every NTT buffer they
 * use, the tensor-core path's digit planes included, from the caller's scratch, so calls on
 * one context may run at the same time on different streams with separate scratch buffers.
 * fhe_ntt_fwd / fhe_ntt_inv with a two-pass plain variant or the tensor-core path use buffers
 * owned by the context and must not overlap one another in time on one context. Calls that
 * change the context (fhe_ntt_set_variant, fhe_autotune_ntt, fhe_conv_set_path) must not
 * race with any call using it; the tensor-core tables of a ring degree are built on its first
 * tensor-core call, under a lock.
 * Allocates device memory (cudaMalloc) on the current device: the tables, and for
 * logN_max >= 15 a 1 GiB scratch for the two-pass plain NTT; *out = NULL on failure.
 */
int fhe_ctx_create(uint32_t logN_max, const uint32_t* q, int nq, const uint32_t* p, int np,
                   int alpha, int default_path, fhe_ctx** out);

/* Frees the context's device tables. Work using the context must have completed. */
int fhe_ctx_destroy(fhe_ctx* ctx);

/*
 * fhe_ntt_fwd -- in-place negacyclic NTT of Eq. (4), Sec. II-A:
 *     A_k = sum_{n<N} a_n * psi^(2nk+n) mod q,   k in [0, N), natural order in and out,
 * psi = x^((q-1)/2N) for the smallest quadratic non-residue x of q.
 *   d          : device (n_limbs, batch, N) uint32, transformed in place.
 *   first_limb : modulus index of limb 0; limb l uses modulus first_limb + l.
 *   path       : FHE_NTT_DEFAULT, FHE_NTT_U32 or FHE_NTT_TC.
 * n_limbs >= 1, first_limb + n_limbs <= nq + np, batch >= 0 (0 is a no-op).
 */
int fhe_ntt_fwd(const fhe_ctx* ctx, int path, uint32_t logN, uint32_t* d, int first_limb,
                int n_limbs, int batch, void* stream);

/*
 * Plain-path variants that run in two passes (and the tensor-core path) use buffers owned
 * by the context: fhe_ntt_fwd / fhe_ntt_inv calls on one context must not overlap in time on
 * different streams (see fhe_ctx_create; the CKKS calls below may overlap).
 *
 * fhe_ntt_inv -- in-place inverse of fhe_ntt_fwd (Sec. II-A, Eq. (2) with the psi^-n
 * post-twist of Eq. (3); Sec. IV-C Stage 5 names the N^-1 factor):
 *     a_n = N^-1 * psi^-n * sum_{k<N} A_k * psi^(-2nk) mod q.
 * Arguments as fhe_ntt_fwd.
 */
int fhe_ntt_inv(const fhe_ctx* ctx, int path, uint32_t logN, uint32_t* d, int first_limb,
                int n_limbs, int batch, void* stream);

/*
 * NTT variants (an interface of this library; the paper picks batch sizes per kernel from the
 * hardware in its API layer, Sec. IV-E, but gives no tuning procedure). Ids 0..31 are
 * plain-path variants: a CTA shape, how a thread-block cluster shares a limb, where last-round
 * twiddles live and the register budget. FHE_NTT_VARIANT_TC64 and FHE_NTT_VARIANT_TC32 are the
 * tensor-core path with output tiles of 64 or 32 columns. Variants change only speed, never
 * results. Per ring degree and direction the context keeps the choice that FHE_NTT_DEFAULT
 * runs (initially the context's default path: plain variants chosen per N, or TC64), the
 * plain-path variant that FHE_NTT_U32 calls run and the tile width that FHE_NTT_TC calls run.
 * fhe_ntt_variant_count -- number of variant ids for logN (ids 0..count-1, not all of which
 *   apply at every logN), or -1 on bad input.
 * fhe_ntt_get_variant -- the choice FHE_NTT_DEFAULT runs for logN, forward (inverse = 0) or
 *   inverse (inverse != 0), HMULT and the other CKKS operations included; -1 on bad input.
 * fhe_ntt_set_variant -- select the forward and the inverse choice for logN (a plain id also
 *   becomes the variant of FHE_NTT_U32 calls, a tensor-core id the tile width of FHE_NTT_TC
 *   calls); FHE_EINVAL if either does not apply. Must not race with calls that use the
 *   context. fhe_scratch_bytes grows where a tensor-core choice is made.
 * fhe_autotune_ntt -- times every applicable choice on forward and inverse transforms of
 *   `d` (device (n_limbs, batch, N), limbs use moduli 0..n_limbs-1; restored bit-exactly on
 *   return), keeps the fastest for each direction (and the fastest plain variant and tile
 *   width for explicit-path calls), and writes milliseconds per call to host array
 *   ms_out[2 * fhe_ntt_variant_count] (nullable): forward times at [v], inverse times at
 *   [count + v], -1 where choice v does not apply. Synchronises `stream`.
 */
#define FHE_NTT_VARIANT_TC64 32
#define FHE_NTT_VARIANT_TC32 33
int fhe_ntt_variant_count(const fhe_ctx* ctx, uint32_t logN);
int fhe_ntt_get_variant(const fhe_ctx* ctx, uint32_t logN, int inverse);
int fhe_ntt_set_variant(fhe_ctx* ctx, uint32_t logN, int fwd_variant, int inv_variant);
int fhe_autotune_ntt(fhe_ctx* ctx, uint32_t logN, uint32_t* d, int n_limbs, int batch, int reps,
                     float* ms_out, void* stream);

/*
 * Basis conversion (Conv of ModUp and ModDown, Sec. IV-A) kernels; both compute the same exact
 * residues sum_i [x_i (B/b_i)^-1]_{b_i} [B/b_i]_t mod q_t.
 *   FHE_CONV_CUDA : 64-bit multiply-adds on the CUDA cores (the default: faster on GB300).
 *   FHE_CONV_TC   : the same products as an exact fp16 GEMM of 8-bit segments on the tcgen05
 *                   tensor cores; with at most 15 terms per output the reconstruction costs
 *                   about as much as the multiply-adds it replaces.
 * fhe_conv_set_path -- select the kernel used by this context's key switching (HMULT,
 *   HROTATE, fhe_keyswitch); FHE_EINVAL for another value. Must not race with calls that use
 *   the context.
 * fhe_conv_get_path -- the selected kernel, or -1 if ctx is NULL.
 */
#define FHE_CONV_CUDA 0
#define FHE_CONV_TC 1
int fhe_conv_set_path(fhe_ctx* ctx, int path);
int fhe_conv_get_path(const fhe_ctx* ctx);

/* Operations for fhe_scratch_bytes. */
#define FHE_OP_HMULT 1
#define FHE_OP_KEYSWITCH 2
#define FHE_OP_RESCALE 3
#define FHE_OP_HMULT_RELIN 4
#define FHE_OP_HROTATE 5
#define FHE_OP_HROTATE_HOISTED 6

/*
 * fhe_scratch_bytes -- device scratch (bytes) that fhe_hmult / fhe_keyswitch /
 * fhe_rescale / fhe_hmult_relin / fhe_hrotate / fhe_hrotate_hoisted need for these sizes
 * (op = the matching FHE_OP_*; the hoisted size does not depend on the number of
 * rotations); 0 for invalid arguments.
 */
size_t fhe_scratch_bytes(const fhe_ctx* ctx, int op, uint32_t logN, int n_limbs, int batch);

/*
 * fhe_keyswitch -- generalized (hybrid) key switching of Sec. II-B / Sec. IV-A (Alg. 1):
 * Dcomp + ModUp per slice, inner product with the evaluation key, ModDown.
 *   d2     : device (n_limbs, batch, N), NTT domain, limbs q_0..q_{n_limbs-1}.
 *   evk    : device (dnum, 2, nq + np, N), NTT domain, dnum = ceil(nq / alpha); slice j,
 *            component c, modulus index t at ((j*2 + c)*(nq+np) + t) * N. Only limbs
 *            t < n_limbs and t >= nq are read.
 *   ks_out : device (2, n_limbs, batch, N): (ks0, ks1) with ks0 + ks1*s ~ d2 * s^2.
 *   scratch: device buffer of at least fhe_scratch_bytes(ctx, FHE_OP_KEYSWITCH, ...) bytes.
 * 1 <= n_limbs <= nq. ks_out must not overlap d2 or scratch.
 */
int fhe_keyswitch(const fhe_ctx* ctx, uint32_t logN, int n_limbs, int batch, const uint32_t* d2,
                  const uint32_t* evk, uint32_t* ks_out, void* scratch, size_t scratch_bytes,
                  void* stream);

/*
 * fhe_hmult_relin -- HMULT of Sec. II-B without rescale:
 *   (d0, d1, d2) = (a0*b0, a0*b1 + a1*b0, a1*b1);  out = (d0 + ks0, d1 + ks1), (ks0, ks1) =
 *   KeySwitch(d2).
 *   ct_a, ct_b : device (2, n_limbs, batch, N) NTT domain.   out : device (2, n_limbs, batch, N).
 * out must not overlap the inputs or scratch. 1 <= n_limbs <= nq.
 */
int fhe_hmult_relin(const fhe_ctx* ctx, uint32_t logN, int n_limbs, int batch,
                    const uint32_t* ct_a, const uint32_t* ct_b, const uint32_t* evk,
                    uint32_t* out, void* scratch, size_t scratch_bytes, void* stream);

/*
 * fhe_rescale -- RESCALE of Sec. II-B (Alg. 6): divide by the last prime q_l, rounding to
 * nearest (the last limb is centred to (-q_l/2, q_l/2] before subtraction).
 *   ct_in  : device (2, n_limbs, batch, N), NTT domain.
 *   ct_out : device (2, n_limbs - 1, batch, N); may not overlap ct_in.
 * 2 <= n_limbs <= nq.
 */
int fhe_rescale(const fhe_ctx* ctx, uint32_t logN, int n_limbs, int batch, const uint32_t* ct_in,
                uint32_t* ct_out, void* scratch, size_t scratch_bytes, void* stream);

/*
 * fhe_hmult -- HMULT with relinearisation followed by RESCALE (Sec. II-B; Alg. 2 then Alg. 6):
 *   ct_a, ct_b : device (2, n_limbs, batch, N); ct_out : device (2, n_limbs - 1, batch, N).
 * 2 <= n_limbs <= nq. ct_out must not overlap inputs or scratch.
 */
int fhe_hmult(const fhe_ctx* ctx, uint32_t logN, int n_limbs, int batch, const uint32_t* ct_a,
              const uint32_t* ct_b, const uint32_t* evk, uint32_t* ct_out, void* scratch,
              size_t scratch_bytes, void* stream);

/*
 * The other ciphertext operations of Sec. II-B's table (HROTATE with its FrobeniusMap,
 * CMULT, HADD). Ciphertexts are (2, n_limbs, batch, N) in the NTT domain over q_0.., as for
 * fhe_hmult; device pointers 16-byte aligned; asynchronous on `stream`.
 *
 * fhe_automorph -- FrobeniusMap a(X) -> a(X^galois) of `rows` NTT-domain rows of length N
 *   (any moduli: in the NTT domain the map is the permutation out[j] = in[j'] with
 *   2j' + 1 = (2j + 1) galois mod 2N). galois odd and < 2N; in and out must not overlap.
 * fhe_hrotate -- HROTATE: (c0(X^k) + ks0, ks1) with (ks0, ks1) = KeySwitch(c1(X^k)) and
 *   k = galois (5^r mod 2N rotates the slots by r, 2N - 1 conjugates them). `ksk` is the
 *   key from s(X^k) to s in the layout of `evk` above. Scratch: fhe_scratch_bytes(
 *   FHE_OP_HROTATE); ct_out must not overlap ct_in. No rescale.
 * fhe_hrotate_hoisted -- n_rot HROTATEs of one ciphertext batch sharing one ModUp (hoisted
 *   rotations): ModUp of c1 is formed once in the NTT domain and each rotation key-switches
 *   those digits permuted by its automorphism (computed as the inner product of the unpermuted
 *   digits with the key permuted by the inverse automorphism, then permuted: the same values,
 *   since the product is pointwise), followed by ModDown. The approximate Conv
 *   does not commute exactly with X -> X^k, so each result is a valid key switch of c1(X^k)
 *   but not bit-identical to fhe_hrotate's: the automorphism of ModUp(c1) differs from ModUp
 *   of c1(X^k) by B_j times the number of nonzero Conv terms at every negated coefficient.
 *   galois: host array of n_rot odd elements < 2N; ksk: host array of n_rot device pointers,
 *   key r from s(X^galois[r]) to s in the layout of `evk`; ct_out: (n_rot, 2, n_limbs, batch,
 *   N), which must not overlap ct_in. Scratch: fhe_scratch_bytes(FHE_OP_HROTATE_HOISTED),
 *   independent of n_rot. n_rot = 0 or batch = 0 does nothing. No rescale.
 * fhe_cmult -- CMULT: both components times the plaintext `pt` ((n_limbs, batch, N), NTT
 *   domain, one plaintext per ciphertext), limbwise mod q_i. No rescale. May run in place.
 * fhe_hadd -- HADD: ct_a + ct_b limbwise mod q_i. May run in place.
 * Errors: FHE_EINVAL for bad sizes, pointers or galois elements; FHE_ENOMEM for a short
 * scratch; FHE_ECUDA for launch failures.
 */
int fhe_automorph(const fhe_ctx* ctx, uint32_t logN, long long rows, uint32_t galois, const uint32_t* in,
                  uint32_t* out, void* stream);
int fhe_hrotate(const fhe_ctx* ctx, uint32_t logN, int n_limbs, int batch, uint32_t galois,
                const uint32_t* ct_in, const uint32_t* ksk, uint32_t* ct_out, void* scratch,
                size_t scratch_bytes, void* stream);
int fhe_hrotate_hoisted(const fhe_ctx* ctx, uint32_t logN, int n_limbs, int batch, int n_rot,
                        const uint32_t* galois, const uint32_t* ct_in, const uint32_t* const* ksk,
                        uint32_t* ct_out, void* scratch, size_t scratch_bytes, void* stream);
int fhe_cmult(const fhe_ctx* ctx, uint32_t logN, int n_limbs, int batch, const uint32_t* ct,
              const uint32_t* pt, uint32_t* ct_out, void* stream);
int fhe_hadd(const fhe_ctx* ctx, uint32_t logN, int n_limbs, int batch, const uint32_t* ct_a,
             const uint32_t* ct_b, uint32_t* ct_out, void* stream);

/*
 * Operation-level batching (Sec. IV-D) of many independent operations with uneven ring
 * degree and level, replayed as one CUDA graph launch.
 *   fhe_op: one operation. kind FHE_OPK_NTT_FWD / FHE_OPK_NTT_INV transform `data`
 *     (n_limbs, batch, N) in place with moduli first_limb.. (plain 32-bit path); kind
 *     FHE_OPK_HMULT computes out = fhe_hmult(a, b, evk) at n_limbs ciphertext limbs
 *     (first_limb ignored). All device pointers 16-byte aligned; operations must not
 *     overlap in memory; their results equal those of the single-operation calls.
 *   fhe_batch_create -- validates and plans the list (mode FHE_BATCH_PERSISTENT, default slot
 *     budget). Allocates the plan's device tables (cudaMalloc). The op list may be freed
 *     afterwards; the buffers it names must outlive the plan's runs.
 *   fhe_batch_create_ex -- the same with a mode:
 *     FHE_BATCH_PERSISTENT: every operation at N >= 2^14 runs inside ONE persistent kernel
 *       launch whose CTAs (a grid sized from the SM count and the kernel's occupancy) pop
 *       tiles of the operations' stages from a device queue: NTT/INTT local passes of one row
 *       part, and chunks of 16384 residues of the HMULT's tensor product, basis conversions,
 *       inner product and last-limb steps. A tile starts once the stages it reads have
 *       completed (device counters, bounded waits: an expired wait records FHE_ETIMEOUT in the
 *       context's status word, the remaining tiles are skipped, the kernel ends; see
 *       fhe_device_status). HMULTs run in scratch slots of at most `slot_bytes` in total
 *       (0: 8 GiB; at least one slot); an HMULT waits for the previous one of its slot.
 *       Operations at N < 2^14 run in the grouped form below, before the persistent launch.
 *       The transforms inside the persistent launch are plain 32-bit two-pass tiles whatever
 *       the context's default path (results are identical on either path).
 *     FHE_BATCH_GROUPED: every limb transform of one (N, direction) becomes a row of one NTT
 *       launch (plain path); HMULTs sharing (N, n_limbs, evk) are gathered into one batched
 *       fhe_hmult, which follows the context's default path; the groups run one after another.
 *   fhe_batch_scratch_bytes -- device scratch needed by fhe_batch_run / _capture.
 *   fhe_batch_run -- enqueues the plan on `stream` (capturable in a CUDA graph). A persistent
 *     plan's first run on a scratch buffer (and the first after a change of buffer) uploads
 *     its tables, which hold absolute addresses inside that buffer, synchronously: it fails
 *     with FHE_EINVAL during stream capture, and earlier runs on other buffers must be done.
 *   fhe_batch_capture -- runs the plan once, then captures it into a graph owned by the plan
 *     (bound to this scratch buffer); fhe_batch_launch replays that graph on `stream`.
 *   fhe_batch_destroy -- frees the plan and its graph (no work may be pending).
 */
#define FHE_OPK_NTT_FWD 1
#define FHE_OPK_NTT_INV 2
#define FHE_OPK_HMULT 3
typedef struct fhe_op {
    int kind;
    uint32_t logN;
    int first_limb;
    int n_limbs;
    int batch;
    uint32_t* data;
    const uint32_t* a;
    const uint32_t* b;
    const uint32_t* evk;
    uint32_t* out;
} fhe_op;
typedef struct fhe_batch fhe_batch;
#define FHE_BATCH_PERSISTENT 0
#define FHE_BATCH_GROUPED 1
int fhe_batch_create(const fhe_ctx* ctx, const fhe_op* ops, int n, fhe_batch** out);
int fhe_batch_create_ex(const fhe_ctx* ctx, const fhe_op* ops, int n, int mode, size_t slot_bytes,
                        fhe_batch** out);
size_t fhe_batch_scratch_bytes(const fhe_batch* b);
int fhe_batch_run(const fhe_batch* b, void* scratch, size_t scratch_bytes, void* stream);
int fhe_batch_capture(fhe_batch* b, void* scratch, size_t scratch_bytes);
int fhe_batch_launch(const fhe_batch* b, void* stream);
int fhe_batch_destroy(fhe_batch* b);

/*
 * fhe_rescale_noalloc -- the same RESCALE as fhe_rescale, for callers that cannot allocate
 * device memory: a serving loop that must not stall the device (cudaMalloc/cudaFree may
 * synchronise it), code whose device memory is all owned by another allocator under a fixed
 * budget, or a plugin host that forbids device allocations. The paper has no counterpart; it
 * is an interface convenience of this library.
 *   Scratch comes from a fixed array of FHE_RESCALE_NOALLOC_MAX_BYTES bytes compiled into the
 *   library's device image; every GPU that loads the library holds it until process exit.
 *   The call allocates nothing. A size whose scratch (fhe_scratch_bytes(ctx, FHE_OP_RESCALE,
 *   ...)) exceeds the array is rejected with FHE_ENOMEM.
 *   The first call on a device looks up the array's device address (cudaGetSymbolAddress,
 *   with that device current) and caches it; make that first call before any stream capture.
 *   The cached address does not survive cudaDeviceReset (neither does any context).
 *   The current device must be the context's device (FHE_EINVAL otherwise).
 *   All calls share the one array and it keeps the last call's contents: calls whose GPU work
 *   overlaps (other streams, other threads) race on it, so serialise them on one stream.
 * Arguments and layouts as fhe_rescale.
 */
#define FHE_RESCALE_NOALLOC_MAX_BYTES (32u << 20)
int fhe_rescale_noalloc(const fhe_ctx* ctx, uint32_t logN, int n_limbs, int batch,
                        const uint32_t* ct_in, uint32_t* ct_out, void* stream);

/*
 * fhe_device_status -- reads (and with clear != 0 resets) the context's device error word,
 * which kernels set when a bounded device-side wait expires (their work is then incomplete).
 * Returns FHE_OK, or FHE_ETIMEOUT. Synchronous: waits for the device copy of the word.
 */
int fhe_device_status(const fhe_ctx* ctx, int clear);

/*
 * fhe_selftest_wait_timeout -- checks the failure path of fhe_device_status without faulting
 * the GPU: launches on `stream` one kernel whose mbarrier wait can never complete (nothing
 * arrives) and which gives up after limit_cycles SM clock cycles (0 < limit_cycles <= 4e9,
 * about two seconds at the maximum clock), recording FHE_ETIMEOUT in the context's device
 * error word exactly as the library's kernels do when one of their bounded waits expires.
 * The context stays usable; fhe_device_status(ctx, 1) then reports and clears the word.
 */
int fhe_selftest_wait_timeout(const fhe_ctx* ctx, long long limit_cycles, void* stream);

/*
 * fhe_selftest_queue_timeout -- the same check for the persistent batch kernel's dependency
 * waits (fhe_batch_create_ex, FHE_BATCH_PERSISTENT): runs that kernel on `stream` over a queue
 * of one tile whose dependency counter nothing increments, with the wait limited to
 * limit_cycles (0 < limit_cycles <= 4e9). The wait expires, FHE_ETIMEOUT is recorded in the
 * context's device error word and the kernel returns. Allocates a few bytes of device memory
 * and waits for the stream before returning.
 */
int fhe_selftest_queue_timeout(const fhe_ctx* ctx, long long limit_cycles, void* stream);

/*
 * fhe_last_error -- copy the calling thread's last error message (NUL-terminated, truncated
 * to n bytes) into buf; returns the status code of that failure (FHE_OK if none).
 */
int fhe_last_error(char* buf, size_t n);

#ifdef __cplusplus
}
#endif

#endif /* FHE_H */

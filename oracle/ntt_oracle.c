/*
 * CPU oracle for the negacyclic NTT / INTT (TensorFHE, arXiv 2212.14191).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the plain, slow, obviously correct
 * definition that the GPU library is checked against. Only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg may load it; the GPU
 * library never links it and shares no code with it.
 *
 * Arithmetic: residues are u32 values below a prime q < 2^32, every product is
 * formed exactly in u64 and reduced with the C '%' operator. Nothing here is
 * lazy, blocked or fused.
 *
 * Definitions implemented (paper section II-A):
 *   forward, Eq. (4):  A_k = sum_{n<N} a_n * psi^(2nk+n)        mod q, k in [0,N)
 *   inverse:           a_n = N^-1 * psi^-n * sum_{k<N} A_k * psi^(-2nk)  mod q
 *     (the inverse of Eq. (4); Eq. (2) gives the N^-1 and the psi^-1 = psi^(q-2)
 *      inverse root, Eq. (3) the psi^-n post-twist of the negacyclic form)
 *   schoolbook product in Z_q[X]/(X^N+1), the ring named in Sec. II-A.
 * psi is a primitive 2N-th root of unity mod q (psi^N = -1).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static uint32_t mulmod(uint32_t a, uint32_t b, uint32_t q) {
    return (uint32_t)(((uint64_t)a * (uint64_t)b) % q);
}

uint32_t oracle_powmod(uint32_t base, uint64_t e, uint32_t q) {
    uint32_t r = 1 % q, b = base % q;
    while (e) {
        if (e & 1) r = mulmod(r, b, q);
        b = mulmod(b, b, q);
        e >>= 1;
    }
    return r;
}

/* Eq. (4) evaluated term by term: O(N^2). */
void oracle_ntt_brute(const uint32_t* a, uint32_t* A, int N, uint32_t q, uint32_t psi) {
    uint64_t two_n = 2ull * (uint64_t)N;
    for (int k = 0; k < N; k++) {
        uint64_t acc = 0;
        for (int n = 0; n < N; n++) {
            uint64_t e = ((2ull * (uint64_t)n * (uint64_t)k + (uint64_t)n) % two_n);
            acc = (acc + mulmod(a[n], oracle_powmod(psi, e, q), q)) % q;
        }
        A[k] = (uint32_t)acc;
    }
}

/* The inverse of Eq. (4), term by term: O(N^2). */
void oracle_intt_brute(const uint32_t* A, uint32_t* a, int N, uint32_t q, uint32_t psi) {
    uint64_t two_n = 2ull * (uint64_t)N;
    uint32_t psi_inv = oracle_powmod(psi, (uint64_t)q - 2, q);
    uint32_t n_inv = oracle_powmod((uint32_t)N % q, (uint64_t)q - 2, q);
    for (int n = 0; n < N; n++) {
        uint64_t acc = 0;
        for (int k = 0; k < N; k++) {
            uint64_t e = (2ull * (uint64_t)n * (uint64_t)k) % two_n;
            acc = (acc + mulmod(A[k], oracle_powmod(psi_inv, e, q), q)) % q;
        }
        acc = mulmod((uint32_t)acc, n_inv, q);
        a[n] = mulmod((uint32_t)acc, oracle_powmod(psi_inv, (uint64_t)n, q), q);
    }
}

/*
 * Textbook iterative radix-2 cyclic DFT over Z_q (decimation in time with an
 * explicit bit-reversal permutation first), natural order in and out:
 *   X_k = sum_n x_n * w^(nk) mod q,  w a primitive N-th root of unity.
 */
static void cyclic_dft(uint32_t* x, int N, uint32_t q, uint32_t w) {
    int logn = 0;
    while ((1 << logn) < N) logn++;
    for (int i = 0; i < N; i++) {
        int r = 0;
        for (int b = 0; b < logn; b++) r |= ((i >> b) & 1) << (logn - 1 - b);
        if (r > i) { uint32_t t = x[i]; x[i] = x[r]; x[r] = t; }
    }
    for (int len = 2; len <= N; len <<= 1) {
        uint32_t wl = oracle_powmod(w, (uint64_t)(N / len), q); /* primitive len-th root */
        for (int s = 0; s < N; s += len) {
            uint32_t wj = 1;
            for (int j = 0; j < len / 2; j++) {
                uint32_t u = x[s + j];
                uint32_t v = mulmod(x[s + j + len / 2], wj, q);
                x[s + j] = (uint32_t)(((uint64_t)u + v) % q);
                x[s + j + len / 2] = (uint32_t)(((uint64_t)u + q - v) % q);
                wj = mulmod(wj, wl, q);
            }
        }
    }
}

/*
 * Eq. (4) in O(N log N): A_k = sum_n (a_n psi^n) (psi^2)^(nk), i.e. a pre-twist
 * by psi^n followed by the cyclic DFT with the N-th root psi^2.
 */
void oracle_ntt(const uint32_t* a, uint32_t* A, int N, uint32_t q, uint32_t psi) {
    uint32_t t = 1;
    for (int n = 0; n < N; n++) { A[n] = mulmod(a[n] % q, t, q); t = mulmod(t, psi, q); }
    cyclic_dft(A, N, q, mulmod(psi, psi, q));
}

/* Inverse: cyclic DFT with root psi^-2, then scale by N^-1 psi^-n. */
void oracle_intt(const uint32_t* A, uint32_t* a, int N, uint32_t q, uint32_t psi) {
    uint32_t psi_inv = oracle_powmod(psi, (uint64_t)q - 2, q);
    uint32_t n_inv = oracle_powmod((uint32_t)N % q, (uint64_t)q - 2, q);
    for (int n = 0; n < N; n++) a[n] = A[n] % q;
    cyclic_dft(a, N, q, mulmod(psi_inv, psi_inv, q));
    uint32_t t = n_inv;
    for (int n = 0; n < N; n++) { a[n] = mulmod(a[n], t, q); t = mulmod(t, psi_inv, q); }
}

/* c = a*b in Z_q[X]/(X^N+1): X^N = -1 wraps the high half with a minus sign. */
void oracle_negacyclic_mul(const uint32_t* a, const uint32_t* b, uint32_t* c, int N, uint32_t q) {
    for (int k = 0; k < N; k++) {
        uint64_t acc = 0;
        for (int i = 0; i < N; i++) {
            int j = k - i;
            if (j >= 0) {
                acc = (acc + mulmod(a[i], b[j], q)) % q;
            } else {
                acc = (acc + q - mulmod(a[i], b[j + N], q)) % q;
            }
        }
        c[k] = (uint32_t)acc;
    }
}

/*
 * Batched transform over a (L, B, N) limb-major array (Sec. IV-D layout):
 * limb l uses q[l] and psi[l]. inverse != 0 selects the INTT. Parallel over
 * the L*B independent rows when built with OpenMP; threads <= 0 keeps the
 * runtime default. Returns the number of threads used.
 */
int oracle_ntt_batch(const uint32_t* in, uint32_t* out, int L, int B, int N,
                     const uint32_t* q, const uint32_t* psi, int inverse, int threads) {
    int used = 1;
    long rows = (long)L * (long)B;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel
    {
#pragma omp single
        used = omp_get_num_threads();
    }
#pragma omp parallel for schedule(dynamic, 1)
#else
    (void)threads;
#endif
    for (long r = 0; r < rows; r++) {
        int l = (int)(r / B);
        const uint32_t* src = in + (size_t)r * (size_t)N;
        uint32_t* dst = out + (size_t)r * (size_t)N;
        if (inverse) oracle_intt(src, dst, N, q[l], psi[l]);
        else oracle_ntt(src, dst, N, q[l], psi[l]);
    }
    return used;
}

// Basis conversion (Sec. IV-A, the Conv step of ModUp and ModDown) on the tcgen05 tensor cores.
//
// For coefficient n and destination modulus q_t:
//     dst_t[n] = sum_i y_i[n] c_{i,t} mod q_t,   y_i = [x_i (B/b_i)^-1]_{b_i},  c_{i,t} = [B/b_i]_{q_t}.
// Both factors are split into balanced base-256 digits, y_i = sum_j d_{ij} 256^j and
// [c_{i,t} 256^j]_{q_t} = sum_k e_{ijk} 256^k, so that
//     sum_i y_i c_{i,t} = sum_k 256^k acc_{t,k} (mod q_t),   acc_{t,k} = sum_{i,j} d_{ij} e_{ijk},
// a GEMM of the (coefficient x 4 nsrc) data digits with the (4 nsrc x 4 ndst) constant digits.
// |d e| <= 128 * 128 and 4 nsrc <= 60 terms keep every partial sum below 2^20, exact in the fp32
// accumulators; the digits are exact in fp16. The reconstruction stays in 32 bits: two
// shift-adds, then two Shoup products (by [2^16]_q and by 1) per output, where the CUDA-core
// conversion spends nsrc 64-bit multiply-adds and a 64-bit reduction.
//
// One CTA (4 warps) per 128 coefficients, persistent: each thread owns one coefficient (one A
// row, one TMEM lane). The data digits go straight from registers into tensor memory, which
// the MMA reads as its A operand (no shared-memory round trip and no proxy fence); the
// constant digits of this call's destinations are staged in shared memory once per CTA.
#include <algorithm>

#include "common.cuh"
#include "ptx.cuh"

namespace fhe {
namespace {

constexpr int kRows = 128;

__global__ void __launch_bounds__(128) tc_conv_kernel(const TcConvArgs a, int* status) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* Bs = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    __shared__ uint64_t done;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int nb = (4 * a.ndst + 15) & ~15;  // MMA N (multiple of 16)
    const int nk = (4 * a.nsrc + 15) / 16;   // K steps of 16
    const int acol = (nb + 31) & ~31;        // TMEM: D in columns [0, nb), A in [acol, acol + 8 nk)
    int ncols = 32;
    while (ncols < acol + 8 * nk) ncols *= 2;

    // constant digits: B row n = 4 t + k, reduction index K' = 4 i + j; 16-byte chunk c of a row
    // holds K' = 8 c .. 8 c + 7 and sits at position c ^ (n % 8)
    for (int idx = tid; idx < nb * 8; idx += kRows) {
        const int n = idx >> 3, c = idx & 7;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (n < 4 * a.ndst && c < 2 * nk)
            v = __ldg(reinterpret_cast<const uint4*>(a.bdig + ((size_t)a.dst_mod[n >> 2] * 4 + (n & 3)) * kConvKPad) + c);
        *reinterpret_cast<uint4*>(Bs + n * 128 + ((c ^ (n & 7)) << 4)) = v;
    }
    if (tid == 0) {
        ptx::mbar_init(&done, 1);
        ptx::fence_mbar_init();
    }
    if (warp == 0) {
        ptx::tmem_alloc(&tmem_base, ncols);
        ptx::tmem_relinquish();
    }
    ptx::fence_proxy_async();  // B is read by the MMA through the async proxy
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = ptx::idesc_f16(kRows, nb);
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    const size_t ntiles = (a.ncoef + kRows - 1) / kRows;

    // this thread's source residues of a tile, loaded one tile ahead
    uint32_t xv[16];
    auto load = [&](size_t tile) {
        const size_t n = tile * kRows + tid;
#pragma unroll
        for (int i = 0; i < 16; ++i)
            xv[i] = (i < a.nsrc && tile < ntiles && n < a.ncoef) ? __ldcs(&a.src[(size_t)i * a.src_stride + n]) : 0u;
    };
    load(blockIdx.x);
    int it = 0;
    bool ok = true;
    for (size_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
        const size_t n = tile * kRows + tid;
        const bool valid = n < a.ncoef;
        // A row (TMEM lane tid): digits of y_i, K' = 4 i + j, two fp16 per column; sources
        // 4 kk .. 4 kk + 3 fill the 8 columns read by MMA step kk
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            if (kk >= nk) break;
            uint32_t w[8];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int i = 4 * kk + h;
                const uint2 p = i < a.nsrc ? split_f16x4(mul_shoup(xv[i], a.hat_inv[i].x, a.hat_inv[i].y, a.src_q[i]))
                                           : make_uint2(0, 0);
                w[2 * h] = p.x;
                w[2 * h + 1] = p.y;
            }
            ptx::tmem_st8(lane_base + acol + 8 * kk, w);
        }
        ptx::tmem_wait_st();
        ptx::tc_fence_before();  // these stores and the previous tile's TMEM loads precede the MMA
        __syncthreads();
        if (tid == 0) {
            ptx::tc_fence_after();
            for (int kk = 0; kk < nk; ++kk)
                ptx::mma_f16_ts(tmem, tmem + acol + 8 * kk, ptx::sdesc_sw128(ptx::smem_u32(Bs) + kk * 32), idesc,
                                kk > 0 ? 1u : 0u);
            ptx::mma_commit(&done);
        }
        load(tile + gridDim.x);  // the next tile's sources travel while this one finishes
        ok = __syncthreads_and(ptx::mbar_wait(&done, (uint32_t)(it & 1), status, FHE_ETIMEOUT));
        if (!ok) break;
        ptx::tc_fence_after();
        // epilogue: 16 TMEM columns = 4 destinations x 4 digits per load
        for (int t0 = 0; t0 < a.ndst; t0 += 4) {
            uint32_t r[16];
            ptx::tmem_ld<16>(lane_base + 4 * t0, r);
            ptx::tmem_wait_ld();
            if (!valid) continue;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int t = t0 + u;
                if (t >= a.ndst) break;
                // |acc| < 2^20: adding 1.5 * 2^23 leaves acc in the low mantissa bits exactly
                int acc[4];
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    acc[k] = __float_as_int(__uint_as_float(r[4 * u + k]) + 12582912.0f) - 0x4B400000;
                // y = lo + 2^16 hi with |lo|, |hi| < 2^28; adding the multiple of q_t at or above 2^29
                // makes both positive, then y = lo + [2^16 hi]_q (mod q_t) stays below 2^32
                const uint32_t q = a.dst_q[t], off = a.dst_off[t];
                const uint32_t lo = (uint32_t)(acc[0] + acc[1] * 256) + off;
                const uint32_t hi = (uint32_t)(acc[2] + acc[3] * 256) + off;
                const uint32_t th = mul_shoup(hi, a.dst_c16[t].x, a.dst_c16[t].y, q);
                __stcs(&a.dst[(size_t)t * a.dst_stride + n], mul_shoup(lo + th, a.dst_one[t].x, a.dst_one[t].y, q));
            }
        }
    }
    // an MMA that did not complete in time must not be running when TMEM is released
    if (!ok && tid == 0) ptx::mbar_wait(&done, (uint32_t)(it & 1), nullptr, 0);
    ptx::tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        __syncwarp();
        ptx::tmem_dealloc(tmem, ncols);
    }
}

}  // namespace

int launch_conv_tc(const fhe_ctx* ctx, const TcConvArgs& a, cudaStream_t st) {
    if (a.nsrc < 1 || a.nsrc > 15 || a.ndst < 1 || a.ndst > 64 || !a.bdig)
        return set_error(FHE_EINVAL, "tensor-core Conv: 1..15 sources, 1..64 destinations");
    if (a.ncoef == 0) return FHE_OK;
    TcConvArgs b = a;
    for (int t = 0; t < a.ndst; ++t) {
        const uint32_t q = a.dst_q[t];
        const uint32_t c16 = (uint32_t)((1ull << 16) % q);
        b.dst_c16[t] = make_uint2(c16, shoup_h(c16, q));
        b.dst_one[t] = make_uint2(1u, shoup_h(1u, q));
        b.dst_off[t] = (uint32_t)((((1ull << 29) + q - 1) / q) * q);
    }
    const int nb = (4 * a.ndst + 15) & ~15, nk = (4 * a.nsrc + 15) / 16;
    int ncols = 32;
    while (ncols < ((nb + 31) & ~31) + 8 * nk) ncols *= 2;
    // CTAs per SM bounded by TMEM (512 columns) and at most 4; the shared-memory request keeps
    // the residency there so that no CTA waits for TMEM
    const int cps = std::min(4, 512 / ncols);
    const size_t need = (size_t)nb * 128 + 1024;  // the B tile, 1024-byte alignment
    const size_t smem = std::max(need, (size_t)(226 * 1024) / cps - 1024);
    FHE_CUDA_TRY(cudaFuncSetAttribute(tc_conv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const size_t ntiles = (a.ncoef + kRows - 1) / kRows;
    const size_t grid = std::min(ntiles, (size_t)ctx->num_sms * cps);
    tc_conv_kernel<<<(unsigned)grid, kRows, smem, st>>>(b, ctx->d_status);
    FHE_CUDA_TRY(cudaGetLastError());
    return FHE_OK;
}

}  // namespace fhe

// fhe_rescale_noalloc: RESCALE with library-owned, statically sized scratch.
//
// Some callers cannot call cudaMalloc: a serving loop that must not stall the device
// (cudaMalloc/cudaFree may synchronise it), code whose device memory is all owned by another
// allocator under a fixed budget (for example a framework's caching allocator), or a plugin
// host that forbids device allocations. For them this entry point runs the same rescale as
// fhe_rescale but takes its scratch from a fixed array that lives in this library's device
// image, so the call itself allocates nothing.
#include <mutex>

#include "common.cuh"

namespace {

// The scratch array. Every GPU that loads libfhe holds these bytes until the process exits.
// In host code `g_rescale_scratch` names a host-side stand-in, never the device memory: the
// device address is obtained with cudaGetSymbolAddress below.
static __device__ __align__(256) uint32_t g_rescale_scratch[FHE_RESCALE_NOALLOC_MAX_BYTES / 4];

std::mutex g_mu;
void* g_scratch_ptr[256];
bool g_scratch_ready[256];

// Looks up the scratch array's device address once per device, with that device current.
// The cached address belongs to the CUDA context in which it was looked up: it does not
// survive cudaDeviceReset (which also invalidates every fhe_ctx on that device).
int scratch_address(const fhe_ctx* ctx, void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fhe::cuda_error(e, "cudaGetDevice");
    if (dev < 0 || dev >= 256) return fhe::set_error(FHE_EINVAL, "device ordinal out of range");
    // the array is per device: the context's tables and the scratch must be on the same GPU
    if (dev != ctx->device)
        return fhe::set_error(FHE_EINVAL, "fhe_rescale_noalloc: the current device is not the context's device");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ready[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_rescale_scratch);
        if (e != cudaSuccess) return fhe::cuda_error(e, "cudaGetSymbolAddress(g_rescale_scratch)");
        g_scratch_ptr[dev] = p;
        g_scratch_ready[dev] = true;
    }
    *out = g_scratch_ptr[dev];
    return FHE_OK;
}

}  // namespace

extern "C" int fhe_rescale_noalloc(const fhe_ctx* ctx, uint32_t logN, int n_limbs, int batch,
                                   const uint32_t* ct_in, uint32_t* ct_out, void* stream) {
    if (ctx == nullptr) return fhe::set_error(FHE_EINVAL, "ctx is NULL");
    const size_t need = fhe_scratch_bytes(ctx, FHE_OP_RESCALE, logN, n_limbs, batch);
    if (need == 0 && batch != 0)
        return fhe::set_error(FHE_EINVAL, "invalid rescale arguments (logN, n_limbs or batch)");
    if (need > (size_t)FHE_RESCALE_NOALLOC_MAX_BYTES)
        return fhe::set_error(FHE_ENOMEM,
                              "fhe_rescale_noalloc: needs " + std::to_string(need) +
                                  " bytes of scratch, above the fixed FHE_RESCALE_NOALLOC_MAX_BYTES = " +
                                  std::to_string((size_t)FHE_RESCALE_NOALLOC_MAX_BYTES) +
                                  "; use fhe_rescale with caller-provided scratch");
    void* scratch = nullptr;
    int rc = scratch_address(ctx, &scratch);
    if (rc) return rc;
    // The rescale overwrites every scratch word it reads, so nothing needs clearing first.
    return fhe_rescale(ctx, logN, n_limbs, batch, ct_in, ct_out, scratch, need, stream);
}

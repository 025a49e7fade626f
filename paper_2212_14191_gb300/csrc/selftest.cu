// Self-test of the device-side failure path. Every spin-wait in this library is bounded: when
// its limit passes it records FHE_ETIMEOUT in the context's device error word and lets the
// kernel finish, so the context stays usable and fhe_device_status reports the failure. The
// kernel here waits on an mbarrier that nothing ever arrives at, with the caller's cycle
// limit, so that path can be checked on a GPU without faulting or hanging it.
#include "common.cuh"
#include "ptx.cuh"

namespace fhe {
namespace {

__global__ void k_wait_never(int* status, long long limit) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        ptx::mbar_init(&bar, 1);
        ptx::fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const long long t0 = clock64();
        while (!ptx::mbar_try_wait(&bar, 0)) {
            if (clock64() - t0 > limit) {
                atomicCAS(status, 0, FHE_ETIMEOUT);
                break;
            }
        }
    }
}

}  // namespace
}  // namespace fhe

using namespace fhe;

extern "C" int fhe_selftest_wait_timeout(const fhe_ctx* ctx, long long limit_cycles, void* stream) {
    FHE_CHECK(ctx != nullptr, "ctx is NULL");
    FHE_CHECK(limit_cycles > 0 && limit_cycles <= 4000000000LL, "limit_cycles out of (0, 4e9]");
    k_wait_never<<<1, 32, 0, (cudaStream_t)stream>>>(ctx->d_status, limit_cycles);
    FHE_CUDA_TRY(cudaGetLastError());
    return FHE_OK;
}

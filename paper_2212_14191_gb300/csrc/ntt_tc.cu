// Tensor-core NTT path (Sec. IV-C): see the kernels below.
#include "common.cuh"

namespace fhe {

int build_tc_tables(fhe_ctx* ctx, uint32_t logN) {
    (void)ctx;
    (void)logN;
    return FHE_OK;
}

int ntt_tc(const fhe_ctx* ctx, uint32_t logN, bool inverse, uint32_t* d, int n_limbs, int batch,
           const LimbMap& map, cudaStream_t stream) {
    (void)ctx; (void)logN; (void)inverse; (void)d; (void)n_limbs; (void)batch; (void)map; (void)stream;
    return set_error(FHE_EINVAL, "tensor-core NTT path not available in this build");
}

}  // namespace fhe

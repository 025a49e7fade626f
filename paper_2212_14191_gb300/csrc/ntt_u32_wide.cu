// Plain 32-bit NTT / INTT: instantiation and dispatch of the shapes whose clusters have four
// or more CTAs (N = 2^16 with 512 threads per CTA, N = 2^15 and 2^16 with 256).
#include "ntt_u32_kernels.cuh"

namespace fhe {

int ntt_u32_launch_wide(const fhe_ctx* ctx, const NttTables& t, uint32_t logN, int log_t, int log_c, int v,
                        bool inverse, uint32_t* d, int rows, int batch, const LimbMap& map, const RowRef* rowtab,
                        cudaStream_t stream, NttScratch scr) {
    FHE_NTT_CASE(9, 2)
    FHE_NTT_CASE(8, 2)
    FHE_NTT_CASE(8, 3)
    return set_error(FHE_EINVAL, "no kernel for this NTT shape");
}

}  // namespace fhe

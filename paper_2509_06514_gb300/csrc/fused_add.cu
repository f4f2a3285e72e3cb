// fused_add.cu — instantiations of the fused kernel for the additive answer over Z_2^32
// (qc queries per warp tile, 1 or 2, 2 for records up to 2 KiB; nk uint4 words per lane per record).
#include "fused.cuh"

namespace impir {

cudaError_t launch_fused_add(uint32_t qc, uint32_t nk, dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                             const FusedParams& p) {
    switch (qc * 16 + nk) {
        case 1 * 16 + 1: return launch_fused_t<1, 1, 1>(grid, block, smem, s, p);
        case 1 * 16 + 2: return launch_fused_t<1, 2, 1>(grid, block, smem, s, p);
        case 1 * 16 + 4: return launch_fused_t<1, 4, 1>(grid, block, smem, s, p);
        case 1 * 16 + 8: return launch_fused_t<1, 8, 1>(grid, block, smem, s, p);
        case 2 * 16 + 1: return launch_fused_t<2, 1, 1>(grid, block, smem, s, p);
        case 2 * 16 + 2: return launch_fused_t<2, 2, 1>(grid, block, smem, s, p);
        case 2 * 16 + 4: return launch_fused_t<2, 4, 1>(grid, block, smem, s, p);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace impir

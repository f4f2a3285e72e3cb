// fused_q8.cu — instantiations of the fused EvalAll + dpXOR kernel for 8 queries per warp.
#include "fused.cuh"

namespace impir {

cudaError_t launch_fused_q8(uint32_t nk, dim3 grid, dim3 block, size_t smem, cudaStream_t s, const FusedParams& p) {
    switch (nk) {
        case 1: return launch_fused_t<8, 1>(grid, block, smem, s, p);
        case 2: return launch_fused_t<8, 2>(grid, block, smem, s, p);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t prepare_fused_q8() {
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = prepare_fused_t<8, 1>();
    if (e == cudaSuccess) e = prepare_fused_t<8, 2>();
    return e;
}

}  // namespace impir

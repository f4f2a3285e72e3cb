// fused_q2.cu — instantiations of the fused EvalAll + dpXOR kernel for 2 queries per warp.
#include "fused.cuh"

namespace impir {

cudaError_t launch_fused_q2(uint32_t nk, dim3 grid, dim3 block, size_t smem, cudaStream_t s, const FusedParams& p) {
    switch (nk) {
        case 1: return launch_fused_t<2, 1>(grid, block, smem, s, p);
        case 2: return launch_fused_t<2, 2>(grid, block, smem, s, p);
        case 4: return launch_fused_t<2, 4>(grid, block, smem, s, p);
        case 8: return launch_fused_t<2, 8>(grid, block, smem, s, p);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t prepare_fused_q2() {
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = prepare_fused_t<2, 1>();
    if (e == cudaSuccess) e = prepare_fused_t<2, 2>();
    if (e == cudaSuccess) e = prepare_fused_t<2, 4>();
    if (e == cudaSuccess) e = prepare_fused_t<2, 8>();
    return e;
}

}  // namespace impir

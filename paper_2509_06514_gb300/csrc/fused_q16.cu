// fused_q16.cu — instantiations of the fused EvalAll + dpXOR kernel for 16 queries per warp
// (records of at most 512 bytes: one uint4 accumulator per query per lane).
#include "fused.cuh"

namespace impir {

cudaError_t launch_fused_q16(uint32_t nk, dim3 grid, dim3 block, size_t smem, cudaStream_t s, const FusedParams& p) {
    switch (nk) {
        case 1: return launch_fused_t<16, 1>(grid, block, smem, s, p);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t prepare_fused_q16() {
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = prepare_fused_t<16, 1>();
    return e;
}

}  // namespace impir

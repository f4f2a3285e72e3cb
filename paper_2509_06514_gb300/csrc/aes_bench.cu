// aes_bench.cu — AES-only calibration kernel: the fused kernel's PRF engine with nothing
// around it (no tree walk, no stack, no scan). Each thread iterates the node expansion of
// Eq. (3) with zero correction words, p <- PRF_p(0) XOR PRF_p(1), in registers, so the
// measured rate is the ceiling of the T-table AES engine on this GPU; the final states let
// a test check the engine against an independent AES.
#include "../../include/impir.h"
#include "fused.cuh"

namespace impir {

impir_status set_error(impir_status st, const char* msg);

namespace {

template <int PRF>
__global__ void __launch_bounds__(512, 1) aes_bench_kernel(const __grid_constant__ FusedParams P, const uint4* seeds,
                                                           uint4* out, uint32_t iters, uint32_t n_threads) {
    const uint32_t tid = threadIdx.x, nthr = blockDim.x;
#ifdef IMPIR_BOUNDS
    if (tid == 0) s_bctx = BoundsCtx{P.bounds, nullptr, nullptr, 0, nullptr, 0, kTableBytes, 0};
#endif
    for (uint32_t i = tid; i < 256 * 32; i += nthr) {
        const uint32_t x = i >> 5, l = i & 31;
        const uint32_t t0 = __ldg(P.te0 + x);
        uint32_t* ra = reinterpret_cast<uint32_t*>(g_smem + x * 256);
        uint32_t* rb = reinterpret_cast<uint32_t*>(g_smem + 65536 + x * 256);
        ra[l] = t0;
        ra[32 + l] = __funnelshift_l(t0, t0, 8);
        rb[l] = __funnelshift_l(t0, t0, 16);
        rb[32 + l] = __funnelshift_l(t0, t0, 24);
    }
    __syncthreads();
    const uint32_t g = blockIdx.x * blockDim.x + tid;
    if (g >= n_threads) return;
    const uint32_t L = (tid & 31) * 4;
    const uint4 s0 = seeds[g];
    Blk p{s0.x, s0.y, s0.z, s0.w};
    const Blk zero{0, 0, 0, 0};
    for (uint32_t it = 0; it < iters; ++it) {
        Blk a, b;
        if (PRF == 0)
            keyed_pair(p, L, zero, zero, a, b);
        else
            mmo_pair(p, L, P.mmo_rk, zero, zero, a, b);
        p = bxor(a, b);
    }
    out[g] = make_uint4(p.x, p.y, p.z, p.w);
}

}  // namespace
}  // namespace impir

using namespace impir;

extern "C" impir_status impir_aes_calibrate(int prf, uint32_t iters, uint32_t n_threads, uint32_t threads_per_cta,
                                            const uint8_t* seeds, uint8_t* out, double* ms) {
    if (!seeds || !out || !ms || (prf != 0 && prf != 1) || n_threads == 0 || threads_per_cta == 0 ||
        threads_per_cta > 512 || threads_per_cta % 32)
        return set_error(IMPIR_EINVAL, "bad calibration arguments");
    uint32_t te0[256];
    host_aes_te0(te0);
    FusedParams fp{};
    host_aes_expand(reinterpret_cast<const uint8_t*>(IMPIR_MMO_KEY0), fp.mmo_rk[0]);
    host_aes_expand(reinterpret_cast<const uint8_t*>(IMPIR_MMO_KEY1), fp.mmo_rk[1]);
    uint32_t* d_te0 = nullptr;
    uint4 *d_seeds = nullptr, *d_out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    impir_status st = IMPIR_OK;
    const size_t nb = size_t(n_threads) * 16;
    cudaError_t e = cudaMalloc(&d_te0, sizeof te0);
    if (e == cudaSuccess) e = cudaMalloc(&d_seeds, nb);
    if (e == cudaSuccess) e = cudaMalloc(&d_out, nb);
    if (e == cudaSuccess) e = cudaMemcpy(d_te0, te0, sizeof te0, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_seeds, seeds, nb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        fp.te0 = d_te0;
        fp.bounds = bounds_record();
        const unsigned blocks = (n_threads + threads_per_cta - 1) / threads_per_cta;
        auto k = prf == 0 ? aes_bench_kernel<0> : aes_bench_kernel<1>;
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kTableBytes));
        if (e == cudaSuccess) {
            k<<<blocks, threads_per_cta, kTableBytes>>>(fp, d_seeds, d_out, 1, n_threads);  // warm-up
            e = cudaEventRecord(e0);
        }
        if (e == cudaSuccess) {
            k<<<blocks, threads_per_cta, kTableBytes>>>(fp, d_seeds, d_out, iters, n_threads);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float f = 0;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&f, e0, e1);
        *ms = f;
        if (e == cudaSuccess) e = cudaMemcpy(out, d_out, nb, cudaMemcpyDeviceToHost);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        st = set_error(IMPIR_ECUDA, cudaGetErrorString(e));
    }
    cudaFree(d_te0);
    cudaFree(d_seeds);
    cudaFree(d_out);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return st;
}

// aes_bench.cu — AES-only calibration kernels: the fused kernel's PRF engine with nothing
// around it (no tree walk, no stack, no scan), and a bitsliced engine to compare it with. Each
// thread iterates the node expansion of Eq. (3) with zero correction words,
// p <- PRF_p(0) XOR PRF_p(1), in registers, so the measured rate is the ceiling of each AES
// engine on this GPU; the final states let a test check the engines against an independent AES.
//
// The bitsliced engine computes the fixed-key PRF (Matyas-Meyer-Oseas, PRF_p(x) = AES_{K_x}(p)
// XOR p) on bit-slices: word 8b + i of a thread's 128-word state holds bit i of byte b of 16
// seeds in bits 0..15 (encrypted under K_0) and of the same 16 seeds in bits 16..31 (under
// K_1), so one 32-bit logic operation advances 32 AES computations. The round keys are
// per-slice masks in constant memory; SubBytes is the generated S-box circuit (bs_sbox.cuh);
// ShiftRows is folded into the order SubBytes writes its outputs; MixColumns is
// out_r = a_r ^ t ^ xtime(a_r ^ a_(r+1)) with t = a_0 ^ a_1 ^ a_2 ^ a_3 (FIPS-197 §5.1.3), where
// xtime on bit-slices is a rotation of the eight slices with the top slice folded into bits
// 1, 3 and 4. One iteration ends with p <- AES_K0(p) ^ AES_K1(p) (the two p terms cancel): each
// slice's halves XORed and copied to both halves. The keyed PRF cannot be bitsliced this way:
// its AES key is the node seed itself, so each instance needs its own key schedule, another
// 128 words of slices per thread beyond the registers a thread has.
#include "../../include/impir.h"
#include "bs_sbox.cuh"
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

// Round keys of K_0 and K_1 as slice masks: word [r][8b + i] has bits 0..15 set if bit i of byte
// b of K_0's round key r is 1, and bits 16..31 set if K_1's is.
__constant__ uint32_t c_bs_rk[11][128];

// SubBytes and ShiftRows: byte r + 4c receives S(byte r + 4((c + r) mod 4)). Row 0 stays in
// place; each other row is a cycle (rows 1 and 3) or two swaps (row 2), followed with one byte
// of slices held aside.
__device__ __forceinline__ void bs_sub_shift(uint32_t (&s)[128]) {
#define BS_S(dst, src)                                                                                       \
    IMPIR_BS_SBOX(s[8 * (src)], s[8 * (src) + 1], s[8 * (src) + 2], s[8 * (src) + 3], s[8 * (src) + 4],        \
                  s[8 * (src) + 5], s[8 * (src) + 6], s[8 * (src) + 7], dst[0], dst[1], dst[2], dst[3], dst[4], \
                  dst[5], dst[6], dst[7])
    uint32_t t[8];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        uint32_t* d = &s[8 * (4 * c)];
        BS_S(d, 4 * c);
    }
    // row 1: 1 <- 5 <- 9 <- 13 <- 1
    BS_S(t, 1);
    {
        uint32_t* d = &s[8 * 1];
        BS_S(d, 5);
    }
    {
        uint32_t* d = &s[8 * 5];
        BS_S(d, 9);
    }
    {
        uint32_t* d = &s[8 * 9];
        BS_S(d, 13);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) s[8 * 13 + i] = t[i];
    // row 2: 2 <-> 10, 6 <-> 14
    BS_S(t, 2);
    {
        uint32_t* d = &s[8 * 2];
        BS_S(d, 10);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) s[8 * 10 + i] = t[i];
    BS_S(t, 6);
    {
        uint32_t* d = &s[8 * 6];
        BS_S(d, 14);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) s[8 * 14 + i] = t[i];
    // row 3: 3 <- 15 <- 11 <- 7 <- 3
    BS_S(t, 15);
    {
        uint32_t* d = &s[8 * 15];
        BS_S(d, 11);
    }
    {
        uint32_t* d = &s[8 * 11];
        BS_S(d, 7);
    }
    {
        uint32_t* d = &s[8 * 7];
        BS_S(d, 3);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) s[8 * 3 + i] = t[i];
#undef BS_S
}

// MixColumns and AddRoundKey, column by column in place.
__device__ __forceinline__ void bs_mix_add(uint32_t (&s)[128], int r) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        uint32_t a[4][8], t[8];
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int i = 0; i < 8; ++i) a[q][i] = s[8 * (4 * c + q) + i];
#pragma unroll
        for (int i = 0; i < 8; ++i) t[i] = a[0][i] ^ a[1][i] ^ a[2][i] ^ a[3][i];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint32_t u[8], x[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) u[i] = a[q][i] ^ a[(q + 1) & 3][i];
            // xtime(u): multiply by {02} modulo x^8 + x^4 + x^3 + x + 1
            x[0] = u[7];
            x[1] = u[0] ^ u[7];
            x[2] = u[1];
            x[3] = u[2] ^ u[7];
            x[4] = u[3] ^ u[7];
            x[5] = u[4];
            x[6] = u[5];
            x[7] = u[6];
#pragma unroll
            for (int i = 0; i < 8; ++i) s[8 * (4 * c + q) + i] = a[q][i] ^ t[i] ^ x[i] ^ c_bs_rk[r][8 * (4 * c + q) + i];
        }
    }
}

__global__ void __launch_bounds__(256, 1) aes_bs_kernel(const uint4* seeds, uint4* out, uint32_t iters,
                                                         uint32_t n_threads) {
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_threads) return;
    uint32_t s[128];
#pragma unroll
    for (int k = 0; k < 128; ++k) s[k] = 0;
    // 16 seeds into slices, in both halves
    for (int j = 0; j < 16; ++j) {
        const uint4 v = seeds[size_t(g) * 16 + j];
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < 128; ++k) s[k] |= ((w[k >> 5] >> (k & 31)) & 1u) * (0x10001u << j);
    }
    for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 128; ++k) s[k] ^= c_bs_rk[0][k];
#pragma unroll 1
        for (int r = 1; r <= 9; ++r) {
            bs_sub_shift(s);
            bs_mix_add(s, r);
        }
        bs_sub_shift(s);
#pragma unroll
        for (int k = 0; k < 128; ++k) s[k] ^= c_bs_rk[10][k];
        // p <- AES_K0(p) ^ AES_K1(p) in both halves
#pragma unroll
        for (int k = 0; k < 128; ++k) s[k] ^= __byte_perm(s[k], 0, 0x1032);
    }
    for (int j = 0; j < 16; ++j) {
        uint32_t w[4] = {0, 0, 0, 0};
#pragma unroll
        for (int k = 0; k < 128; ++k) w[k >> 5] |= ((s[k] >> j) & 1u) << (k & 31);
        out[size_t(g) * 16 + j] = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

}  // namespace
}  // namespace impir

using namespace impir;

extern "C" impir_status impir_aes_calibrate_bitsliced(uint32_t iters, uint32_t n_threads, uint32_t threads_per_cta,
                                                      const uint8_t* seeds, uint8_t* out, double* ms) {
    if (!seeds || !out || !ms || n_threads == 0 || threads_per_cta == 0 || threads_per_cta > 256 ||
        threads_per_cta % 32)
        return set_error(IMPIR_EINVAL, "bad calibration arguments");
    // round-key slice masks of K_0 (bits 0..15) and K_1 (bits 16..31)
    uint32_t rk[2][44], masks[11][128];
    host_aes_expand(reinterpret_cast<const uint8_t*>(IMPIR_MMO_KEY0), rk[0]);
    host_aes_expand(reinterpret_cast<const uint8_t*>(IMPIR_MMO_KEY1), rk[1]);
    for (int r = 0; r < 11; ++r)
        for (int k = 0; k < 128; ++k) {
            const int b = k >> 3, i = k & 7;  // byte b = column b / 4, row b % 4
            uint32_t m = 0;
            for (int x = 0; x < 2; ++x)
                if ((rk[x][4 * r + (b >> 2)] >> (8 * (b & 3) + i)) & 1u) m |= x ? 0xffff0000u : 0x0000ffffu;
            masks[r][k] = m;
        }
    uint4 *d_seeds = nullptr, *d_out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    impir_status st = IMPIR_OK;
    const size_t nb = size_t(n_threads) * 16 * 16;
    cudaError_t e = cudaMemcpyToSymbol(c_bs_rk, masks, sizeof masks);
    if (e == cudaSuccess) e = cudaMalloc(&d_seeds, nb);
    if (e == cudaSuccess) e = cudaMalloc(&d_out, nb);
    if (e == cudaSuccess) e = cudaMemcpy(d_seeds, seeds, nb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        const unsigned blocks = (n_threads + threads_per_cta - 1) / threads_per_cta;
        aes_bs_kernel<<<blocks, threads_per_cta>>>(d_seeds, d_out, 1, n_threads);  // warm-up
        e = cudaEventRecord(e0);
        if (e == cudaSuccess) {
            aes_bs_kernel<<<blocks, threads_per_cta>>>(d_seeds, d_out, iters, n_threads);
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
    cudaFree(d_seeds);
    cudaFree(d_out);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return st;
}

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

// combine.cu — combines the partial answers of the row shards of a database (each shard's
// answer covers only its rows): the XOR of the parts for the XOR answer (the reconstruction
// by XOR of §2.3, applied to partial results as in Algorithm 1's aggregation), or their
// sum mod 2^32 word by word for the additive answer.
#include "../../include/impir.h"
#include "impir_internal.h"

namespace impir {

impir_status set_error(impir_status st, const char* msg);

namespace {

// out[i] = op over p of parts[p * n + i], 16-byte words
template <int MODE>
__global__ void combine16_kernel(const uint4* __restrict__ parts, uint32_t n_parts, size_t n, uint4* __restrict__ out) {
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
        uint4 a = parts[i];
        for (uint32_t p = 1; p < n_parts; ++p) {
            const uint4 b = parts[size_t(p) * n + i];
            if (MODE == 0) {
                a.x ^= b.x; a.y ^= b.y; a.z ^= b.z; a.w ^= b.w;
            } else {
                a.x += b.x; a.y += b.y; a.z += b.z; a.w += b.w;
            }
        }
        out[i] = a;
    }
}

// the same over 32-bit words (additive answer) or bytes (XOR answer) for unaligned sizes
__global__ void combine4_add_kernel(const uint32_t* __restrict__ parts, uint32_t n_parts, size_t n,
                                    uint32_t* __restrict__ out) {
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
        uint32_t a = parts[i];
        for (uint32_t p = 1; p < n_parts; ++p) a += parts[size_t(p) * n + i];
        out[i] = a;
    }
}

__global__ void combine1_xor_kernel(const uint8_t* __restrict__ parts, uint32_t n_parts, size_t n,
                                    uint8_t* __restrict__ out) {
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
        uint8_t a = parts[i];
        for (uint32_t p = 1; p < n_parts; ++p) a ^= parts[size_t(p) * n + i];
        out[i] = a;
    }
}

unsigned blocks_for(size_t n) { return unsigned(n / 256 + 1 < 4096 ? n / 256 + 1 : 4096); }

}  // namespace
}  // namespace impir

using namespace impir;

extern "C" impir_status impir_combine_partials(int mode, const uint8_t* d_parts, uint32_t n_parts, uint64_t part_bytes,
                                               uint8_t* d_out, void* cuda_stream) {
    if (mode != 0 && mode != 1) return set_error(IMPIR_EINVAL, "mode must be 0 (XOR) or 1 (sum mod 2^32)");
    if (!d_parts || !d_out || n_parts == 0) return set_error(IMPIR_EINVAL, "NULL buffer or no parts");
    if (part_bytes == 0) return IMPIR_OK;
    const uintptr_t pa = reinterpret_cast<uintptr_t>(d_parts), po = reinterpret_cast<uintptr_t>(d_out);
    const uint64_t span = uint64_t(n_parts) * part_bytes;
    if (po < pa + span && pa < po + part_bytes) return set_error(IMPIR_EINVAL, "d_out overlaps d_parts");
    if (mode == 1 && (part_bytes % 4 || (pa & 3) || (po & 3)))
        return set_error(IMPIR_EINVAL, "the additive combine needs 4-byte aligned buffers and sizes");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (part_bytes % 16 == 0 && (pa & 15) == 0 && (po & 15) == 0) {
        const size_t n = part_bytes / 16;
        if (mode == 0)
            combine16_kernel<0><<<blocks_for(n), 256, 0, st>>>(reinterpret_cast<const uint4*>(d_parts), n_parts, n,
                                                              reinterpret_cast<uint4*>(d_out));
        else
            combine16_kernel<1><<<blocks_for(n), 256, 0, st>>>(reinterpret_cast<const uint4*>(d_parts), n_parts, n,
                                                              reinterpret_cast<uint4*>(d_out));
    } else if (mode == 1) {
        const size_t n = part_bytes / 4;
        combine4_add_kernel<<<blocks_for(n), 256, 0, st>>>(reinterpret_cast<const uint32_t*>(d_parts), n_parts, n,
                                                          reinterpret_cast<uint32_t*>(d_out));
    } else {
        combine1_xor_kernel<<<blocks_for(part_bytes), 256, 0, st>>>(d_parts, n_parts, part_bytes, d_out);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(IMPIR_ECUDA, cudaGetErrorString(e));
    return IMPIR_OK;
}

// impir_internal.h — types shared by the host runtime and the CUDA kernels of libimpir.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace impir {

constexpr uint32_t kMaxDomainBits = 40;
constexpr uint32_t kMaxLaneBits = 10;     // 2^10 leaves per lane at most
constexpr uint32_t kMaxSegments = 48;     // one per distinct domain size (<= 41) + slack
constexpr uint32_t kTableBytes = 128 * 1024;

// Largest byte count of a database, a workspace or an answer buffer the library accepts
// (1 PiB): products of record counts and strides are checked against it before any
// allocation or launch, so they never wrap.
constexpr uint64_t kMaxBytes = 1ull << 50;
inline bool bytes_ok(uint64_t count, uint64_t unit) { return unit == 0 || count <= kMaxBytes / unit; }

// Workspace header at the start of the device workspace (256 bytes).
struct WsHeader {
    unsigned long long counter;   // next work unit to hand out
    unsigned long long n_units;   // total work units of this launch
    uint32_t n_bad;               // malformed keys seen by the setup kernel
    uint32_t first_bad;           // smallest malformed query index (UINT32_MAX if none)
    uint32_t n_groups;
    uint32_t n_segs;
    uint32_t pad[56];
};
static_assert(sizeof(WsHeader) == 256, "header is 256 bytes");

// A group of up to queries_per_warp queries with one domain size, evaluated together on
// a warp tile and scanned once: [first, first + count) indexes the sorted query list.
struct GroupDesc {
    uint32_t first;
    uint32_t count;
    uint32_t m;
    uint32_t pad;
};

// Work units u in [unit_lo, next segment's unit_lo) cover warp tiles
// tile_lo + (u - unit_lo) / count with groups (u - unit_lo) % count.
struct SegDesc {
    unsigned long long tile_lo;
    unsigned long long unit_lo;
    uint32_t count;
    uint32_t pad;
    unsigned long long pad2;
};
static_assert(sizeof(SegDesc) == 32, "segment descriptors are 32 bytes");
constexpr uint32_t kSegSmemBytes = kMaxSegments * sizeof(SegDesc);

struct WsLayout {
    size_t off_perm, off_qm, off_groups, off_segs, off_acc, total;
};

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

inline WsLayout ws_layout(uint32_t n_queries, uint32_t stride_bytes) {
    WsLayout L;
    size_t o = sizeof(WsHeader);
    L.off_perm = o;
    o = align256(o + size_t(n_queries) * 4);
    L.off_qm = o;
    o = align256(o + size_t(n_queries) * 4);
    L.off_groups = o;
    o = align256(o + (size_t(n_queries) + kMaxDomainBits + 8) * sizeof(GroupDesc));
    L.off_segs = o;
    o = align256(o + kMaxSegments * sizeof(SegDesc));
    L.off_acc = o;
    o = align256(o + size_t(n_queries) * stride_bytes);
    L.total = o;
    return L;
}

struct SetupParams {
    const uint8_t* keys;
    const uint32_t* key_off;
    uint8_t* ws;
    WsLayout lay;
    uint64_t n_records;
    uint32_t n_queries;
    uint32_t words;          // stride / 16
    uint32_t lane_bits;
    uint32_t qpw;            // queries per warp (group size)
    // A chunk of a streamed database or a row shard: only warp tiles in [tile_lo, tile_hi)
    // are scheduled (tile_hi == 0: no upper limit), and keep_acc != 0 keeps the accumulators
    // of the previous chunks instead of zeroing them. Zero values give the whole-database
    // launch.
    unsigned long long tile_lo, tile_hi;
    uint32_t keep_acc;
};

struct FusedParams {
    const uint4* db;
    const uint8_t* keys;
    const uint32_t* key_off;
    uint8_t* ws;
    const uint32_t* te0;     // 256-entry AES T-table (global memory), see host_aes.cpp
    WsLayout lay;
    uint64_t n_records;
    uint32_t n_queries;
    uint32_t words;          // uint4 words per record (stride / 16)
    uint32_t lane_bits;
    uint32_t bits_words;     // 32-bit words of selection bits (additive: shares) per (warp, query slot)
    uint32_t mmo_rk[2][44];  // round keys of the fixed MMO keys K_0, K_1
    unsigned long long rec_lo;  // global index of the record at db[0] (0 unless a chunk or a row shard)
};

struct FinalizeParams {
    const uint8_t* ws;
    WsLayout lay;
    uint8_t* out;
    uint32_t n_queries;
    uint32_t record_bytes;
    uint32_t stride;
};

// Kernel launchers (defined in the .cu files).
cudaError_t launch_setup(const SetupParams& p, cudaStream_t s);
cudaError_t launch_finalize(const FinalizeParams& p, cudaStream_t s);
// qpw in {1,2,4,8,16}, nk in {1,2,4,8} with qpw * nk <= 16.
cudaError_t launch_fused(uint32_t qpw, uint32_t nk, dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                         const FusedParams& p);
cudaError_t launch_fused_q1(uint32_t nk, dim3 grid, dim3 block, size_t smem, cudaStream_t s, const FusedParams& p);
cudaError_t launch_fused_q2(uint32_t nk, dim3 grid, dim3 block, size_t smem, cudaStream_t s, const FusedParams& p);
cudaError_t launch_fused_q4(uint32_t nk, dim3 grid, dim3 block, size_t smem, cudaStream_t s, const FusedParams& p);
cudaError_t launch_fused_add(uint32_t qc, uint32_t nk, dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                             const FusedParams& p);
cudaError_t launch_fused_q16(uint32_t nk, dim3 grid, dim3 block, size_t smem, cudaStream_t s, const FusedParams& p);
cudaError_t launch_fused_q8(uint32_t nk, dim3 grid, dim3 block, size_t smem, cudaStream_t s, const FusedParams& p);

// Host AES pieces of the product (independent of the oracle): T-table and key schedule.
void host_aes_te0(uint32_t te0[256]);
void host_aes_expand(const uint8_t key[16], uint32_t rk[44]);
void host_aes_encrypt(const uint32_t rk[44], const uint8_t in[16], uint8_t out[16]);

}  // namespace impir

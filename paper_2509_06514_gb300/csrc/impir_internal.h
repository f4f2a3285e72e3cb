// impir_internal.h — types shared by the host runtime and the CUDA kernels of libimpir.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/impir.h"

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
    uint32_t bounds_failed;       // failed index checks of this launch (debug build only)
    uint32_t pad[55];
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

// Failed index checks of the debug build (compiled with IMPIR_BOUNDS), one record per device:
// how many failed since the record was last cleared, and the site and index of the first.
struct BoundsRecord {
    unsigned int n_failed;
    unsigned int first_site;
    unsigned long long first_index;
};

// Site codes of the index checks.
enum BoundsSite : uint32_t {
    kSiteTable = 1,      // T-table offset in shared memory
    kSiteBits = 2,       // selection-bit / node / share buffer in shared memory
    kSiteRecord = 3,     // database word
    kSiteKey = 4,        // key byte (inside the key, and inside the key buffer when its size is known)
    kSiteQuery = 5,      // query index (sorted permutation, key offsets)
    kSiteSchedule = 6,   // group or segment index
    kSiteAcc = 7,        // accumulator word
    kSiteStack = 8,      // a lane's stack of pending right children
    kSiteWorkspace = 9,  // schedule written by the setup kernel
    kSiteOut = 10,       // answer byte
};

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

// ---- launch shape of the XOR answer (shared by every answer path) ----

constexpr size_t kSmemMax = 227 * 1024;

// uint4 words per lane and pass that cover a record in one pass (1, 2, 4 or 8)
inline uint32_t nk_need(uint32_t words) {
    if (words <= 32) return 1;
    const uint32_t need = (words + 31) / 32;
    return need <= 2 ? 2 : need <= 4 ? 4 : 8;
}

// uint4 words per lane and pass of the XOR scan for qpw queries per warp: records above 512 B
// are scanned in column passes of nk words per lane, with qpw * nk <= 16 accumulators per lane,
// so that more queries share every tile read (records of 1 KiB: one pass at 8 queries per warp;
// 4 KiB: four)
inline uint32_t nk_xor(uint32_t words, uint32_t qpw) {
    if (words <= 32) return 1;
    return std::min(nk_need(words), std::max(2u, 16u / qpw));
}

// Widest CTA the fused kernel is built for (its launch bounds): 20 warps for the XOR answer
// with one column pass (records of at most 512 bytes) and at most 8 queries per warp, else 16.
inline uint32_t max_warps(uint32_t qpw, uint32_t words) { return nk_need(words) == 1 && qpw <= 8 ? 20u : 16u; }

// Dynamic shared memory of the XOR kernels: T-tables, segment table, per-warp selection bits.
inline size_t smem_for(const impir_config& c) {
    return kTableBytes + kSegSmemBytes + size_t(c.warps_per_cta) * c.queries_per_warp * (size_t(1) << c.lane_bits) * 4;
}

// Largest lane_bits that keeps enough warp tiles for every warp of the grid busy.
inline impir_config default_config_warps(uint64_t n_records, uint32_t words, uint32_t n_queries, int sms,
                                         uint32_t warps) {
    impir_config c{};
    c.warps_per_cta = warps;
    c.queries_per_launch = 0;
    uint32_t qpw = 8;
    while (qpw > 1 && (qpw * nk_xor(words, qpw) > 16 || qpw > n_queries)) qpw >>= 1;
    c.queries_per_warp = qpw;
    const double all_warps = double(sms) * c.warps_per_cta;
    const double groups = std::ceil(double(n_queries) / qpw);
    c.lane_bits = 0;
    for (uint32_t s = kMaxLaneBits; s + 1 > 0; --s) {
        impir_config t = c;
        t.lane_bits = s;
        if (smem_for(t) > kSmemMax) continue;
        const double tiles = std::ceil(double(n_records) / double(32ull << s));
        if (groups * tiles >= 3.0 * all_warps || s == 0) {
            c.lane_bits = s;
            break;
        }
    }
    if (c.lane_bits > 8) c.lane_bits = 8;
    return c;
}

// 20 warps per CTA where the kernel allows it and the lane subtrees stay as large as with 16.
inline impir_config default_config(uint64_t n_records, uint32_t words, uint32_t n_queries, int sms) {
    const impir_config c16 = default_config_warps(n_records, words, n_queries, sms, 16);
    if (max_warps(c16.queries_per_warp, words) < 20) return c16;
    const impir_config c20 = default_config_warps(n_records, words, n_queries, sms, 20);
    return c20.lane_bits == c16.lane_bits && c20.queries_per_warp == c16.queries_per_warp ? c20 : c16;
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
    BoundsRecord* bounds;             // debug build: where failed checks are recorded
    unsigned long long keys_bytes;    // size of the key buffer (0: unknown)
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
    // extents for the debug build's index checks
    BoundsRecord* bounds;
    unsigned long long db_words;    // uint4 words of db[] the launch may read
    unsigned long long keys_bytes;  // size of the key buffer (0: unknown)
    uint32_t smem_bytes;            // dynamic shared memory of the launch
};

struct FinalizeParams {
    const uint8_t* ws;
    WsLayout lay;
    uint8_t* out;
    uint32_t n_queries;
    uint32_t record_bytes;
    uint32_t stride;
    BoundsRecord* bounds;
};

// Kernel launchers (defined in the .cu files). Each fused launcher first sets the kernel's
// dynamic shared-memory limit on the current device (once per device).
cudaError_t launch_setup(const SetupParams& p, cudaStream_t s);
// The current device's record of failed index checks in the debug build, else nullptr.
BoundsRecord* bounds_record();
// uint4 words of a database the index checks allow the kernels to read: n_words, less the
// records a debug-build test withholds (IMPIR_BOUNDS_TEST_WITHHOLD_RECORDS) to see a check fire.
unsigned long long bounds_db_words(unsigned long long n_words, uint32_t words_per_record);
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
// Sets the dynamic shared-memory limit of every instantiation of the XOR answer's kernels on
// the current device and loads their code there (with lazy module loading the first launch of
// a kernel otherwise does this, which may allocate device memory).
cudaError_t prepare_xor_kernels();
cudaError_t prepare_fused_q1();
cudaError_t prepare_fused_q2();
cudaError_t prepare_fused_q4();
cudaError_t prepare_fused_q8();
cudaError_t prepare_fused_q16();

// Host AES pieces of the product (independent of the oracle): T-table and key schedule.
void host_aes_te0(uint32_t te0[256]);
void host_aes_expand(const uint8_t key[16], uint32_t rk[44]);
void host_aes_encrypt(const uint32_t rk[44], const uint8_t in[16], uint8_t out[16]);

}  // namespace impir

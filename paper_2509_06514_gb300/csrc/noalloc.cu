// noalloc.cu — an answer entry point that allocates no memory at all.
//
// Who needs it: code that runs where allocating device memory is not allowed or not safe —
// for example inside an allocator or memory-pool callback, in a process whose device memory
// is fully reserved up front by a framework, or on a path that must not synchronize the
// device (cudaMalloc and cudaFree can implicitly synchronize). Such callers still own their
// inputs and outputs; what they cannot provide is the scratch workspace that
// impir_answer_async asks for. This file keeps that scratch in a fixed-size device array
// that exists for the life of the process on every GPU that loads the library.
//
// The same setup, fused and finalize kernels as the asynchronous path run here; only the
// workspace and the T-table pointer differ.
#include <mutex>

#include "../../include/impir.h"
#include "impir_internal.h"

namespace impir {

// Scratch: per-batch schedule and the per-query accumulators (see ws_layout). Every call
// shares it and it keeps the previous call's contents; the setup kernel zeroes what has to
// start at zero (work counter, accumulators) at the start of every call.
static __device__ __align__(256) uint8_t g_noalloc_scratch[IMPIR_NOALLOC_SCRATCH_BYTES];
// The 256-entry AES T-table the fused kernel expands into shared memory.
static __device__ __align__(16) uint32_t g_noalloc_te0[256];

impir_status set_error(impir_status st, const char* msg);

namespace {

constexpr int kMaxDevices = 64;

struct NoallocDevice {
    bool ready = false;
    uint8_t* scratch = nullptr;   // device address of g_noalloc_scratch on this device
    uint32_t* te0 = nullptr;      // device address of g_noalloc_te0 on this device
    int sms = 0;
    uint32_t mmo_rk[2][44];
    BoundsRecord* bounds = nullptr;  // debug build: the device's record of failed index checks
};

std::mutex g_mu;
NoallocDevice g_dev[kMaxDevices];

// One-time set-up for the current device: look up the arrays' device addresses (host code
// must not use the symbols themselves as addresses), fill the T-table, read the SM count, and
// prepare every kernel the entry point launches.
impir_status device_setup(NoallocDevice** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return set_error(IMPIR_ECUDA, "no current CUDA device");
    if (dev >= kMaxDevices) return set_error(IMPIR_EINVAL, "device index beyond the no-alloc table");
    std::lock_guard<std::mutex> lk(g_mu);
    NoallocDevice& d = g_dev[dev];
    if (!d.ready) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p)
            return set_error(IMPIR_ECUDA, "cudaGetSymbolAddress(scratch) failed");
        d.scratch = static_cast<uint8_t*>(p);
        p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_te0) != cudaSuccess || !p)
            return set_error(IMPIR_ECUDA, "cudaGetSymbolAddress(T-table) failed");
        d.te0 = static_cast<uint32_t*>(p);
        uint32_t te0[256];
        host_aes_te0(te0);
        if (cudaMemcpyToSymbol(g_noalloc_te0, te0, sizeof te0) != cudaSuccess)
            return set_error(IMPIR_ECUDA, "T-table upload failed");
        if (cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return set_error(IMPIR_ECUDA, "SM count query failed");
        host_aes_expand(reinterpret_cast<const uint8_t*>(IMPIR_MMO_KEY0), d.mmo_rk[0]);
        host_aes_expand(reinterpret_cast<const uint8_t*>(IMPIR_MMO_KEY1), d.mmo_rk[1]);
        // every kernel a later call can launch: shared-memory limit set and code loaded on this
        // device now, so that no later call does first-use work
        if (prepare_xor_kernels() != cudaSuccess) {
            cudaGetLastError();
            return set_error(IMPIR_ECUDA, "kernel preparation failed");
        }
        d.bounds = bounds_record();
        d.ready = true;
    }
    *out = &d;
    return IMPIR_OK;
}

}  // namespace
}  // namespace impir

using namespace impir;

extern "C" impir_status impir_answer_noalloc(const void* d_records, uint64_t n_records, uint32_t record_bytes,
                                             uint32_t stride_bytes, const uint8_t* d_keys,
                                             const uint32_t* d_key_offsets, uint32_t n_queries, uint8_t* d_out,
                                             void* cuda_stream) {
    if (!d_records || !d_keys || !d_key_offsets || !d_out) return set_error(IMPIR_EINVAL, "NULL device buffer");
    if (n_records == 0 || record_bytes == 0 || n_records > (1ull << IMPIR_MAX_DOMAIN_BITS))
        return set_error(IMPIR_EINVAL, "bad database size");
    if (stride_bytes % 16 || stride_bytes < record_bytes || (reinterpret_cast<uintptr_t>(d_records) & 15))
        return set_error(IMPIR_EINVAL, "records need a 16-byte stride >= record_bytes and 16-byte alignment");
    if (n_queries == 0) return IMPIR_OK;
    if (!bytes_ok(n_records, stride_bytes) || !bytes_ok(n_queries, stride_bytes))
        return set_error(IMPIR_EINVAL, "database or batch too large");
    const WsLayout lay = ws_layout(n_queries, stride_bytes);
    if (lay.total > IMPIR_NOALLOC_SCRATCH_BYTES)
        return set_error(IMPIR_EINVAL,
                         "batch too large for the fixed no-alloc scratch: n_queries * stride_bytes plus the "
                         "schedule must fit in IMPIR_NOALLOC_SCRATCH_BYTES");
    NoallocDevice* dev = nullptr;
    if (impir_status s = device_setup(&dev)) return s;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);

    // launch shape: the asynchronous path's default for this database and batch
    const uint32_t words = stride_bytes / 16;
    const impir_config cfg = default_config(n_records, words, n_queries, dev->sms);
    const uint32_t qpw = cfg.queries_per_warp, lane_bits = cfg.lane_bits;
    const uint32_t nk = nk_xor(words, qpw);
    const size_t smem = smem_for(cfg);

    SetupParams sp{};
    sp.keys = d_keys;
    sp.key_off = d_key_offsets;
    sp.ws = dev->scratch;
    sp.lay = lay;
    sp.n_records = n_records;
    sp.n_queries = n_queries;
    sp.words = words;
    sp.lane_bits = lane_bits;
    sp.qpw = qpw;
    sp.bounds = dev->bounds;
    if (launch_setup(sp, st) != cudaSuccess) {
        cudaGetLastError();
        return set_error(IMPIR_ECUDA, "setup kernel launch failed");
    }

    FusedParams fp{};
    fp.db = static_cast<const uint4*>(d_records);
    fp.keys = d_keys;
    fp.key_off = d_key_offsets;
    fp.ws = dev->scratch;
    fp.te0 = dev->te0;
    fp.lay = lay;
    fp.n_records = n_records;
    fp.n_queries = n_queries;
    fp.words = words;
    fp.lane_bits = lane_bits;
    fp.bits_words = 1u << lane_bits;
    for (int x = 0; x < 2; ++x)
        for (int i = 0; i < 44; ++i) fp.mmo_rk[x][i] = dev->mmo_rk[x][i];
    fp.bounds = dev->bounds;
    fp.db_words = bounds_db_words(n_records * words, words);
    fp.smem_bytes = uint32_t(smem);
    if (launch_fused(qpw, nk, dim3(dev->sms), dim3(cfg.warps_per_cta * 32), smem, st, fp) != cudaSuccess) {
        cudaGetLastError();
        return set_error(IMPIR_ECUDA, "fused kernel launch failed");
    }

    FinalizeParams zp{};
    zp.ws = dev->scratch;
    zp.lay = lay;
    zp.out = d_out;
    zp.n_queries = n_queries;
    zp.record_bytes = record_bytes;
    zp.stride = stride_bytes;
    zp.bounds = dev->bounds;
    if (launch_finalize(zp, st) != cudaSuccess) {
        cudaGetLastError();
        return set_error(IMPIR_ECUDA, "finalize kernel launch failed");
    }
    return IMPIR_OK;
}

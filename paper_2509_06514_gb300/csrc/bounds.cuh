// bounds.cuh — index checks of the debug build (compiled with -DIMPIR_BOUNDS).
//
// In the debug build every shared-memory, record, key, query, schedule and accumulator index
// the kernels use is compared with the extent of its buffer before the access. A failed check
// skips the access (a load yields zero) and is recorded: a per-device record (count, and the
// site and index of the first failure) that impir_bounds_status reads and clears, and a
// counter in the launch's workspace header. Nothing traps and nothing waits. In the normal
// build IMPIR_IN_BOUNDS(...) is the constant true and every check compiles away.
#pragma once

#include "impir_internal.h"

namespace impir {

#ifdef IMPIR_BOUNDS

// Where the checked buffers of the running launch are, shared by the block's threads (set by
// thread 0 at kernel entry, before the first __syncthreads).
struct BoundsCtx {
    BoundsRecord* rec;
    WsHeader* hdr;
    const uint8_t* keys;
    unsigned long long keys_bytes;   // 0: the key buffer's size is not known (asynchronous calls)
    const uint4* db;
    unsigned long long db_words;
    uint32_t smem_bytes;             // dynamic shared memory of the launch
    uint32_t warp_slice_bytes;       // each warp's slice of the bit / node / share buffer
};

__shared__ BoundsCtx s_bctx;

static __device__ __noinline__ bool bounds_failed(uint32_t site, unsigned long long idx) {
    if (s_bctx.rec && atomicAdd(&s_bctx.rec->n_failed, 1u) == 0) {
        s_bctx.rec->first_site = site;
        s_bctx.rec->first_index = idx;
    }
    if (s_bctx.hdr) atomicAdd(&s_bctx.hdr->bounds_failed, 1u);
    return false;
}

#define IMPIR_IN_BOUNDS(cond, site, idx) ((cond) || ::impir::bounds_failed((site), (unsigned long long)(idx)))

#else

#define IMPIR_IN_BOUNDS(cond, site, idx) (true)

#endif

}  // namespace impir

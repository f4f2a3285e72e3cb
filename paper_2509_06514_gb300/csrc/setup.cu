// setup.cu — per-batch scheduling and answer write-out kernels.
//
// setup_kernel (one CTA) reads the key headers on the device, validates them, sorts the
// queries by domain size (largest first), forms query groups of one domain size (the
// paper's queries handled together, §3.4), and builds the tile-major work-unit schedule the
// fused kernel walks: warp tile i is covered by every group whose DB prefix min(N, 2^m)
// reaches it, so the schedule is a handful of segments (one per distinct domain size). It
// also zeroes the per-query accumulators and the work counter.
//
// finalize_kernel copies each query's accumulator (record stride) into the caller's
// answer buffer (record_bytes per query).
#include <cstdlib>

#include "bounds.cuh"
#include "impir_internal.h"

namespace impir {

#ifdef IMPIR_BOUNDS
// The per-device record of failed index checks (debug build).
static __device__ BoundsRecord g_bounds_rec;
#endif

__global__ void __launch_bounds__(1024) setup_kernel(const SetupParams S) {
    __shared__ uint32_t hist[kMaxDomainBits + 1], cursor[kMaxDomainBits + 1];
    __shared__ uint32_t bstart[kMaxDomainBits + 1], gstart[kMaxDomainBits + 1], ngrp[kMaxDomainBits + 1];
    __shared__ uint32_t s_nbad, s_first_bad, s_ngroups;
    const uint32_t tid = threadIdx.x, nthr = blockDim.x;
    WsHeader* hdr = reinterpret_cast<WsHeader*>(S.ws);
    uint32_t* perm = reinterpret_cast<uint32_t*>(S.ws + S.lay.off_perm);
    uint32_t* qm = reinterpret_cast<uint32_t*>(S.ws + S.lay.off_qm);
    GroupDesc* groups = reinterpret_cast<GroupDesc*>(S.ws + S.lay.off_groups);
    SegDesc* segs = reinterpret_cast<SegDesc*>(S.ws + S.lay.off_segs);
    uint4* acc = reinterpret_cast<uint4*>(S.ws + S.lay.off_acc);

    if (tid <= kMaxDomainBits) hist[tid] = cursor[tid] = 0;
    if (tid == 0) {
        s_nbad = 0;
        s_first_bad = 0xffffffffu;
        hdr->bounds_failed = 0;
#ifdef IMPIR_BOUNDS
        s_bctx = BoundsCtx{S.bounds, hdr, S.keys, S.keys_bytes, nullptr, 0, 0, 0};
#endif
    }
    __syncthreads();

    // 1. validate each key's header and column 0 (a1 key intake)
    for (uint32_t q = tid; q < S.n_queries; q += nthr) {
        const uint32_t off = S.key_off[q];
        bool ok = (off & 7u) == 0;
        uint32_t m = 0;
        if (ok && !IMPIR_IN_BOUNDS(S.keys_bytes == 0 || off + 8ull <= S.keys_bytes, kSiteKey, off)) ok = false;
        if (ok) {
            const uint8_t* k = S.keys + off;
            const uint2 h = *reinterpret_cast<const uint2*>(k);
            const uint32_t ver = h.x & 0xffu, prf = (h.x >> 8) & 0xffu;
            m = (h.x >> 16) & 0xffu;
            ok = ver == 1 && prf <= 1 && m >= 1 && m <= kMaxDomainBits && (h.x >> 24) <= 1 && h.y == 0;
            if (ok) {
                const size_t z[3] = {8 + size_t(m + 1) * 16, 8 + size_t(m + 1) * 32, 8 + size_t(m + 1) * 48};
                for (int i = 0; i < 3; ++i) {
                    if (!IMPIR_IN_BOUNDS(S.keys_bytes == 0 || off + z[i] + 16 <= S.keys_bytes, kSiteKey, off + z[i])) {
                        ok = false;
                        break;
                    }
                    const uint2* p = reinterpret_cast<const uint2*>(k + z[i]);
                    const uint2 a = p[0], b = p[1];
                    ok = ok && (a.x | a.y | b.x | b.y) == 0;
                }
            }
        }
        qm[q] = ok ? m : 0;
        if (ok) {
            atomicAdd(&hist[m], 1u);
        } else {
            atomicAdd(&s_nbad, 1u);
            atomicMin(&s_first_bad, q);
        }
    }
    __syncthreads();

    // 2. buckets by domain size, largest first; groups of at most qpw queries per bucket;
    //    tile-major segments (a tile is 32 << lane_bits leaves for m >= 5 + lane_bits,
    //    otherwise the whole domain is one tile)
    if (tid == 0) {
        uint32_t pos = 0, g = 0;
        for (int m = kMaxDomainBits; m >= 1; --m) {
            bstart[m] = pos;
            gstart[m] = g;
            ngrp[m] = (hist[m] + S.qpw - 1) / S.qpw;
            pos += hist[m];
            g += ngrp[m];
        }
        s_ngroups = g;
        const unsigned long long tbig = 32ull << S.lane_bits;
        unsigned long long prev = 0, unit = 0;
        uint32_t nseg = 0;
        for (uint32_t m = 1; m <= kMaxDomainBits; ++m) {
            if (hist[m] == 0) continue;
            const unsigned long long dom = 1ull << m;
            const unsigned long long n_eff = S.n_records < dom ? S.n_records : dom;
            const unsigned long long tiles = m >= 5 + S.lane_bits ? (n_eff + tbig - 1) / tbig : 1ull;
            if (tiles > prev) {
                if (!IMPIR_IN_BOUNDS(nseg < kMaxSegments, kSiteWorkspace, nseg)) break;
                const uint32_t gcum = gstart[m] + ngrp[m];  // groups with domain bits >= m
                // clip to the tiles this launch covers (a chunk of a streamed database)
                const unsigned long long lo = prev > S.tile_lo ? prev : S.tile_lo;
                const unsigned long long hi = (S.tile_hi == 0 || tiles < S.tile_hi) ? tiles : S.tile_hi;
                if (hi > lo) {
                    segs[nseg].tile_lo = lo;
                    segs[nseg].unit_lo = unit;
                    segs[nseg].count = gcum;
                    segs[nseg].pad = 0;
                    segs[nseg].pad2 = 0;
                    unit += (hi - lo) * gcum;
                    ++nseg;
                }
                prev = tiles;
            }
        }
        hdr->counter = 0;
        hdr->n_units = unit;
        hdr->n_bad = s_nbad;
        hdr->first_bad = s_first_bad;
        hdr->n_groups = g;
        hdr->n_segs = nseg;
    }
    __syncthreads();

    // 3. scatter queries into their buckets (order inside a bucket does not matter: XOR
    //    answers are independent of which queries share a group)
    for (uint32_t q = tid; q < S.n_queries; q += nthr) {
        const uint32_t m = qm[q];
        if (m) {
            const uint32_t i = bstart[m] + atomicAdd(&cursor[m], 1u);
            if (IMPIR_IN_BOUNDS(i < S.n_queries, kSiteWorkspace, i)) perm[i] = q;
        }
    }
    // 4. group descriptors
    for (uint32_t gi = tid; gi < s_ngroups; gi += nthr) {
        uint32_t m = kMaxDomainBits;
        while (m > 1 && !(gi >= gstart[m] && gi < gstart[m] + ngrp[m])) --m;
        const uint32_t k = gi - gstart[m];
        GroupDesc d;
        d.first = bstart[m] + k * S.qpw;
        d.count = min(S.qpw, hist[m] - k * S.qpw);
        d.m = m;
        d.pad = 0;
        if (IMPIR_IN_BOUNDS(gi < S.n_queries + kMaxDomainBits + 8, kSiteWorkspace, gi)) groups[gi] = d;
    }
    // 5. zero the accumulators (kept across the chunks of a streamed database)
    if (!S.keep_acc) {
        const size_t nacc = size_t(S.n_queries) * S.words;
        for (size_t i = tid; i < nacc; i += nthr) acc[i] = make_uint4(0, 0, 0, 0);
    }
}

__global__ void finalize_kernel(const FinalizeParams F) {
#ifdef IMPIR_BOUNDS
    if (threadIdx.x == 0) s_bctx = BoundsCtx{F.bounds, nullptr, nullptr, 0, nullptr, 0, 0, 0};
    __syncthreads();
#endif
    const uint8_t* acc = F.ws + F.lay.off_acc;
    const size_t n = size_t(F.n_queries) * F.record_bytes;
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
        const size_t q = i / F.record_bytes, b = i - q * F.record_bytes;
        const size_t a = q * F.stride + b;
        if (IMPIR_IN_BOUNDS(b < F.stride && a < size_t(F.n_queries) * F.stride, kSiteAcc, a)) F.out[i] = acc[a];
    }
}

BoundsRecord* bounds_record() {
#ifdef IMPIR_BOUNDS
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_bounds_rec) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return static_cast<BoundsRecord*>(p);
#else
    return nullptr;
#endif
}

unsigned long long bounds_db_words(unsigned long long n_words, uint32_t words_per_record) {
#ifdef IMPIR_BOUNDS
    // a debug-build test withholds the last records of every database from the checked extent
    // (the memory stays valid), so that the checks on record reads fire
    if (const char* w = std::getenv("IMPIR_BOUNDS_TEST_WITHHOLD_RECORDS")) {
        const unsigned long long k = std::strtoull(w, nullptr, 10) * words_per_record;
        return k < n_words ? n_words - k : 0;
    }
#else
    (void)words_per_record;
#endif
    return n_words;
}

cudaError_t launch_setup(const SetupParams& p, cudaStream_t s) {
    setup_kernel<<<1, 1024, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const FinalizeParams& p, cudaStream_t s) {
    const size_t n = size_t(p.n_queries) * p.record_bytes;
    const unsigned blocks = unsigned(n / 256 + 1 < 1024 ? n / 256 + 1 : 1024);
    finalize_kernel<<<blocks, 256, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_fused(uint32_t qpw, uint32_t nk, dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                         const FusedParams& p) {
    switch (qpw) {
        case 1: return launch_fused_q1(nk, grid, block, smem, s, p);
        case 2: return launch_fused_q2(nk, grid, block, smem, s, p);
        case 4: return launch_fused_q4(nk, grid, block, smem, s, p);
        case 8: return launch_fused_q8(nk, grid, block, smem, s, p);
        case 16: return launch_fused_q16(nk, grid, block, smem, s, p);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t prepare_xor_kernels() {
    cudaError_t e = prepare_fused_q1();
    if (e == cudaSuccess) e = prepare_fused_q2();
    if (e == cudaSuccess) e = prepare_fused_q4();
    if (e == cudaSuccess) e = prepare_fused_q8();
    if (e == cudaSuccess) e = prepare_fused_q16();
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, setup_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, finalize_kernel);
    return e;
}

}  // namespace impir

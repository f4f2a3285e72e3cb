// impir_host.cpp — host runtime behind include/impir.h: database registry, key intake,
// launch configuration and autotuning, the synchronous and asynchronous answer paths, and
// the client-side key generator used by tests.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/impir.h"
#include "impir_internal.h"

using namespace impir;

namespace {
thread_local std::string g_err;
}  // namespace

namespace impir {
// Records a message for impir_last_error (used by units outside this file).
impir_status set_error(impir_status st, const char* msg) {
    g_err = msg;
    return st;
}
}  // namespace impir

namespace {

impir_status fail(impir_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

// A failed runtime call also sets the runtime's last error; consume it so that the next
// unrelated CUDA call in the process (ours or the caller's) does not report it again.
impir_status cuda_fail(cudaError_t e, const char* what) {
    cudaGetLastError();
    return fail(IMPIR_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call, what)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

// ---- per-process device state (the current device at first use) ----
struct DeviceState {
    bool ok = false;
    std::string err;
    int device = -1;
    int sms = 0;
    uint32_t* d_te0 = nullptr;
    uint32_t mmo_rk[2][44];
};

DeviceState& device_state() {
    static DeviceState st;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaError_t e = cudaGetDevice(&st.device);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&st.sms, cudaDevAttrMultiProcessorCount, st.device);
        uint32_t te0[256];
        host_aes_te0(te0);
        if (e == cudaSuccess) e = cudaMalloc(&st.d_te0, sizeof te0);
        if (e == cudaSuccess) e = cudaMemcpy(st.d_te0, te0, sizeof te0, cudaMemcpyHostToDevice);
        host_aes_expand(reinterpret_cast<const uint8_t*>(IMPIR_MMO_KEY0), st.mmo_rk[0]);
        host_aes_expand(reinterpret_cast<const uint8_t*>(IMPIR_MMO_KEY1), st.mmo_rk[1]);
        if (e != cudaSuccess) {
            st.err = cudaGetErrorString(e);
            return;
        }
        st.ok = true;
    });
    return st;
}

impir_status need_device(DeviceState** out) {
    DeviceState& st = device_state();
    if (!st.ok) return fail(IMPIR_ECUDA, "CUDA device unavailable: %s", st.err.c_str());
    *out = &st;
    return IMPIR_OK;
}

// ---- database registry ----
struct Db {
    const void* d = nullptr;
    uint64_t n = 0;
    uint32_t bytes = 0, stride = 0;
    bool owned = false;
    bool live = false;
    bool cfg_set = false;
    impir_config cfg{};
    uint64_t version = 0;  // bumped by every bulk update
    uint64_t row_lo = 0;   // a row shard: global index of its first row
    uint64_t n_total = 0;  // and the whole database's record count (n for a whole database)
};

std::mutex g_db_mu;
std::vector<Db> g_dbs;

impir_status get_db(int32_t h, Db* out) {
    std::lock_guard<std::mutex> lk(g_db_mu);
    if (h < 1 || size_t(h) > g_dbs.size() || !g_dbs[h - 1].live) return fail(IMPIR_EINVAL, "unknown database handle %d", h);
    *out = g_dbs[h - 1];
    return IMPIR_OK;
}

int32_t add_db(const Db& d) {
    std::lock_guard<std::mutex> lk(g_db_mu);
    g_dbs.push_back(d);
    g_dbs.back().live = true;
    return int32_t(g_dbs.size());
}

// ---- configuration (launch-shape helpers shared with the no-alloc path: impir_internal.h) ----
size_t smem_add(const impir_config& c);

// mode 0: the XOR answer's kernels; mode 1: the additive answer's (after add_config)
impir_status check_config(const impir_config& c, uint32_t words, int mode = 0) {
    if (c.lane_bits > kMaxLaneBits) return fail(IMPIR_EINVAL, "lane_bits %u > %u", c.lane_bits, kMaxLaneBits);
    if (c.queries_per_warp != 1 && c.queries_per_warp != 2 && c.queries_per_warp != 4 && c.queries_per_warp != 8 &&
        c.queries_per_warp != 16)
        return fail(IMPIR_EINVAL, "queries_per_warp must be 1, 2, 4, 8 or 16");
    if (c.queries_per_warp * (mode == 0 ? nk_xor(words, c.queries_per_warp) : nk_need(words)) > 16)
        return fail(IMPIR_EINVAL, "queries_per_warp %u too large for %u-byte records", c.queries_per_warp, words * 16);
    if (c.warps_per_cta < 4 || c.warps_per_cta > max_warps(c.queries_per_warp, words))
        return fail(IMPIR_EINVAL, "warps_per_cta must be 4..%u for this record size and queries_per_warp",
                    max_warps(c.queries_per_warp, words));
    if (c.queries_per_launch > 1) return fail(IMPIR_EINVAL, "queries_per_launch must be 0 or 1");
    const size_t smem = mode == 0 ? smem_for(c) : smem_add(c);
    if (smem > kSmemMax) return fail(IMPIR_EINVAL, "configuration needs %zu bytes of shared memory", smem);
    return IMPIR_OK;
}

impir_config config_for(const Db& db, uint32_t n_queries, int sms) {
    if (db.cfg_set) return db.cfg;
    return default_config(db.n, db.stride / 16, n_queries, sms);
}

// ---- key intake on the host (validation before any launch) ----
impir_status parse_host_keys(const uint8_t* keys, uint32_t n, std::vector<uint32_t>& offs, size_t& total) {
    offs.resize(n);
    size_t o = 0;
    for (uint32_t q = 0; q < n; ++q) {
        const uint8_t* k = keys + o;
        const uint32_t m = k[2];
        if (k[0] != IMPIR_KEY_VERSION) return fail(IMPIR_EINVAL, "key %u: version %u", q, k[0]);
        if (k[1] > 1) return fail(IMPIR_EINVAL, "key %u: unknown prf %u", q, k[1]);
        if (m < 1 || m > IMPIR_MAX_DOMAIN_BITS) return fail(IMPIR_EINVAL, "key %u: domain bits %u", q, m);
        if (k[3] > 1) return fail(IMPIR_EINVAL, "key %u: party index %u is not 0 or 1", q, k[3]);
        for (int i = 4; i < 8; ++i)
            if (k[i]) return fail(IMPIR_EINVAL, "key %u: reserved header byte %d is not zero", q, i);
        const size_t z[3] = {8 + size_t(m + 1) * 16, 8 + size_t(m + 1) * 32, 8 + size_t(m + 1) * 48};
        for (size_t zi : z)
            for (int b = 0; b < 16; ++b)
                if (k[zi + b]) return fail(IMPIR_EINVAL, "key %u: column-0 codeword other than the root is not zero", q);
        if (o > 0xffffffffull) return fail(IMPIR_EINVAL, "keys exceed 4 GiB");
        offs[q] = uint32_t(o);
        o += impir_key_bytes(m);
    }
    total = o;
    return IMPIR_OK;
}

// ---- index checks of the debug build ----

// Reads and clears the current device's record of failed index checks (the caller has waited
// for the launches it wants covered). Without IMPIR_BOUNDS: EINVAL.
impir_status bounds_take(uint32_t* n_failed, uint32_t* site, uint64_t* index) {
    BoundsRecord* rec = bounds_record();
    if (!rec) return fail(IMPIR_EINVAL, "the library was built without IMPIR_BOUNDS");
    BoundsRecord h{}, zero{};
    CK(cudaDeviceSynchronize(), "wait for the device");
    CK(cudaMemcpy(&h, rec, sizeof h, cudaMemcpyDeviceToHost), "bounds record read");
    CK(cudaMemcpy(rec, &zero, sizeof zero, cudaMemcpyHostToDevice), "bounds record clear");
    if (n_failed) *n_failed = h.n_failed;
    if (site) *site = h.first_site;
    if (index) *index = h.first_index;
    return IMPIR_OK;
}

// Synchronous calls of the debug build end here: an error if any index check failed.
impir_status bounds_verdict() {
#ifdef IMPIR_BOUNDS
    uint32_t n = 0, site = 0;
    uint64_t idx = 0;
    if (impir_status s = bounds_take(&n, &site, &idx)) return s;
    if (n) return fail(IMPIR_ECUDA, "%u index checks failed; the first at site %u, index %llu", n, site,
                       (unsigned long long)idx);
#endif
    return IMPIR_OK;
}

// ---- kernel timing (events around fused launches) ----
struct Timing {
    std::mutex mu;
    bool on = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
    double fused_ms = 0;
    uint64_t fused = 0, all = 0;
};
Timing g_timing;

bool timing_on() {
    std::lock_guard<std::mutex> lk(g_timing.mu);
    return g_timing.on;
}

void count_launches(uint64_t n) {
    std::lock_guard<std::mutex> lk(g_timing.mu);
    if (g_timing.on) g_timing.all += n;
}

// ---- launches ----
// The additive answer takes 1 or 2 queries per warp tile (records up to 2 KiB: 2, else 1; with
// 4 the extra walk states and smaller chunks cost more than the shared record loads save), and
// keeps one 32-bit share per leaf for 32 / queries leaves per lane at a time and query (larger
// lane subtrees are scanned in chunks): 4 KiB per warp.
uint32_t max_add_qpw(uint32_t words) { return nk_need(words) <= 4 ? 2u : 1u; }

// 32-bit share words per query slot of a warp.
uint32_t add_share_words(const impir_config& c) {
    const uint32_t ch = std::min(1u << c.lane_bits, 32u / c.queries_per_warp);
    return 32u * ch;
}

impir_config add_config(impir_config c, uint32_t words) {
    c.queries_per_warp = std::min(c.queries_per_warp, max_add_qpw(words));
    if (c.warps_per_cta > 16 && nk_need(words) > 1) c.warps_per_cta = 16;  // wider records: 16-warp kernels
    return c;
}

// Default shape of the additive answer: as many queries per unit as the record size allows
// (up to 2, and no more than the batch), and the largest lane subtree, up to 256 leaves, that
// still leaves three units per resident warp.
impir_config default_add_config(uint64_t n_records, uint32_t words, uint32_t n_queries, int sms) {
    impir_config c{};
    c.warps_per_cta = 16;
    c.queries_per_warp = max_add_qpw(words);
    while (c.queries_per_warp > 1 && c.queries_per_warp > n_queries) c.queries_per_warp >>= 1;
    c.queries_per_launch = 0;
    const double warps = double(sms) * c.warps_per_cta;
    const double groups = std::ceil(double(n_queries) / c.queries_per_warp);
    c.lane_bits = 0;
    for (uint32_t s = 8; s > 0; --s) {
        const double tiles = std::ceil(double(n_records) / double(32ull << s));
        if (groups * tiles >= 3.0 * warps) {
            c.lane_bits = s;
            break;
        }
    }
    return c;
}

size_t smem_add(const impir_config& c) {
    return kTableBytes + kSegSmemBytes + size_t(c.warps_per_cta) * c.queries_per_warp * add_share_words(c) * 4;
}

// keys_bytes: size of the key buffer when the library knows it (0: unknown; only the debug
// build's index checks use it)
impir_status launch_batch(const DeviceState& dev, const Db& db, const impir_config& cfg, const uint8_t* d_keys,
                          const uint32_t* d_off, uint32_t n, uint8_t* d_out, uint8_t* d_ws, cudaStream_t st,
                          int mode = 0, size_t keys_bytes = 0) {
    const WsLayout lay = ws_layout(n, db.stride);
    // a row shard covers the warp tiles of its rows (shard bounds are whole tiles) of a
    // database of n_total records; its device rows start at global row row_lo
    const uint64_t T = 32ull << cfg.lane_bits;
    const bool shard = db.row_lo != 0 || db.n_total != db.n;
    SetupParams sp{};
    sp.keys = d_keys;
    sp.key_off = d_off;
    sp.ws = d_ws;
    sp.lay = lay;
    sp.n_records = db.n_total;
    sp.n_queries = n;
    sp.words = db.stride / 16;
    sp.lane_bits = cfg.lane_bits;
    sp.qpw = cfg.queries_per_warp;
    sp.tile_lo = shard ? db.row_lo / T : 0;
    sp.tile_hi = shard ? (db.row_lo + db.n + T - 1) / T : 0;
    sp.bounds = bounds_record();
    sp.keys_bytes = keys_bytes;
    CK(launch_setup(sp, st), "setup kernel launch");

    FusedParams fp{};
    fp.db = static_cast<const uint4*>(db.d);
    fp.keys = d_keys;
    fp.key_off = d_off;
    fp.ws = d_ws;
    fp.te0 = dev.d_te0;
    fp.lay = lay;
    fp.n_records = db.n_total;
    fp.n_queries = n;
    fp.words = db.stride / 16;
    fp.lane_bits = cfg.lane_bits;
    fp.bits_words = mode == 0 ? 1u << cfg.lane_bits : add_share_words(cfg);
    fp.rec_lo = db.row_lo;
    std::memcpy(fp.mmo_rk, dev.mmo_rk, sizeof fp.mmo_rk);
    const size_t smem = mode == 0 ? smem_for(cfg) : smem_add(cfg);
    fp.bounds = sp.bounds;
    fp.db_words = bounds_db_words(db.n * (db.stride / 16), db.stride / 16);
    fp.keys_bytes = keys_bytes;
    fp.smem_bytes = uint32_t(smem);
    const bool timed = timing_on();
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (timed) {
        CK(cudaEventCreate(&ev0), "event create");
        CK(cudaEventCreate(&ev1), "event create");
        CK(cudaEventRecord(ev0, st), "event record");
    }
    if (mode == 0)
        CK(launch_fused(cfg.queries_per_warp, nk_xor(fp.words, cfg.queries_per_warp), dim3(dev.sms),
                        dim3(cfg.warps_per_cta * 32), smem, st, fp),
           "fused kernel launch");
    else
        CK(launch_fused_add(cfg.queries_per_warp, nk_need(fp.words), dim3(dev.sms), dim3(cfg.warps_per_cta * 32), smem,
                            st, fp),
           "fused kernel launch (additive)");
    if (timed) {
        CK(cudaEventRecord(ev1, st), "event record");
        std::lock_guard<std::mutex> lk(g_timing.mu);
        g_timing.pending.emplace_back(ev0, ev1);
        g_timing.fused += 1;
    }
    if (!d_out) {  // the caller reads the answers from the accumulators itself
        count_launches(2);
        return IMPIR_OK;
    }
    count_launches(3);

    FinalizeParams zp{};
    zp.ws = d_ws;
    zp.lay = lay;
    zp.out = d_out;
    zp.n_queries = n;
    zp.record_bytes = db.bytes;
    zp.stride = db.stride;
    zp.bounds = sp.bounds;
    CK(launch_finalize(zp, st), "finalize kernel launch");
    return IMPIR_OK;
}

// direct_out: no finalize kernel; the answers stay in the workspace's accumulators (one
// launch for the batch only), where the synchronous path downloads them from
impir_status answer_async_impl(const Db& db, const impir_config* cfg_in, const uint8_t* d_keys, const uint32_t* d_off,
                               uint32_t n, uint8_t* d_out, void* d_ws, size_t ws_bytes, cudaStream_t st, int mode = 0,
                               bool direct_out = false, size_t keys_bytes = 0) {
    DeviceState* dev = nullptr;
    if (impir_status s = need_device(&dev)) return s;
    if (n == 0) return IMPIR_OK;
    if (!d_keys || !d_off || (!d_out && !direct_out) || !d_ws) return fail(IMPIR_EINVAL, "NULL device buffer");
    if (!bytes_ok(n, db.stride)) return fail(IMPIR_EINVAL, "batch too large: %u answers of %u bytes", n, db.stride);
    if (reinterpret_cast<uintptr_t>(d_ws) & 255) return fail(IMPIR_EINVAL, "workspace must be 256-byte aligned");
    impir_config cfg = cfg_in                      ? *cfg_in
                       : (mode == 1 && !db.cfg_set) ? default_add_config(db.n, db.stride / 16, n, dev->sms)
                                                    : config_for(db, n, dev->sms);
    if (mode == 1) {
        if (db.bytes % 4) return fail(IMPIR_EINVAL, "the additive answer needs records of a multiple of 4 bytes");
        cfg = add_config(cfg, db.stride / 16);
    }
    if (impir_status s = check_config(cfg, db.stride / 16, mode)) return s;
    if (cfg.queries_per_launch == 1) {
        if (direct_out) return fail(IMPIR_EINVAL, "direct answers need one launch for the batch");
        if (ws_bytes < ws_layout(1, db.stride).total) return fail(IMPIR_ENOMEM, "workspace too small");
        for (uint32_t q = 0; q < n; ++q)
            if (impir_status s = launch_batch(*dev, db, cfg, d_keys, d_off + q, 1, d_out + size_t(q) * db.bytes,
                                              static_cast<uint8_t*>(d_ws), st, mode, keys_bytes))
                return s;
        return IMPIR_OK;
    }
    if (ws_bytes < ws_layout(n, db.stride).total)
        return fail(IMPIR_ENOMEM, "workspace of %zu bytes is smaller than the %zu needed", ws_bytes,
                    ws_layout(n, db.stride).total);
    return launch_batch(*dev, db, cfg, d_keys, d_off, n, direct_out ? nullptr : d_out, static_cast<uint8_t*>(d_ws), st,
                        mode, keys_bytes);
}

// ---- synchronous path context: cached device and pinned buffers ----
struct SyncCtx {
    std::mutex mu;
    cudaStream_t stream = nullptr;
    void *d_keys = nullptr, *d_ws = nullptr, *d_out = nullptr;  // d_keys: keys, then their offsets
    size_t c_keys = 0, c_ws = 0, c_out = 0;
    uint8_t* h_stage = nullptr;
    size_t c_stage = 0;
};

SyncCtx g_sync;

// ---- streamed path context: staging buffers, workspace, streams and events kept for reuse ----
struct StreamCtx {
    std::mutex mu;
    void *d_buf[2] = {nullptr, nullptr}, *d_keys = nullptr, *d_off = nullptr, *d_ws = nullptr, *d_out = nullptr;
    size_t c_buf[2] = {0, 0}, c_keys = 0, c_off = 0, c_ws = 0, c_out = 0;
    uint32_t zeroed_stride = 0;  // padding of both buffers is zero for this record layout (0: unknown)
    cudaStream_t cs = nullptr, ks[2] = {nullptr, nullptr};
    cudaEvent_t copied[2] = {nullptr, nullptr}, consumed[2] = {nullptr, nullptr}, ready = nullptr, done1 = nullptr;
    bool ok = false;
};

StreamCtx g_streamed;

cudaError_t streamed_ctx_init(StreamCtx& c) {
    if (c.ok) return cudaSuccess;
    cudaError_t e = cudaStreamCreateWithFlags(&c.cs, cudaStreamNonBlocking);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithFlags(&c.ks[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c.copied[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c.consumed[i], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c.ready, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c.done1, cudaEventDisableTiming);
    c.ok = e == cudaSuccess;
    return e;
}

impir_status grow(void** p, size_t* cap, size_t need, bool pinned = false) {
    if (*cap >= need) return IMPIR_OK;
    size_t n = std::max(need, *cap * 2);
    if (*p) {
        if (pinned)
            cudaFreeHost(*p);
        else
            cudaFree(*p);
        *p = nullptr;
        *cap = 0;
    }
    cudaError_t e = pinned ? cudaMallocHost(p, n) : cudaMalloc(p, n);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(IMPIR_ENOMEM, "allocation of %zu bytes failed: %s", n, cudaGetErrorString(e));
    }
    *cap = n;
    return IMPIR_OK;
}

// ---- tuning cache: (SMs, N, stride, batch, config hint) -> best configuration ----
std::mutex g_tune_mu;
std::map<std::tuple<int, uint64_t, uint32_t, uint32_t>, impir_config> g_tune;

}  // namespace

extern "C" {

size_t impir_key_bytes(uint32_t m) { return 8 + size_t(64) * (m + 1); }

const char* impir_last_error(void) { return g_err.c_str(); }

impir_status impir_timing_enable(int enable) {
    std::lock_guard<std::mutex> lk(g_timing.mu);
    for (auto& p : g_timing.pending) {
        cudaEventSynchronize(p.second);
        cudaEventDestroy(p.first);
        cudaEventDestroy(p.second);
    }
    g_timing.pending.clear();
    g_timing.on = enable != 0;
    g_timing.fused_ms = 0;
    g_timing.fused = g_timing.all = 0;
    return IMPIR_OK;
}

impir_status impir_timing_read(double* fused_ms, uint64_t* fused_launches, uint64_t* all_launches) {
    std::lock_guard<std::mutex> lk(g_timing.mu);
    for (auto& p : g_timing.pending) {
        CK(cudaEventSynchronize(p.second), "event sync");
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, p.first, p.second), "event time");
        g_timing.fused_ms += ms;
        cudaEventDestroy(p.first);
        cudaEventDestroy(p.second);
    }
    g_timing.pending.clear();
    if (fused_ms) *fused_ms = g_timing.fused_ms;
    if (fused_launches) *fused_launches = g_timing.fused;
    if (all_launches) *all_launches = g_timing.all;
    return IMPIR_OK;
}

impir_status impir_bounds_status(uint32_t* n_failed, uint32_t* first_site, uint64_t* first_index) {
    return bounds_take(n_failed, first_site, first_index);
}

int32_t impir_device_sm_count(void) {
    DeviceState& st = device_state();
    return st.ok ? st.sms : 0;
}

impir_status impir_db_load(const void* records, uint64_t n_records, uint32_t record_bytes, int32_t* db_handle) {
    if (!records || !db_handle) return fail(IMPIR_EINVAL, "NULL argument");
    if (n_records == 0 || record_bytes == 0) return fail(IMPIR_EINVAL, "empty database");
    if (n_records > (1ull << IMPIR_MAX_DOMAIN_BITS)) return fail(IMPIR_EINVAL, "more than 2^40 records");
    const uint64_t stride = (uint64_t(record_bytes) + 15u) & ~uint64_t(15);
    if (stride > 0xfffffff0ull || !bytes_ok(n_records, stride))
        return fail(IMPIR_EINVAL, "database of %llu records of %u bytes is too large", (unsigned long long)n_records,
                    record_bytes);
    DeviceState* dev = nullptr;
    if (impir_status s = need_device(&dev)) return s;
    void* d = nullptr;
    cudaError_t e = cudaMalloc(&d, size_t(n_records) * stride);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(IMPIR_ENOMEM, "device allocation of %llu bytes failed: %s",
                    (unsigned long long)(n_records * stride), cudaGetErrorString(e));
    }
    if (stride != record_bytes) {
        e = cudaMemset(d, 0, size_t(n_records) * stride);
        if (e == cudaSuccess)
            e = cudaMemcpy2D(d, stride, records, record_bytes, record_bytes, n_records, cudaMemcpyHostToDevice);
    } else {
        e = cudaMemcpy(d, records, size_t(n_records) * stride, cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        cudaFree(d);
        return cuda_fail(e, "database copy");
    }
    Db db;
    db.d = d;
    db.n = n_records;
    db.n_total = n_records;
    db.bytes = record_bytes;
    db.stride = uint32_t(stride);
    db.owned = true;
    *db_handle = add_db(db);
    return IMPIR_OK;
}

impir_status impir_db_load_rows(const void* records, uint64_t n_rows, uint32_t record_bytes, uint64_t row_lo,
                                uint64_t n_total, int32_t* db_handle) {
    if (!db_handle) return fail(IMPIR_EINVAL, "NULL argument");
    if (n_total > (1ull << IMPIR_MAX_DOMAIN_BITS)) return fail(IMPIR_EINVAL, "more than 2^40 records");
    if (!bytes_ok(n_total, (uint64_t(record_bytes) + 15u) & ~uint64_t(15)))
        return fail(IMPIR_EINVAL, "database too large");
    if (n_rows == 0 || row_lo >= n_total || n_rows > n_total - row_lo)
        return fail(IMPIR_EINVAL, "rows [%llu, +%llu) are not inside a database of %llu records",
                    (unsigned long long)row_lo, (unsigned long long)n_rows, (unsigned long long)n_total);
    if (row_lo % IMPIR_SHARD_ALIGN || (row_lo + n_rows != n_total && (row_lo + n_rows) % IMPIR_SHARD_ALIGN))
        return fail(IMPIR_EINVAL, "shard bounds must be multiples of %u records (or the database end)",
                    IMPIR_SHARD_ALIGN);
    int32_t h = 0;
    if (impir_status s = impir_db_load(records, n_rows, record_bytes, &h)) return s;
    std::lock_guard<std::mutex> lk(g_db_mu);
    g_dbs[h - 1].row_lo = row_lo;
    g_dbs[h - 1].n_total = n_total;
    *db_handle = h;
    return IMPIR_OK;
}

impir_status impir_db_rows(int32_t h, uint64_t* row_lo, uint64_t* n_total) {
    Db db;
    if (impir_status s = get_db(h, &db)) return s;
    if (row_lo) *row_lo = db.row_lo;
    if (n_total) *n_total = db.n_total;
    return IMPIR_OK;
}

impir_status impir_db_attach(const void* d_records, uint64_t n_records, uint32_t record_bytes, uint32_t stride_bytes,
                             int32_t* db_handle) {
    if (!d_records || !db_handle) return fail(IMPIR_EINVAL, "NULL argument");
    if (n_records == 0 || record_bytes == 0) return fail(IMPIR_EINVAL, "empty database");
    if (n_records > (1ull << IMPIR_MAX_DOMAIN_BITS)) return fail(IMPIR_EINVAL, "more than 2^40 records");
    if (stride_bytes % 16 || stride_bytes < record_bytes) return fail(IMPIR_EINVAL, "bad stride %u", stride_bytes);
    if (!bytes_ok(n_records, stride_bytes)) return fail(IMPIR_EINVAL, "database too large");
    if (reinterpret_cast<uintptr_t>(d_records) & 15) return fail(IMPIR_EINVAL, "records must be 16-byte aligned");
    Db db;
    db.d = d_records;
    db.n = n_records;
    db.n_total = n_records;
    db.bytes = record_bytes;
    db.stride = stride_bytes;
    db.owned = false;
    *db_handle = add_db(db);
    return IMPIR_OK;
}

impir_status impir_db_free(int32_t h) {
    Db db;
    {
        std::lock_guard<std::mutex> lk(g_db_mu);
        if (h < 1 || size_t(h) > g_dbs.size() || !g_dbs[h - 1].live) return fail(IMPIR_EINVAL, "unknown database handle %d", h);
        db = g_dbs[h - 1];
        g_dbs[h - 1].live = false;
    }
    if (db.owned) cudaFree(const_cast<void*>(db.d));
    return IMPIR_OK;
}

impir_status impir_db_info(int32_t h, uint64_t* n, uint32_t* bytes, uint32_t* stride, const void** d) {
    Db db;
    if (impir_status s = get_db(h, &db)) return s;
    if (n) *n = db.n;
    if (bytes) *bytes = db.bytes;
    if (stride) *stride = db.stride;
    if (d) *d = db.d;
    return IMPIR_OK;
}

impir_status impir_db_version(int32_t h, uint64_t* version) {
    Db db;
    if (impir_status s = get_db(h, &db)) return s;
    if (version) *version = db.version;
    return IMPIR_OK;
}

impir_status impir_db_update_async(int32_t h, uint64_t first, uint64_t n, const void* records, void* stream,
                                   uint64_t* new_version) {
    if (!records && n) return fail(IMPIR_EINVAL, "NULL records");
    std::lock_guard<std::mutex> lk(g_db_mu);
    if (h < 1 || size_t(h) > g_dbs.size() || !g_dbs[h - 1].live) return fail(IMPIR_EINVAL, "unknown database handle %d", h);
    Db& db = g_dbs[h - 1];
    if (first > db.n || n > db.n - first) return fail(IMPIR_EINVAL, "update range beyond the database");
    if (n) {
        uint8_t* dst = static_cast<uint8_t*>(const_cast<void*>(db.d)) + first * db.stride;
        // one contiguous copy when records carry no padding; row-by-row otherwise
        if (db.stride == db.bytes)
            CK(cudaMemcpyAsync(dst, records, n * db.bytes, cudaMemcpyHostToDevice, static_cast<cudaStream_t>(stream)),
               "database update copy");
        else
            CK(cudaMemcpy2DAsync(dst, db.stride, records, db.bytes, db.bytes, n, cudaMemcpyHostToDevice,
                                 static_cast<cudaStream_t>(stream)),
               "database update copy");
    }
    db.version += 1;
    if (new_version) *new_version = db.version;
    return IMPIR_OK;
}

impir_status impir_db_update(int32_t h, uint64_t first, uint64_t n, const void* records) {
    DeviceState* dev = nullptr;
    if (impir_status s = need_device(&dev)) return s;
    CK(cudaDeviceSynchronize(), "wait for answers in flight");
    if (impir_status s = impir_db_update_async(h, first, n, records, nullptr, nullptr)) return s;
    CK(cudaDeviceSynchronize(), "database update");
    return IMPIR_OK;
}

size_t impir_workspace_bytes(uint32_t n_queries, uint32_t stride_bytes) {
    return ws_layout(n_queries, (stride_bytes + 15u) & ~15u).total;
}

impir_status impir_answer_async(int32_t h, const uint8_t* d_keys, const uint32_t* d_off, uint32_t n, uint8_t* d_out,
                                void* d_ws, size_t ws_bytes, void* stream) {
    Db db;
    if (impir_status s = get_db(h, &db)) return s;
    return answer_async_impl(db, nullptr, d_keys, d_off, n, d_out, d_ws, ws_bytes, static_cast<cudaStream_t>(stream));
}

impir_status impir_workspace_status(const void* d_ws, uint32_t* n_bad, uint32_t* first_bad) {
    if (!d_ws) return fail(IMPIR_EINVAL, "NULL workspace");
    WsHeader h;
    CK(cudaDeviceSynchronize(), "synchronize");
    CK(cudaMemcpy(&h, d_ws, sizeof h, cudaMemcpyDeviceToHost), "workspace status copy");
    if (n_bad) *n_bad = h.n_bad;
    if (first_bad) *first_bad = h.first_bad;
    return IMPIR_OK;
}

static impir_status answer_sync(int32_t h, const uint8_t* keys, uint32_t n, uint8_t* out, int mode) {
    Db db;
    if (impir_status s = get_db(h, &db)) return s;
    if (n == 0) return IMPIR_OK;
    if (!keys || !out) return fail(IMPIR_EINVAL, "NULL argument");
    DeviceState* dev = nullptr;
    if (impir_status s = need_device(&dev)) return s;
    if (!bytes_ok(n, db.stride)) return fail(IMPIR_EINVAL, "batch too large: %u answers of %u bytes", n, db.stride);
    std::vector<uint32_t> offs;
    size_t total = 0;
    if (impir_status s = parse_host_keys(keys, n, offs, total)) return s;
    std::lock_guard<std::mutex> lk(g_sync.mu);
    if (!g_sync.stream) CK(cudaStreamCreateWithFlags(&g_sync.stream, cudaStreamNonBlocking), "stream create");
    const impir_config cfg = config_for(db, n, dev->sms);
    // records without padding and one launch for the batch: the answers are downloaded straight
    // from the accumulators (no finalize kernel); keys and their offsets go up in one copy
    const bool direct = cfg.queries_per_launch == 0 && db.stride == db.bytes;
    const WsLayout lay = ws_layout(cfg.queries_per_launch == 1 ? 1 : n, db.stride);
    const size_t out_bytes = size_t(n) * db.bytes;
    const size_t koff = (total + 15) & ~size_t(15), up = koff + size_t(n) * 4;
    const size_t stage = std::max(up, out_bytes);
    if (impir_status s = grow(&g_sync.d_keys, &g_sync.c_keys, up)) return s;
    if (impir_status s = grow(&g_sync.d_ws, &g_sync.c_ws, lay.total)) return s;
    if (!direct)
        if (impir_status s = grow(&g_sync.d_out, &g_sync.c_out, out_bytes)) return s;
    if (impir_status s = grow(reinterpret_cast<void**>(&g_sync.h_stage), &g_sync.c_stage, stage, true)) return s;
    std::memcpy(g_sync.h_stage, keys, total);
    std::memcpy(g_sync.h_stage + koff, offs.data(), size_t(n) * 4);
    cudaStream_t st = g_sync.stream;
    uint8_t* d_keys = static_cast<uint8_t*>(g_sync.d_keys);
    CK(cudaMemcpyAsync(d_keys, g_sync.h_stage, up, cudaMemcpyHostToDevice, st), "key upload");
    if (impir_status s = answer_async_impl(db, &cfg, d_keys, reinterpret_cast<const uint32_t*>(d_keys + koff), n,
                                           static_cast<uint8_t*>(g_sync.d_out), g_sync.d_ws, g_sync.c_ws, st, mode,
                                           direct, total))
        return s;
    const void* src = direct ? static_cast<const void*>(static_cast<uint8_t*>(g_sync.d_ws) + lay.off_acc) : g_sync.d_out;
    CK(cudaMemcpyAsync(g_sync.h_stage, src, out_bytes, cudaMemcpyDeviceToHost, st), "answer download");
    CK(cudaStreamSynchronize(st), "answer");
    std::memcpy(out, g_sync.h_stage, out_bytes);
    return bounds_verdict();
}

impir_status impir_answer(int32_t h, const uint8_t* keys, uint32_t n, uint8_t* out) {
    return answer_sync(h, keys, n, out, 0);
}

impir_status impir_answer_add32(int32_t h, const uint8_t* keys, uint32_t n, uint8_t* out) {
    return answer_sync(h, keys, n, out, 1);
}

impir_status impir_answer_add32_async(int32_t h, const uint8_t* d_keys, const uint32_t* d_off, uint32_t n,
                                      uint8_t* d_out, void* d_ws, size_t ws_bytes, void* stream) {
    Db db;
    if (impir_status s = get_db(h, &db)) return s;
    return answer_async_impl(db, nullptr, d_keys, d_off, n, d_out, d_ws, ws_bytes, static_cast<cudaStream_t>(stream), 1);
}

impir_status impir_get_config(int32_t h, uint32_t n_queries, impir_config* cfg) {
    if (!cfg) return fail(IMPIR_EINVAL, "NULL argument");
    Db db;
    if (impir_status s = get_db(h, &db)) return s;
    DeviceState* dev = nullptr;
    if (impir_status s = need_device(&dev)) return s;
    *cfg = config_for(db, n_queries ? n_queries : 1, dev->sms);
    return IMPIR_OK;
}

impir_status impir_get_config_add32(int32_t h, uint32_t n_queries, impir_config* cfg) {
    if (!cfg) return fail(IMPIR_EINVAL, "NULL argument");
    Db db;
    if (impir_status s = get_db(h, &db)) return s;
    DeviceState* dev = nullptr;
    if (impir_status s = need_device(&dev)) return s;
    const uint32_t n = n_queries ? n_queries : 1;
    *cfg = add_config(db.cfg_set ? db.cfg : default_add_config(db.n, db.stride / 16, n, dev->sms), db.stride / 16);
    return IMPIR_OK;
}

impir_status impir_set_config(int32_t h, const impir_config* cfg) {
    if (!cfg) return fail(IMPIR_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(g_db_mu);
    if (h < 1 || size_t(h) > g_dbs.size() || !g_dbs[h - 1].live) return fail(IMPIR_EINVAL, "unknown database handle %d", h);
    if (impir_status s = check_config(*cfg, g_dbs[h - 1].stride / 16)) return s;
    g_dbs[h - 1].cfg = *cfg;
    g_dbs[h - 1].cfg_set = true;
    return IMPIR_OK;
}

impir_status impir_autotune(int32_t h, const uint8_t* d_keys, const uint32_t* d_off, uint32_t n, uint8_t* d_out,
                            void* d_ws, size_t ws_bytes, void* stream, impir_config* best) {
    Db db;
    if (impir_status s = get_db(h, &db)) return s;
    DeviceState* dev = nullptr;
    if (impir_status s = need_device(&dev)) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const auto key = std::make_tuple(dev->sms, db.n, db.stride, n);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            if (best) *best = it->second;
            return impir_set_config(h, &it->second);
        }
    }
    const impir_config base = default_config(db.n, db.stride / 16, n, dev->sms);
    std::vector<impir_config> cands;
    for (uint32_t qpw : {1u, 2u, 4u, 8u, 16u}) {
        if (qpw > 1 && qpw / 2 >= n) continue;
        for (int ds = -3; ds <= 2; ++ds) {
            const int s = int(base.lane_bits) + ds;
            if (s < 0 || s > int(kMaxLaneBits)) continue;
            for (uint32_t w : {16u, 20u}) {
                impir_config c = base;
                c.queries_per_warp = qpw;
                c.lane_bits = uint32_t(s);
                c.warps_per_cta = w;
                if (check_config(c, db.stride / 16) == IMPIR_OK) cands.push_back(c);
            }
        }
    }
    g_err.clear();
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0), "event");
    CK(cudaEventCreate(&e1), "event");
    float best_ms = 1e30f;
    impir_config best_c = base;
    for (const impir_config& c : cands) {
        if (impir_status s = answer_async_impl(db, &c, d_keys, d_off, n, d_out, d_ws, ws_bytes, st)) return s;
        CK(cudaEventRecord(e0, st), "event record");
        if (impir_status s = answer_async_impl(db, &c, d_keys, d_off, n, d_out, d_ws, ws_bytes, st)) return s;
        CK(cudaEventRecord(e1, st), "event record");
        CK(cudaEventSynchronize(e1), "event sync");
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, e0, e1), "event time");
        if (ms < best_ms) {
            best_ms = ms;
            best_c = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[key] = best_c;
    }
    if (best) *best = best_c;
    return impir_set_config(h, &best_c);
}

// ---- databases larger than HBM: streamed in chunks (§3.3) ----

impir_status impir_answer_streamed(const void* records, uint64_t N, uint32_t B, const uint8_t* keys, uint32_t n,
                                   uint8_t* out, uint64_t chunk_bytes, impir_config* used) {
    if (!records || !keys || !out) return fail(IMPIR_EINVAL, "NULL argument");
    if (N == 0 || B == 0 || N > (1ull << IMPIR_MAX_DOMAIN_BITS)) return fail(IMPIR_EINVAL, "bad database size");
    if (B > 0xfffffff0u || !bytes_ok(N, (uint64_t(B) + 15u) & ~uint64_t(15)) ||
        !bytes_ok(n, (uint64_t(B) + 15u) & ~uint64_t(15)))
        return fail(IMPIR_EINVAL, "database or batch too large");
    if (n == 0) return IMPIR_OK;
    DeviceState* dev = nullptr;
    if (impir_status s = need_device(&dev)) return s;
    std::vector<uint32_t> offs;
    size_t total = 0;
    if (impir_status s = parse_host_keys(keys, n, offs, total)) return s;
    const uint32_t stride = (B + 15u) & ~15u, words = stride / 16;
    const impir_config cfg = default_config(N, words, n, dev->sms);
    if (used) *used = cfg;
    const uint64_t T = 32ull << cfg.lane_bits;  // warp tile: chunks hold whole tiles
    if (chunk_bytes == 0) chunk_bytes = 2ull << 30;  // default: 2 GiB (fewer launch tails, small first copy)
    uint64_t chunk = (chunk_bytes / stride) / T * T;
    if (chunk < T) chunk = T;
    if (chunk > N) chunk = (N + T - 1) / T * T;
    // chunk boundaries: a quarter-size first chunk (the only copy nothing overlaps), then full ones
    std::vector<uint64_t> bounds{0};
    const uint64_t first = std::max(T, chunk / 4 / T * T);
    for (uint64_t lo = 0; lo < N;) {
        lo = std::min(N, lo + (bounds.size() == 1 ? first : chunk));
        bounds.push_back(lo);
    }
    const uint64_t nchunks = bounds.size() - 1;
    // Two work schedules, one per compute stream, so that a chunk's launch can start on the SMs
    // the previous chunk's launch frees in its tail; both accumulate into the same answers. One
    // allocation [schedule 1 | schedule 0 | accumulators]: schedule 0 is the usual layout at
    // offset D = lay.off_acc, schedule 1 sits at offset 0 with its accumulator offset moved by D.
    const WsLayout lay = ws_layout(n, stride);
    WsLayout lay1 = lay;
    lay1.off_acc = 2 * lay.off_acc;
    lay1.total = lay.total + lay.off_acc;

    StreamCtx& X = g_streamed;
    std::lock_guard<std::mutex> lk(X.mu);
    if (cudaError_t e = streamed_ctx_init(X)) return cuda_fail(e, "streamed answer streams");
    const size_t buf_bytes = chunk * stride;
    const bool regrow = X.c_buf[0] < buf_bytes || X.c_buf[1] < buf_bytes;
    for (int i = 0; i < 2; ++i)
        if (impir_status s = grow(&X.d_buf[i], &X.c_buf[i], buf_bytes)) return s;
    if (impir_status s = grow(&X.d_keys, &X.c_keys, total)) return s;
    if (impir_status s = grow(&X.d_off, &X.c_off, size_t(n) * 4)) return s;
    if (impir_status s = grow(&X.d_ws, &X.c_ws, lay1.total)) return s;
    if (impir_status s = grow(&X.d_out, &X.c_out, size_t(n) * B)) return s;
    uint8_t* d_buf[2] = {static_cast<uint8_t*>(X.d_buf[0]), static_cast<uint8_t*>(X.d_buf[1])};
    uint8_t* d_keys = static_cast<uint8_t*>(X.d_keys);
    uint32_t* d_off = static_cast<uint32_t*>(X.d_off);
    uint8_t* d_ws = static_cast<uint8_t*>(X.d_ws);
    uint8_t* d_out = static_cast<uint8_t*>(X.d_out);
    cudaStream_t cs = X.cs, *ks = X.ks;
    cudaEvent_t *copied = X.copied, *consumed = X.consumed, ready = X.ready, done1 = X.done1;
    impir_status st = IMPIR_OK;
    cudaError_t e = cudaSuccess;
    // records with padding: the copies write B of every `stride` bytes, the rest must read as zero
    // (a call without padding writes whole rows and leaves the buffers' contents arbitrary)
    if (stride == B) {
        X.zeroed_stride = 0;
    } else if (regrow || X.zeroed_stride != stride) {
        for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaMemsetAsync(d_buf[i], 0, X.c_buf[i], cs);
        if (e == cudaSuccess) X.zeroed_stride = stride;
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_keys, keys, total, cudaMemcpyHostToDevice, ks[0]);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_off, offs.data(), size_t(n) * 4, cudaMemcpyHostToDevice, ks[0]);
    if (e != cudaSuccess) {
        X.zeroed_stride = 0;
        return cuda_fail(e, "streamed answer setup");
    }
    uint8_t* const ws_of[2] = {d_ws + lay.off_acc, d_ws};
    const WsLayout* const lay_of[2] = {&lay, &lay1};
    const uint8_t* src = static_cast<const uint8_t*>(records);
    for (uint64_t c = 0; c < nchunks && e == cudaSuccess; ++c) {
        const int b = int(c & 1);  // buffer, compute stream and schedule of this chunk
        const uint64_t lo = bounds[c], cnt = bounds[c + 1] - lo;
        // copy stream: refill buffer b once the launch two chunks back has read it
        if (c >= 2) e = cudaStreamWaitEvent(cs, consumed[b], 0);
        if (e == cudaSuccess)
            e = stride == B ? cudaMemcpyAsync(d_buf[b], src + lo * B, cnt * B, cudaMemcpyHostToDevice, cs)
                            : cudaMemcpy2DAsync(d_buf[b], stride, src + lo * B, B, B, cnt, cudaMemcpyHostToDevice, cs);
        if (e == cudaSuccess) e = cudaEventRecord(copied[b], cs);
        // compute stream b: this chunk's warp tiles, accumulating into the shared answers
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ks[b], copied[b], 0);
        // stream 1 starts after stream 0 has the keys and has zeroed the accumulators
        if (e == cudaSuccess && c == 1) e = cudaStreamWaitEvent(ks[1], ready, 0);
        if (e != cudaSuccess) break;
        SetupParams sp{};
        sp.keys = d_keys;
        sp.key_off = d_off;
        sp.ws = ws_of[b];
        sp.lay = *lay_of[b];
        sp.n_records = N;
        sp.n_queries = n;
        sp.words = words;
        sp.lane_bits = cfg.lane_bits;
        sp.qpw = cfg.queries_per_warp;
        sp.tile_lo = lo / T;
        sp.tile_hi = (lo + cnt + T - 1) / T;
        sp.keep_acc = c > 0;
        sp.bounds = bounds_record();
        sp.keys_bytes = total;
        e = launch_setup(sp, ks[b]);
        if (e == cudaSuccess && c == 0) e = cudaEventRecord(ready, ks[0]);
        FusedParams fp{};
        fp.db = reinterpret_cast<const uint4*>(d_buf[b]);
        fp.keys = d_keys;
        fp.key_off = d_off;
        fp.ws = ws_of[b];
        fp.te0 = dev->d_te0;
        fp.lay = *lay_of[b];
        fp.n_records = N;
        fp.n_queries = n;
        fp.words = words;
        fp.lane_bits = cfg.lane_bits;
        fp.bits_words = 1u << cfg.lane_bits;
        fp.rec_lo = lo;
        std::memcpy(fp.mmo_rk, dev->mmo_rk, sizeof fp.mmo_rk);
        fp.bounds = sp.bounds;
        fp.db_words = bounds_db_words(cnt * words, words);
        fp.keys_bytes = total;
        fp.smem_bytes = uint32_t(smem_for(cfg));
        if (e == cudaSuccess)
            e = launch_fused(cfg.queries_per_warp, nk_xor(words, cfg.queries_per_warp), dim3(dev->sms),
                             dim3(cfg.warps_per_cta * 32),
                             smem_for(cfg), ks[b], fp);
        if (e == cudaSuccess) e = cudaEventRecord(consumed[b], ks[b]);
        count_launches(2);
    }
    // join: stream 0 finalizes once stream 1's launches are done
    if (e == cudaSuccess) e = cudaEventRecord(done1, ks[1]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ks[0], done1, 0);
    if (e == cudaSuccess) {
        FinalizeParams zp{};
        zp.ws = ws_of[0];
        zp.lay = lay;
        zp.out = d_out;
        zp.n_queries = n;
        zp.record_bytes = B;
        zp.stride = stride;
        zp.bounds = bounds_record();
        e = launch_finalize(zp, ks[0]);
        count_launches(1);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, d_out, size_t(n) * B, cudaMemcpyDeviceToHost, ks[0]);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ks[0]);
    if (e != cudaSuccess) {
        // leave no work of this call behind on the cached streams
        cudaStreamSynchronize(cs);
        cudaStreamSynchronize(ks[0]);
        cudaStreamSynchronize(ks[1]);
        X.zeroed_stride = 0;
        st = cuda_fail(e, "streamed answer");
    }
    return st == IMPIR_OK ? bounds_verdict() : st;
}

// ---- tuning cache on disk ----

impir_status impir_tune_cache_save(const char* path) {
    if (!path) return fail(IMPIR_EINVAL, "NULL path");
    FILE* f = std::fopen(path, "w");
    if (!f) return fail(IMPIR_EINVAL, "cannot write %s", path);
    std::fprintf(f, "# impir tuning cache: sms n_records stride_bytes n_queries lane_bits queries_per_warp "
                    "warps_per_cta queries_per_launch\n");
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        for (const auto& kv : g_tune)
            std::fprintf(f, "%d %llu %u %u %u %u %u %u\n", std::get<0>(kv.first),
                         (unsigned long long)std::get<1>(kv.first), std::get<2>(kv.first), std::get<3>(kv.first),
                         kv.second.lane_bits, kv.second.queries_per_warp, kv.second.warps_per_cta,
                         kv.second.queries_per_launch);
    }
    std::fclose(f);
    return IMPIR_OK;
}

impir_status impir_tune_cache_load(const char* path, uint32_t* n_loaded) {
    if (!path) return fail(IMPIR_EINVAL, "NULL path");
    FILE* f = std::fopen(path, "r");
    if (!f) return fail(IMPIR_EINVAL, "cannot read %s", path);
    char line[512];
    uint32_t n = 0;
    while (std::fgets(line, sizeof line, f)) {
        if (line[0] == '#') continue;
        int sms;
        unsigned long long nrec;
        unsigned stride, nq;
        impir_config c{};
        if (std::sscanf(line, "%d %llu %u %u %u %u %u %u", &sms, &nrec, &stride, &nq, &c.lane_bits,
                        &c.queries_per_warp, &c.warps_per_cta, &c.queries_per_launch) != 8)
            continue;
        if (check_config(c, stride / 16) != IMPIR_OK) continue;  // skip entries this build cannot launch
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[std::make_tuple(sms, uint64_t(nrec), uint32_t(stride), uint32_t(nq))] = c;
        ++n;
    }
    std::fclose(f);
    g_err.clear();
    if (n_loaded) *n_loaded = n;
    return IMPIR_OK;
}

// ---- client side ----

impir_status impir_reconstruct(const uint8_t* r0, const uint8_t* r1, uint32_t record_bytes, uint8_t* out) {
    if (!r0 || !r1 || !out) return fail(IMPIR_EINVAL, "NULL argument");
    for (uint32_t b = 0; b < record_bytes; ++b) out[b] = r0[b] ^ r1[b];
    return IMPIR_OK;
}

impir_status dpf_gen(uint64_t alpha, uint32_t m, impir_prf prf, const uint8_t rng_seed[32], uint8_t* key0,
                     uint8_t* key1) {
    if (!rng_seed || !key0 || !key1) return fail(IMPIR_EINVAL, "NULL argument");
    if (m < 1 || m > IMPIR_MAX_DOMAIN_BITS) return fail(IMPIR_EINVAL, "domain bits %u outside 1..40", m);
    if (prf != IMPIR_PRF_AES_KEYED && prf != IMPIR_PRF_AES_MMO) return fail(IMPIR_EINVAL, "unknown prf");
    if (alpha >> m) return fail(IMPIR_EINVAL, "alpha >= 2^m");
    uint64_t state = 0;
    for (int w = 0; w < 4; ++w) {
        uint64_t v = 0;
        std::memcpy(&v, rng_seed + 8 * w, 8);  // little-endian hosts
        state ^= v;
    }
    auto next64 = [&state]() {
        uint64_t z = (state += 0x9e3779b97f4a7c15ull);
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
        return z ^ (z >> 31);
    };
    auto draw = [&](uint8_t out[16]) {
        uint64_t a = next64(), b = next64();
        std::memcpy(out, &a, 8);
        std::memcpy(out + 8, &b, 8);
    };
    uint32_t rk_mmo[2][44];
    host_aes_expand(reinterpret_cast<const uint8_t*>(IMPIR_MMO_KEY0), rk_mmo[0]);
    host_aes_expand(reinterpret_cast<const uint8_t*>(IMPIR_MMO_KEY1), rk_mmo[1]);
    auto prf_eval = [&](const uint8_t s[16], int x, uint8_t out[16]) {
        if (prf == IMPIR_PRF_AES_KEYED) {
            uint32_t rk[44];
            host_aes_expand(s, rk);
            uint8_t blk[16] = {0};
            blk[0] = uint8_t(x);
            host_aes_encrypt(rk, blk, out);
        } else {
            host_aes_encrypt(rk_mmo[x], s, out);
            for (int i = 0; i < 16; ++i) out[i] ^= s[i];
        }
    };
    const size_t kb = impir_key_bytes(m);
    std::memset(key0, 0, kb);
    std::memset(key1, 0, kb);
    key0[3] = 0;  // party indices
    key1[3] = 1;
    for (uint8_t* k : {key0, key1}) {
        k[0] = IMPIR_KEY_VERSION;
        k[1] = uint8_t(prf);
        k[2] = uint8_t(m);
    }
    auto cw = [m](uint8_t* k, int t, int x, uint32_t d) { return k + 8 + size_t(t) * 32 * (m + 1) + (size_t(x) * (m + 1) + d) * 16; };
    uint8_t pa[16], pb[16];
    draw(pa);
    draw(pb);
    pb[0] = uint8_t((pb[0] & 0xfe) | ((pa[0] & 1) ^ 1));
    std::memcpy(cw(key0, 0, 0, 0), pa, 16);
    std::memcpy(cw(key1, 0, 0, 0), pb, 16);
    for (uint32_t d = 1; d <= m; ++d) {
        const int a = pa[0] & 1;
        const int on = int((alpha >> (m - d)) & 1);
        uint8_t fa[2][16], fb[2][16];
        for (int x = 0; x < 2; ++x) {
            prf_eval(pa, x, fa[x]);
            prf_eval(pb, x, fb[x]);
            uint8_t r[16], delta[16] = {0};
            draw(r);
            if (d == m && x == on) r[0] = uint8_t((r[0] & 0xfe) | ((fa[x][0] & 1) ^ 1));  // lsb(R_A(m, alpha)) = 1
            if (x == on) {
                if (d < m) {
                    draw(delta);
                    delta[0] |= 1;
                } else {
                    delta[0] = 1;
                }
            }
            uint8_t* ca = cw(key0, a, x, d);
            uint8_t* cb = cw(key0, 1 - a, x, d);
            for (int i = 0; i < 16; ++i) {
                ca[i] = r[i];
                cb[i] = uint8_t(r[i] ^ fa[x][i] ^ fb[x][i] ^ delta[i]);
            }
        }
        for (int t = 0; t < 2; ++t)
            for (int x = 0; x < 2; ++x) std::memcpy(cw(key1, t, x, d), cw(key0, t, x, d), 16);
        const uint8_t* ca = cw(key0, a, on, d);
        const uint8_t* cb = cw(key0, 1 - a, on, d);
        for (int i = 0; i < 16; ++i) {
            pa[i] = fa[on][i] ^ ca[i];
            pb[i] = fb[on][i] ^ cb[i];
        }
    }
    return IMPIR_OK;
}

}  // extern "C"

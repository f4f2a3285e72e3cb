// serve.cpp — continuous-batching request loop over resident databases (the GB300 analog of
// the paper's query batching, §3.4: worker threads, a task queue, and scheduling threads
// that hand queries to DPU clusters).
//
// Requests (one DPF key each, for one of the registered databases) are queued by any
// thread. A dispatcher thread keeps up to `streams` batches in flight, one per CUDA stream.
// Whenever a stream is free it admits the oldest pending requests (all for the same
// database as the oldest one, up to max_batch of them, and only as many as the per-query
// accumulator budget still allows), uploads their keys, launches the fused answer on that
// stream and queues the answer download, so batches that arrive while others run overlap on
// the device. Finished batches are harvested by polling their events (host side only; no
// kernel waits on anything), and each answer is handed to whoever calls take().
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <set>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/impir.h"
#include "impir_internal.h"

namespace impir {
impir_status set_error(impir_status st, const char* msg);
}

using namespace impir;
using clk = std::chrono::steady_clock;

namespace {

struct Request {
    uint64_t tag;
    int32_t db;
    std::vector<uint8_t> key;
    clk::time_point t_submit;
};

struct Done {
    uint64_t tag;
    int32_t db;
    impir_status status;
    std::vector<uint8_t> answer;
    uint64_t latency_ns;
    uint32_t batch;
    uint64_t version;
};

// A bulk update waiting for an idle window of its database.
struct Update {
    int32_t db;
    uint64_t first, n;
    std::vector<uint8_t> records;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    uint8_t* d_keys = nullptr;
    uint32_t* d_off = nullptr;
    uint8_t* d_out = nullptr;
    uint8_t* d_ws = nullptr;
    size_t ws_bytes = 0;
    uint8_t* h_in = nullptr;   // pinned: keys then offsets
    uint8_t* h_out = nullptr;  // pinned: answers
    bool busy = false;
    std::vector<Request> reqs;
    uint32_t record_bytes = 0;
    uint64_t acc_bytes = 0;
    int32_t db = 0;
    uint64_t version = 0;
};

size_t max_key_bytes() { return impir_key_bytes(IMPIR_MAX_DOMAIN_BITS); }

}  // namespace

struct impir_server {
    impir_server_config cfg{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request> pending;
    std::deque<Done> done;
    std::deque<Update> updates;
    std::map<int32_t, uint32_t> inflight_per_db;
    cudaStream_t upd_stream = nullptr;
    uint64_t updates_applied = 0;
    std::vector<Slot> slots;
    uint64_t inflight_acc = 0;
    uint64_t batches = 0, queries = 0;
    uint32_t inflight_batches = 0, max_inflight_batches = 0;
    std::atomic<bool> stop{false};
    std::thread th;
};

namespace {

void free_slot(Slot& s) {
    if (s.stream) cudaStreamDestroy(s.stream);
    if (s.done) cudaEventDestroy(s.done);
    cudaFree(s.d_keys);
    cudaFree(s.d_off);
    cudaFree(s.d_out);
    cudaFree(s.d_ws);
    cudaFreeHost(s.h_in);
    cudaFreeHost(s.h_out);
    s = Slot{};
}

// Collects finished batches; called with the lock held.
void harvest(impir_server* S) {
    for (Slot& s : S->slots) {
        if (!s.busy) continue;
        const cudaError_t q = cudaEventQuery(s.done);
        if (q == cudaErrorNotReady) continue;
        const auto now = clk::now();
        for (size_t i = 0; i < s.reqs.size(); ++i) {
            Done d;
            d.tag = s.reqs[i].tag;
            d.db = s.reqs[i].db;
            d.status = q == cudaSuccess ? IMPIR_OK : IMPIR_ECUDA;
            d.answer.assign(s.h_out + i * s.record_bytes, s.h_out + (i + 1) * s.record_bytes);
            d.latency_ns = uint64_t(std::chrono::duration_cast<std::chrono::nanoseconds>(now - s.reqs[i].t_submit).count());
            d.batch = uint32_t(s.reqs.size());
            d.version = s.version;
            S->done.push_back(std::move(d));
        }
        S->inflight_acc -= s.acc_bytes;
        S->inflight_batches -= 1;
        S->inflight_per_db[s.db] -= 1;
        s.reqs.clear();
        s.busy = false;
        S->cv_done.notify_all();
    }
}

// Applies queued bulk updates, oldest first, as long as their database has no batch in
// flight (lock held). The copy completes before any later batch on that database launches.
void apply_updates(impir_server* S) {
    while (!S->updates.empty()) {
        Update& u = S->updates.front();
        if (S->inflight_per_db[u.db] > 0) break;
        uint64_t v = 0;
        if (impir_db_update_async(u.db, u.first, u.n, u.records.data(), S->upd_stream, &v) == IMPIR_OK)
            cudaStreamSynchronize(S->upd_stream);
        S->updates.pop_front();
        S->updates_applied += 1;
    }
}

// Admits and launches as many batches as free slots and the budget allow (lock held).
// Requests for a database with a pending update wait until the update is applied.
void launch_ready(impir_server* S) {
    std::set<int32_t> blocked;
    for (const Update& u : S->updates) blocked.insert(u.db);
    for (Slot& s : S->slots) {
        if (s.busy || S->pending.empty()) continue;
        auto first = S->pending.begin();
        while (first != S->pending.end() && blocked.count(first->db)) ++first;
        if (first == S->pending.end()) break;
        const int32_t db = first->db;
        uint64_t n_records = 0;
        uint32_t rb = 0, stride = 0;
        const void* dptr = nullptr;
        uint64_t version = 0;
        if (impir_db_info(db, &n_records, &rb, &stride, &dptr) != IMPIR_OK || impir_db_version(db, &version) != IMPIR_OK) {
            // the database went away: fail that request
            Request r = std::move(*first);
            S->pending.erase(first);
            Done d{r.tag, r.db, IMPIR_EINVAL, {}, 0, 0, 0};
            S->done.push_back(std::move(d));
            S->cv_done.notify_all();
            continue;
        }
        const uint64_t budget_left = S->cfg.accumulator_budget > S->inflight_acc ? S->cfg.accumulator_budget - S->inflight_acc : 0;
        uint32_t cap = S->cfg.max_batch;
        if (uint64_t(cap) * stride > budget_left) cap = uint32_t(budget_left / stride);
        if (cap == 0) break;  // wait for in-flight batches to release accumulator memory
        // oldest request first, then later ones for the same database, in arrival order
        std::vector<Request> take;
        for (auto it = first; it != S->pending.end() && take.size() < cap;) {
            if (it->db == db) {
                take.push_back(std::move(*it));
                it = S->pending.erase(it);
            } else {
                ++it;
            }
        }
        const uint32_t n = uint32_t(take.size());
        size_t off = 0;
        uint32_t* offs = reinterpret_cast<uint32_t*>(s.h_in + size_t(S->cfg.max_batch) * max_key_bytes());
        for (uint32_t i = 0; i < n; ++i) {
            std::memcpy(s.h_in + off, take[i].key.data(), take[i].key.size());
            offs[i] = uint32_t(off);
            off += take[i].key.size();
        }
        cudaError_t e = cudaMemcpyAsync(s.d_keys, s.h_in, off, cudaMemcpyHostToDevice, s.stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(s.d_off, offs, size_t(n) * 4, cudaMemcpyHostToDevice, s.stream);
        impir_status st = e == cudaSuccess ? impir_answer_async(db, s.d_keys, s.d_off, n, s.d_out, s.d_ws, s.ws_bytes, s.stream)
                                           : IMPIR_ECUDA;
        if (st == IMPIR_OK)
            e = cudaMemcpyAsync(s.h_out, s.d_out, size_t(n) * rb, cudaMemcpyDeviceToHost, s.stream);
        if (st == IMPIR_OK && e == cudaSuccess) e = cudaEventRecord(s.done, s.stream);
        if (st != IMPIR_OK || e != cudaSuccess) {
            for (Request& r : take) {
                Done d{r.tag, r.db, st != IMPIR_OK ? st : IMPIR_ECUDA, {}, 0, n, version};
                S->done.push_back(std::move(d));
            }
            S->cv_done.notify_all();
            continue;
        }
        s.reqs = std::move(take);
        s.record_bytes = rb;
        s.acc_bytes = uint64_t(n) * stride;
        s.db = db;
        s.version = version;
        S->inflight_per_db[db] += 1;
        s.busy = true;
        S->inflight_acc += s.acc_bytes;
        S->inflight_batches += 1;
        if (S->inflight_batches > S->max_inflight_batches) S->max_inflight_batches = S->inflight_batches;
        S->batches += 1;
        S->queries += n;
    }
}

void dispatcher(impir_server* S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (!S->stop.load()) {
        harvest(S);
        apply_updates(S);
        launch_ready(S);
        const bool any_busy = S->inflight_batches > 0;
        if (any_busy) {
            // short host-side poll interval while batches run
            S->cv_work.wait_for(lk, std::chrono::microseconds(20));
        } else if (S->pending.empty() && S->updates.empty()) {
            S->cv_work.wait_for(lk, std::chrono::milliseconds(2));
        }
    }
    // drain: let in-flight batches finish so their buffers can be freed
    for (Slot& s : S->slots)
        if (s.busy) cudaEventSynchronize(s.done);
    harvest(S);
}

}  // namespace

extern "C" {

impir_status impir_server_create(const impir_server_config* cfg, impir_server** out) {
    if (!cfg || !out) return set_error(IMPIR_EINVAL, "NULL argument");
    if (cfg->max_batch == 0 || cfg->streams == 0 || cfg->streams > 64 || cfg->max_record_bytes == 0)
        return set_error(IMPIR_EINVAL, "server needs max_batch >= 1, 1..64 streams and max_record_bytes >= 1");
    const uint32_t stride = (cfg->max_record_bytes + 15u) & ~15u;
    if (cfg->accumulator_budget < stride) return set_error(IMPIR_EINVAL, "accumulator budget below one record");
    impir_server* S = new impir_server;
    S->cfg = *cfg;
    cudaGetDevice(&S->device);
    S->slots.resize(cfg->streams);
    const size_t kb = size_t(cfg->max_batch) * max_key_bytes();
    for (Slot& s : S->slots) {
        s.ws_bytes = impir_workspace_bytes(cfg->max_batch, stride);
        cudaError_t e = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&s.d_keys), kb);
        if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&s.d_off), size_t(cfg->max_batch) * 4);
        if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&s.d_out), size_t(cfg->max_batch) * stride);
        if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&s.d_ws), s.ws_bytes);
        if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&s.h_in), kb + size_t(cfg->max_batch) * 4);
        if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&s.h_out), size_t(cfg->max_batch) * stride);
        if (e != cudaSuccess) {
            cudaGetLastError();
            for (Slot& t : S->slots) free_slot(t);
            delete S;
            return set_error(IMPIR_ENOMEM, "server buffers could not be allocated");
        }
    }
    if (cudaStreamCreateWithFlags(&S->upd_stream, cudaStreamNonBlocking) != cudaSuccess) {
        for (Slot& t : S->slots) free_slot(t);
        delete S;
        return set_error(IMPIR_ENOMEM, "server update stream could not be created");
    }
    S->th = std::thread(dispatcher, S);
    *out = S;
    return IMPIR_OK;
}

impir_status impir_server_submit(impir_server* S, int32_t db, const uint8_t* key, uint64_t tag) {
    if (!S || !key) return set_error(IMPIR_EINVAL, "NULL argument");
    const uint32_t m = key[2];
    if (key[0] != IMPIR_KEY_VERSION || key[1] > 1 || m < 1 || m > IMPIR_MAX_DOMAIN_BITS || key[3] > 1)
        return set_error(IMPIR_EINVAL, "malformed key header");
    for (int i = 4; i < 8; ++i)
        if (key[i]) return set_error(IMPIR_EINVAL, "malformed key header");
    uint32_t rb = 0;
    if (impir_db_info(db, nullptr, &rb, nullptr, nullptr) != IMPIR_OK) return set_error(IMPIR_EINVAL, "unknown database");
    if (rb > S->cfg.max_record_bytes) return set_error(IMPIR_EINVAL, "database records larger than the server's maximum");
    Request r;
    r.tag = tag;
    r.db = db;
    r.key.assign(key, key + impir_key_bytes(m));
    r.t_submit = clk::now();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->pending.push_back(std::move(r));
    }
    S->cv_work.notify_one();
    return IMPIR_OK;
}

impir_status impir_server_take(impir_server* S, uint32_t timeout_us, uint64_t* tag, int32_t* db, uint8_t* answer,
                               uint32_t answer_capacity, uint32_t* answer_bytes, uint64_t* latency_ns,
                               uint32_t* batch_size, uint64_t* db_version) {
    if (!S) return set_error(IMPIR_EINVAL, "NULL server");
    std::unique_lock<std::mutex> lk(S->mu);
    if (!S->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), [S] { return !S->done.empty(); }))
        return set_error(IMPIR_ETIMEOUT, "no finished request within the timeout");
    Done d = std::move(S->done.front());
    S->done.pop_front();
    lk.unlock();
    if (tag) *tag = d.tag;
    if (db) *db = d.db;
    if (latency_ns) *latency_ns = d.latency_ns;
    if (batch_size) *batch_size = d.batch;
    if (db_version) *db_version = d.version;
    if (answer_bytes) *answer_bytes = uint32_t(d.answer.size());
    if (d.status != IMPIR_OK) return set_error(d.status, "request failed");
    if (d.answer.size() > answer_capacity) return set_error(IMPIR_EINVAL, "answer buffer too small");
    if (answer) std::memcpy(answer, d.answer.data(), d.answer.size());
    return IMPIR_OK;
}

impir_status impir_server_stats(impir_server* S, uint64_t* batches, uint64_t* queries,
                                uint32_t* max_inflight_batches, uint32_t* pending) {
    if (!S) return set_error(IMPIR_EINVAL, "NULL server");
    std::lock_guard<std::mutex> lk(S->mu);
    if (batches) *batches = S->batches;
    if (queries) *queries = S->queries;
    if (max_inflight_batches) *max_inflight_batches = S->max_inflight_batches;
    if (pending) *pending = uint32_t(S->pending.size());
    return IMPIR_OK;
}

impir_status impir_server_destroy(impir_server* S) {
    if (!S) return set_error(IMPIR_EINVAL, "NULL server");
    S->stop.store(true);
    S->cv_work.notify_all();
    if (S->th.joinable()) S->th.join();
    for (Slot& s : S->slots) free_slot(s);
    if (S->upd_stream) cudaStreamDestroy(S->upd_stream);
    delete S;
    return IMPIR_OK;
}

impir_status impir_server_update(impir_server* S, int32_t db, uint64_t first_record, uint64_t n_records,
                                 const void* records) {
    if (!S || (!records && n_records)) return set_error(IMPIR_EINVAL, "NULL argument");
    uint64_t n = 0;
    uint32_t rb = 0;
    if (impir_db_info(db, &n, &rb, nullptr, nullptr) != IMPIR_OK) return set_error(IMPIR_EINVAL, "unknown database");
    if (first_record > n || n_records > n - first_record) return set_error(IMPIR_EINVAL, "update range beyond the database");
    Update u;
    u.db = db;
    u.first = first_record;
    u.n = n_records;
    const uint8_t* p = static_cast<const uint8_t*>(records);
    u.records.assign(p, p + n_records * rb);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->updates.push_back(std::move(u));
    }
    S->cv_work.notify_one();
    return IMPIR_OK;
}

}  // extern "C"

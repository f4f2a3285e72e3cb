/*
 * impir.h — C ABI of the GB300 server side of two-server DPF-based PIR (IM-PIR,
 * arXiv 2509.06514): full-domain DPF evaluation fused with dpXOR on one GPU.
 *
 * Conventions for every call below:
 *   - Every call returns an impir_status; nothing throws across this boundary.
 *     On failure impir_last_error() gives a thread-local message.
 *   - The caller owns every buffer it passes. The library owns a database's device
 *     copy from impir_db_load until impir_db_free (impir_db_attach borrows instead).
 *   - "Host" pointers are ordinary CPU memory; "device" pointers are CUDA global memory
 *     of the current device (for example a torch CUDA tensor's data_ptr()).
 *   - Synchronous calls return only after their outputs are written.
 *
 * Key wire format (little-endian), the DPF key of §3.1: two codewords
 * C_0, C_1 in F_{2^128}^{2 x (m+1)}.
 *   byte 0   version, must be IMPIR_KEY_VERSION (1)
 *   byte 1   prf, an impir_prf
 *   byte 2   m, the domain bits, 1..IMPIR_MAX_DOMAIN_BITS; the domain is 2^m leaves
 *   byte 3   party index b (0 or 1): which server the key is for; only the additive
 *            answer (impir_answer_add32) uses it
 *   bytes 4..7 zero
 *   then C_0[2][m+1][16] and C_1[2][m+1][16]: [row = child bit x][column = depth d].
 *   Column 0 holds only the root seed C_0[0][0]; C_0[1][0], C_1[0][0] and C_1[1][0]
 *   must be zero. Total impir_key_bytes(m) = 8 + 64 (m + 1) bytes.
 *
 * A key with domain bits m is answered over records [0, min(2^m, N)): leaves j >= N
 * select nothing, and a key with 2^m < N covers the DB prefix its domain spans.
 */
#ifndef IMPIR_H
#define IMPIR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    IMPIR_OK = 0,
    IMPIR_EINVAL = 1,   /* malformed argument or key; nothing was launched */
    IMPIR_ENOMEM = 2,   /* host or device allocation failed, or a workspace is too small */
    IMPIR_ECUDA = 3,    /* a CUDA runtime call failed (no device, launch error, ...) */
    IMPIR_ETIMEOUT = 4, /* a bounded wait gave up (serving loop) */
    IMPIR_EBUSY = 5     /* the resource is in use (for example a DB with queries in flight) */
} impir_status;

/* The PRF of Eq. (3). The paper's PRF_s(x) "encrypts x with key s" (§3.2): AES-128 keyed
 * by the 128-bit parent seed s over the block enc(x) (byte 0 = x, other bytes 0).
 * IMPIR_PRF_AES_MMO is the fixed-key alternative PRF_s(x) = AES_{K_x}(s) XOR s with the
 * two fixed keys below (Matyas-Meyer-Oseas). */
typedef enum { IMPIR_PRF_AES_KEYED = 0, IMPIR_PRF_AES_MMO = 1 } impir_prf;

#define IMPIR_KEY_VERSION 1
#define IMPIR_MAX_DOMAIN_BITS 40
/* K_0 and K_1 of IMPIR_PRF_AES_MMO: the ASCII strings "IM-PIR MMO key 0" / "... 1". */
#define IMPIR_MMO_KEY0 "IM-PIR MMO key 0"
#define IMPIR_MMO_KEY1 "IM-PIR MMO key 1"

/* Size in bytes of one key with domain bits m: 8 + 64 (m + 1). */
size_t impir_key_bytes(uint32_t m);

/* ---- Database (§3.3 "Database preloading": copied once, resident, not timed) ---- */

/* Copies n_records records of record_bytes each from host memory `records` (row-major,
 * contiguous) into device memory owned by the library, padding each record to a
 * 16-byte-aligned stride with zero bytes. On success *db_handle names the database.
 * EINVAL: records NULL, n_records 0, record_bytes 0, or n_records > 2^40.
 * ENOMEM: the device allocation failed. */
impir_status impir_db_load(const void* records, uint64_t n_records, uint32_t record_bytes, int32_t* db_handle);

/* Registers a database that already lives in device memory (for example a torch tensor):
 * record j starts at d_records + j * stride_bytes. stride_bytes must be a multiple of 16
 * and >= record_bytes, d_records 16-byte aligned, and the padding bytes of every record
 * must be zero. The library does not copy or free it; it must outlive the handle. */
impir_status impir_db_attach(const void* d_records, uint64_t n_records, uint32_t record_bytes,
                             uint32_t stride_bytes, int32_t* db_handle);

/* Releases the handle (and the device copy if impir_db_load made it). EINVAL: unknown handle. */
impir_status impir_db_free(int32_t db_handle);

/* Describes a database: record count, record bytes, device stride and device pointer. */
impir_status impir_db_info(int32_t db_handle, uint64_t* n_records, uint32_t* record_bytes, uint32_t* stride_bytes,
                           const void** d_records);

/* ---- Row shards (a database split by rows across GPUs, the 1-D block layout of §3.3; the
 * servers' per-shard results are combined like the partial results of Algorithm 1) ---- */

/* Shard boundaries are multiples of this many records (so that no warp tile straddles two
 * shards, whatever the launch shape). */
#define IMPIR_SHARD_ALIGN 32768u

/* Loads rows [row_lo, row_lo + n_rows) of a database of n_total records (host memory
 * `records` holds just those rows, record_bytes each) into a new handle, like impir_db_load.
 * Every answer on the handle (impir_answer, impir_answer_async, impir_answer_add32[_async],
 * the server) is the partial answer over these rows only: a query with domain bits m covers
 * global records [0, min(2^m, n_total)), of which this shard contributes the ones it holds.
 * XOR of the shards' XOR answers (sum mod 2^32 of their additive answers), see
 * impir_combine_partials, is the full answer. Bulk updates address rows relative to row_lo.
 * EINVAL: row_lo not a multiple of IMPIR_SHARD_ALIGN, row_lo + n_rows beyond n_total, or an
 * end that is neither n_total nor a multiple of IMPIR_SHARD_ALIGN; ENOMEM as impir_db_load. */
impir_status impir_db_load_rows(const void* records, uint64_t n_rows, uint32_t record_bytes, uint64_t row_lo,
                                uint64_t n_total, int32_t* db_handle);

/* The row range of a handle: its first global row and the whole database's record count
 * (0 and n_records for a handle that is not a shard). */
impir_status impir_db_rows(int32_t db_handle, uint64_t* row_lo, uint64_t* n_total);

/* Combines n_parts partial answers on the device: d_parts holds them back to back,
 * part_bytes each (e.g. n_queries * record_bytes); d_out (part_bytes) receives their XOR
 * (mode 0, the XOR answer) or their sum mod 2^32 word by word (mode 1, the additive answer;
 * part_bytes a multiple of 4 and both pointers 4-byte aligned). Asynchronous on cuda_stream.
 * d_out may not overlap d_parts. EINVAL: bad mode, sizes or alignment. */
impir_status impir_combine_partials(int mode, const uint8_t* d_parts, uint32_t n_parts, uint64_t part_bytes,
                                    uint8_t* d_out, void* cuda_stream);

/* ---- Bulk updates (§3.3: a stable version answers queries while bulk updates are applied
 * in windows when the database is idle) ----
 * Records [first_record, first_record + n_records) are replaced by n_records records of
 * record_bytes each from host memory `records` (row-major). Every update increments the
 * database's version (0 after loading). impir_db_update waits for all work on the device to
 * finish, copies, and returns when later answers will see the new records. The _async form
 * only enqueues the copy on `cuda_stream` and bumps the version: the caller must order it
 * after the answers that should see the old records and before those that should see the
 * new ones, and keep `records` valid until the copy completes. EINVAL: unknown handle or a
 * range beyond the database. */
impir_status impir_db_update(int32_t db_handle, uint64_t first_record, uint64_t n_records, const void* records);
impir_status impir_db_update_async(int32_t db_handle, uint64_t first_record, uint64_t n_records, const void* records,
                                   void* cuda_stream, uint64_t* new_version);
impir_status impir_db_version(int32_t db_handle, uint64_t* version);

/* ---- Answering (Algorithm 1: EvaluateDPF + TaskletXOR + MasterXOR + Aggregate) ---- */

/* Answers n_queries keys against one database: for each key k,
 *   out[q] = XOR over j < min(N, 2^m) of lsb(Eval(k, j)) * D[j]          (§2.3, §3.3)
 * with Eval(k, j) = R(m, j) of Eqs. (1)-(3). `keys` is host memory holding the n_queries
 * keys back to back (each impir_key_bytes(m) long, m read from its header; keys of
 * different m may be mixed). `out` is host memory of n_queries * record_bytes bytes.
 * All keys are validated before any launch: one malformed key gives EINVAL and no output.
 * The keys go to the device, one batched fused launch answers all of them, and the
 * answers come back; the call returns when `out` is written. */
impir_status impir_answer(int32_t db_handle, const uint8_t* keys, uint32_t n_queries, uint8_t* out);

/* The additive (inner-product) answer of §2.2 over Z_2^32, reconstructed by the client as
 * r_0 + r_1: records are read as vectors of little-endian 32-bit words (record_bytes must be
 * a multiple of 4) and the key's party index b (header byte 3) selects the share
 *   out[q] = sum over j < min(N, 2^m) of (-1)^b * low32(Eval(k, j)) * D[j]   (mod 2^32, per word)
 * where low32 is bytes 0..3 of the 128-bit leaf read little-endian. Keys from dpf_gen give
 * r_0 + r_1 = D[alpha]. Same arguments and errors as impir_answer / impir_answer_async, plus
 * EINVAL when record_bytes is not a multiple of 4. Launch shape (impir_get_config_add32): the
 * database's configuration narrowed to 1 or 2 queries per warp tile (2 for records up to
 * 2 KiB) and, for records above 512 bytes, at most 16 warps; any lane_bits (the 32-bit shares
 * are kept in shared memory for 32 / queries leaves per lane at a time and scanned chunk by
 * chunk). */
impir_status impir_answer_add32(int32_t db_handle, const uint8_t* keys, uint32_t n_queries, uint8_t* out);
impir_status impir_answer_add32_async(int32_t db_handle, const uint8_t* d_keys, const uint32_t* d_key_offsets,
                                      uint32_t n_queries, uint8_t* d_out, void* d_workspace, size_t workspace_bytes,
                                      void* cuda_stream);

/* Device workspace an asynchronous answer of n_queries keys against a database of
 * record stride stride_bytes needs (bytes). */
size_t impir_workspace_bytes(uint32_t n_queries, uint32_t stride_bytes);

/* Asynchronous form on a caller stream with caller-owned device memory; it allocates
 * nothing and never synchronizes, so it can be captured into a CUDA graph.
 *   d_keys         device, the keys back to back
 *   d_key_offsets  device, n_queries uint32 byte offsets of each key inside d_keys
 *   d_out          device, n_queries * record_bytes bytes, written
 *   d_workspace    device, >= impir_workspace_bytes(n_queries, stride), 256-byte aligned
 *   cuda_stream    a cudaStream_t (NULL = the legacy default stream)
 * Keys are validated on the device: a malformed key's answer is all zero and the first
 * such query index is recorded; read it with impir_workspace_status after the stream
 * completes. The device checks each key's header, column 0 and 8-byte alignment, not the
 * extent of d_keys (the call has no length for it): the caller guarantees that every offset
 * starts a whole key, impir_key_bytes(m) bytes for the m in its header, inside d_keys.
 * Launch errors return ECUDA. */
impir_status impir_answer_async(int32_t db_handle, const uint8_t* d_keys, const uint32_t* d_key_offsets,
                                uint32_t n_queries, uint8_t* d_out, void* d_workspace, size_t workspace_bytes,
                                void* cuda_stream);

/* Reads the device-side status of the last asynchronous answer that used d_workspace
 * (synchronizes with the device). *n_bad = number of malformed keys, *first_bad = the
 * smallest index among them (UINT32_MAX when none). */
impir_status impir_workspace_status(const void* d_workspace, uint32_t* n_bad, uint32_t* first_bad);

/* ---- Launch configuration and autotuning ---- */

/* Shape of the fused launch (the GPU analog of the paper's tasklets, DPU clusters and
 * subtree split, §3.2-§3.4):
 *   lane_bits          each lane expands a perfect subtree of 2^lane_bits leaves
 *                      (a warp tile is 32 * 2^lane_bits records); 0..10
 *   queries_per_warp   queries evaluated per warp tile before one shared scan of the
 *                      tile (1, 2, 4, 8, or 16 for records of at most 512 bytes): the DB
 *                      tile is read once for all of them (records above 512 bytes in column
 *                      passes of up to 16 / queries_per_warp 16-byte words per lane)
 *   warps_per_cta      4..16; up to 20 for records of at most 512 bytes and at most 8
 *                      queries per warp
 *   queries_per_launch 0 = the whole batch in one persistent launch; 1 = the plain
 *                      one-query-per-launch form (one launch per key, in order) */
typedef struct {
    uint32_t lane_bits;
    uint32_t queries_per_warp;
    uint32_t warps_per_cta;
    uint32_t queries_per_launch;
} impir_config;

/* Gets the configuration a batch of n_queries keys would be launched with on this database
 * (the one set or tuned for it, else the built-in default for that batch size), or sets one
 * for all later batches (set validates it: EINVAL). */
impir_status impir_get_config(int32_t db_handle, uint32_t n_queries, impir_config* cfg);
impir_status impir_set_config(int32_t db_handle, const impir_config* cfg);

/* The launch shape impir_answer_add32[_async] would use for a batch of n_queries keys on this
 * database: the configuration set or tuned for it narrowed to the additive kernels (1 or 2
 * queries per warp tile; at most 16 warps for records above 512 bytes), else the additive
 * default. */
impir_status impir_get_config_add32(int32_t db_handle, uint32_t n_queries, impir_config* cfg);

/* Times candidate configurations on the given asynchronous problem (same arguments as
 * impir_answer_async, which it runs repeatedly on cuda_stream), keeps the fastest for
 * this database, writes it to *best and records it in the process-wide tuning cache
 * keyed by (SM count, N, stride, batch size, largest m). Synchronizes the stream. */
impir_status impir_autotune(int32_t db_handle, const uint8_t* d_keys, const uint32_t* d_key_offsets,
                            uint32_t n_queries, uint8_t* d_out, void* d_workspace, size_t workspace_bytes,
                            void* cuda_stream, impir_config* best);

/* ---- Databases larger than device memory ---- */

/* Database larger than device memory (§3.3: evaluate the linear operations over the DB in
 * batches of chunks): answers n_queries host keys against n_records records of record_bytes
 * each that stay in host memory `records`, streaming them through the device in chunks of
 * about chunk_bytes (0: 2 GiB; rounded to whole warp tiles; the first chunk a quarter of that), two
 * chunk buffers deep, the copy of one chunk overlapping the fused launches on earlier ones.
 * Consecutive chunks alternate between two compute streams with their own work schedules, so
 * one chunk's launch starts on the SMs the previous one frees; per-query accumulators are
 * shared and persist across chunks. Same answers as impir_answer on the same records. Pinned
 * host memory (cudaHostAlloc / cudaHostRegister) lets the copies run at full link bandwidth.
 * `out` is host memory of n_queries * record_bytes bytes; *used (may be NULL) receives the
 * launch shape. The two chunk buffers (2 x chunk_bytes of device memory), the workspace, the
 * streams and the events are allocated by the first call that needs them and kept for later
 * calls (grown when a call needs more); calls are serialised on an internal lock. ENOMEM when
 * the buffers cannot be allocated. */
impir_status impir_answer_streamed(const void* records, uint64_t n_records, uint32_t record_bytes,
                                   const uint8_t* keys, uint32_t n_queries, uint8_t* out, uint64_t chunk_bytes,
                                   impir_config* used);

/* Saves the process-wide tuning cache to a text file (one entry per line), or merges a saved
 * one into it (*n_loaded: entries accepted; lines this build cannot launch are skipped), so a
 * later process's impir_autotune returns without timing anything. EINVAL: unreadable or
 * unwritable path. */
impir_status impir_tune_cache_save(const char* path);
impir_status impir_tune_cache_load(const char* path, uint32_t* n_loaded);

/* ---- Serving: continuous batching over resident databases (§3.4 query batching) ----
 * A server owns `streams` CUDA streams, each with device buffers for one batch of up to
 * max_batch queries. Any thread may submit requests (one key for one registered database,
 * tagged by the caller). A dispatcher thread admits the oldest pending requests into the next
 * batch as soon as a stream is free and the per-query accumulator memory in flight stays
 * within accumulator_budget (a batch of n queries on a database of stride S holds n*S bytes),
 * taking further pending requests for the same database in arrival order; it launches the
 * fused answer on that stream, so batches that arrive while others run overlap on the device.
 * Each result is the same as answering that key alone. No kernel waits on anything; the
 * dispatcher polls batch completion events on the host. */
typedef struct impir_server impir_server;
typedef struct {
    uint32_t max_batch;          /* most queries one launch takes (>= 1) */
    uint32_t streams;            /* batches in flight at once, one CUDA stream each (1..64) */
    uint32_t max_record_bytes;   /* largest record of any database the server will answer */
    uint32_t reserved;           /* zero */
    uint64_t accumulator_budget; /* device bytes of in-flight per-query accumulators (>= one stride) */
} impir_server_config;

/* Creates a server on the current device (allocates its stream buffers up front).
 * EINVAL: bad configuration; ENOMEM: buffers could not be allocated. */
impir_status impir_server_create(const impir_server_config* cfg, impir_server** server);

/* Queues one request: `key` is host memory holding one wire key (copied before return),
 * `db_handle` a loaded database, `tag` any caller value returned with the answer.
 * EINVAL: malformed key header, unknown database, or records beyond max_record_bytes. */
impir_status impir_server_submit(impir_server* server, int32_t db_handle, const uint8_t* key, uint64_t tag);

/* Waits up to timeout_us for any finished request and returns it: its tag, database, answer
 * (copied into `answer`, record_bytes of its database, at most answer_capacity), the latency
 * from submit to completion in nanoseconds, the size of the batch it ran in, and the version
 * of the database the answer was computed on (see impir_db_update).
 * ETIMEOUT: nothing finished in time. A request that failed returns its failure status
 * (with its tag filled in). */
impir_status impir_server_take(impir_server* server, uint32_t timeout_us, uint64_t* tag, int32_t* db_handle,
                               uint8_t* answer, uint32_t answer_capacity, uint32_t* answer_bytes,
                               uint64_t* latency_ns, uint32_t* batch_size, uint64_t* db_version);

/* Queues a bulk update of records [first_record, first_record + n_records) of a database
 * (host `records`, copied before return). The dispatcher applies queued updates in order, each
 * as soon as no batch on its database is in flight; requests for that database wait until it
 * is applied, so every answer is computed on one whole version. EINVAL: unknown database or a
 * range beyond it. */
impir_status impir_server_update(impir_server* server, int32_t db_handle, uint64_t first_record, uint64_t n_records,
                                 const void* records);

/* Counters: batches launched, queries launched, most batches in flight at once, requests
 * still waiting for admission. */
impir_status impir_server_stats(impir_server* server, uint64_t* batches, uint64_t* queries,
                                uint32_t* max_inflight_batches, uint32_t* pending);

/* Stops the dispatcher after the batches in flight finish, and frees the server. */
impir_status impir_server_destroy(impir_server* server);

/* ---- Client side, used by tests (§3.1 Gen, §2.3 reconstruction) ---- */

/* Gen(alpha) for domain bits m: writes key0 and key1 (impir_key_bytes(m) each) such that
 * Eval(key0, j) XOR Eval(key1, j) is the 128-bit integer 1 at j = alpha and 0 elsewhere.
 * Randomness: SplitMix64 seeded with the XOR of the four little-endian 64-bit words of
 * rng_seed (draw order: the two roots, then per depth and child bit a uniform codeword
 * and, on the path above the leaves, a uniform offset with lsb 1). key0 is party 0 and
 * key1 party 1; the leaf codeword on the path is chosen so that lsb(Eval(key0, alpha)) = 1,
 * which makes the additive shares (-1)^b low32(Eval(key_b, j)) sum to exactly 1 at alpha.
 * EINVAL: m outside 1..40, alpha >= 2^m, unknown prf, NULL buffers. */
impir_status dpf_gen(uint64_t alpha, uint32_t m, impir_prf prf, const uint8_t rng_seed[32], uint8_t* key0,
                     uint8_t* key1);

/* D[i] = r0 XOR r1 (§2.3): the client combines the two servers' answers. */
impir_status impir_reconstruct(const uint8_t* r0, const uint8_t* r1, uint32_t record_bytes, uint8_t* out);

/* Thread-local message describing the last failure on this thread ("" if none). */
const char* impir_last_error(void);

/* ---- Answering without any allocation ----
 * The paper has no counterpart to this call; it exists for callers that may not allocate
 * device memory at the moment they answer (code running inside an allocator or memory-pool
 * callback, a process whose device memory a framework reserved up front, or a path that must
 * not risk the implicit synchronization of cudaMalloc/cudaFree). It computes exactly what
 * impir_answer_async computes, on a database given by pointer (no handle), with keys, key
 * offsets and answers in caller-owned device memory, but takes no workspace: its scratch is
 * a fixed array of IMPIR_NOALLOC_SCRATCH_BYTES in the library's device memory, present on
 * every GPU that loads the library until the process exits.
 *   - It calls no cudaMalloc, cudaFree or other allocating routine.
 *   - The batch must fit: the workspace of impir_workspace_bytes(n_queries, stride_bytes)
 *     must be <= IMPIR_NOALLOC_SCRATCH_BYTES, else EINVAL and nothing is launched.
 *   - The first call on a device does a one-time set-up for that device: it looks up the
 *     scratch array's device address, uploads a 1 KiB AES table, and prepares every kernel a
 *     later call can launch (sets their shared-memory limit on that device and loads their
 *     code, which with lazy module loading could otherwise take device memory at a later
 *     call). Make that first call before any stream capture; later calls do no set-up work.
 *   - The launch shape is the one impir_answer_async picks by default for the same database
 *     size, record stride and batch size.
 *   - Every call shares the one scratch array, which keeps the last call's contents (each
 *     call clears what must start at zero). Calls whose kernels overlap on the GPU race on
 *     it: issue them on one stream, or otherwise order them.
 * d_records: n_records records, record j at d_records + j * stride_bytes (stride a multiple
 * of 16, >= record_bytes, padding bytes zero, 16-byte aligned). Malformed keys give zero
 * answers, as in impir_answer_async (their status is not reported here). */
#define IMPIR_NOALLOC_SCRATCH_BYTES (8u << 20)
impir_status impir_answer_noalloc(const void* d_records, uint64_t n_records, uint32_t record_bytes,
                                  uint32_t stride_bytes, const uint8_t* d_keys, const uint32_t* d_key_offsets,
                                  uint32_t n_queries, uint8_t* d_out, void* cuda_stream);

/* ---- Kernel timing (measurement support; off by default) ----
 * While enabled, each fused EvalAll + dpXOR launch is bracketed by two CUDA events recorded
 * on the stream it is launched on. impir_timing_read waits for those events and returns the
 * summed device time of the fused launches (milliseconds), their count, and the count of
 * every kernel the library launched (setup, fused, finalize) since the last enable.
 * Do not enable it while a stream is being captured into a CUDA graph. */
impir_status impir_timing_enable(int enable);
impir_status impir_timing_read(double* fused_ms, uint64_t* fused_launches, uint64_t* all_launches);

/* AES-only calibration (measurement support; the paper has no counterpart): runs the fused
 * kernel's PRF engine with nothing around it. Each of n_threads threads (threads_per_cta per
 * CTA, a multiple of 32, <= 512) starts from its 16-byte seed in `seeds` (host) and applies
 * iters times p <- PRF_p(0) XOR PRF_p(1) with the given prf; the final states go to `out`
 * (host, n_threads * 16 bytes) and *ms receives the device time of the timed launch
 * (2 * iters * n_threads AES-128 blocks). Allocates and frees its own device buffers. */
impir_status impir_aes_calibrate(int prf, uint32_t iters, uint32_t n_threads, uint32_t threads_per_cta,
                                 const uint8_t* seeds, uint8_t* out, double* ms);

/* Bitsliced AES calibration (measurement support; the paper has no counterpart): the same
 * iteration p <- PRF_p(0) XOR PRF_p(1) for the fixed-key PRF (IMPIR_PRF_AES_MMO), computed by an
 * engine with no table lookups: AES on bit-slices, each thread carrying 16 seeds under both keys
 * in 32-bit words (one logic operation advances 32 AES computations; the S-box is a 154-gate
 * composite-field circuit). seeds: n_threads * 16 seeds of 16 bytes (host), thread g taking seeds
 * 16g .. 16g + 15; out receives the final states in the same layout; *ms the device time of the
 * timed launch (2 * iters * 16 * n_threads AES-128 blocks). threads_per_cta: a multiple of 32,
 * <= 256. Allocates and frees its own device buffers. */
impir_status impir_aes_calibrate_bitsliced(uint32_t iters, uint32_t n_threads, uint32_t threads_per_cta,
                                           const uint8_t* seeds, uint8_t* out, double* ms);

/* Index checks of the debug build (measurement and test support; the paper has no
 * counterpart). A library compiled with IMPIR_BOUNDS (libimpir_bounds.so, built by
 * `python -m paper_2509_06514_gb300.build --bounds`) compares every shared-memory, database
 * record, key, query, schedule and accumulator index its kernels use with the extent of its
 * buffer before the access; a failed check skips the access (a load reads zero) and is
 * recorded per device and in the launch's workspace header. Nothing traps or waits. Its
 * synchronous calls (impir_answer, impir_answer_add32, impir_answer_streamed) return ECUDA
 * when a check failed during the call. This call waits for the device, then returns the
 * number of failed checks since the last call, the site code and index of the first one
 * (sites: 1 T-table, 2 selection-bit/node/share buffer, 3 database word, 4 key byte, 5 query
 * index, 6 schedule, 7 accumulator word, 8 lane stack, 9 setup writes, 10 answer byte), and
 * clears the record. EINVAL in a library built without IMPIR_BOUNDS. For testing the checks
 * themselves, the debug library reads IMPIR_BOUNDS_TEST_WITHHOLD_RECORDS=k from the environment
 * and withholds the last k records of every database from the checked extent (their memory stays
 * valid), so that reads of them fail the check; the normal library ignores it. */
impir_status impir_bounds_status(uint32_t* n_failed, uint32_t* first_site, uint64_t* first_index);

/* Number of streaming multiprocessors of the current device (0 if none). */
int32_t impir_device_sm_count(void);

#ifdef __cplusplus
}
#endif

#endif /* IMPIR_H */

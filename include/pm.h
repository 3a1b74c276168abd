/*
 * pm.h -- C ABI of libpm: multi-pattern matching by the parallel
 * failure-less Aho-Corasick (PFAC) scan over a compressed-row-storage trie,
 * on one GB300 GPU (sm_103a).
 *
 * Problem (Section II-B of "Trie Compression for GPU Accelerated
 * Multi-Pattern Matching"): find the patterns of a set P in a text T.
 * Method (Section II-C): one walk starts at every byte of T, follows the
 * pattern trie while the text keeps matching and terminates at the first
 * mismatch -- no failure links. Trie (Section III): built breadth-first,
 * stored pointer-free in BFS order and compressed as compressed row storage
 * (row_ptr, sorted byte column, next state), 2*nnz+n+1 elements.
 *
 * Output of a scan, for every start position i of a text:
 *   ids[i] = id of the longest pattern p with T[i .. i+|p|) == p, else -1;
 *   count  = number of (start position, distinct pattern) occurrences.
 * A pattern's id is the index of its first occurrence in the list given to
 * pm_build; later duplicates are dropped. A walk never crosses the end of
 * its own text (no padding, no wrap-around).
 *
 * Conventions
 *  - Every function returns PM_OK (0) or a negative PM_ERR_* code and also
 *    records it for pm_last_error() on the calling thread. No C++ exception
 *    crosses this boundary.
 *  - Pointers named d_* are CUDA device pointers on the current device;
 *    h_* are host pointers. The caller owns every buffer it passes; libpm
 *    owns only what a pm_trie, pm_server or pm_scanner handle holds.
 *  - pm_stream is the CUDA stream type (CUstream_st *, identical to
 *    cudaStream_t); NULL is the legacy default stream. Scans are
 *    asynchronous on that stream.
 *  - Errors raised inside a kernel (a bounded wait that ran out, a bounds
 *    violation in the checked scan) are recorded in a device word and
 *    reported by pm_device_error(); the kernel returns instead of trapping.
 */
#ifndef PM_H
#define PM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------ */
#define PM_OK                    0
#define PM_ERR_INVAL            -1  /* bad argument (null, size, alignment)   */
#define PM_ERR_NOMEM            -2  /* host or device allocation failed       */
#define PM_ERR_EMPTY_PATTERN    -3  /* a pattern of length 0                  */
#define PM_ERR_PATTERN_TOO_LONG -4  /* a pattern longer than PM_MAX_PATTERN_LEN */
#define PM_ERR_CUDA             -5  /* a CUDA runtime call failed             */
#define PM_ERR_TIMEOUT          -6  /* a bounded wait ran out                 */
#define PM_ERR_BOUNDS           -7  /* checked scan saw an out-of-range index */
#define PM_ERR_BUSY             -8  /* serving: no slot or arena space now    */
#define PM_ERR_NOT_FOUND        -9  /* serving: unknown request id            */
#define PM_ERR_HOST_ONLY       -10  /* handle has no device copy              */

#define PM_MAX_PATTERN_LEN 4096u

typedef struct CUstream_st *pm_stream;
typedef struct pm_trie pm_trie;

/* Result buffers of one scan, both caller-owned DEVICE memory:
 *   ids   int32[len], one entry per start position;
 *   count int64[1], overwritten (not accumulated) by the scan. */
typedef struct {
    int32_t *ids;
    int64_t *count;
} pm_result;

/* Sizes of a built trie (Section III; Section V for the 36-byte node). */
typedef struct {
    uint64_t n_patterns;     /* distinct patterns (= final nodes)               */
    uint64_t n_duplicates;   /* input patterns dropped as repeats               */
    uint64_t n_nodes;        /* trie nodes including the root (CRS rows n)      */
    uint64_t nnz;            /* CRS non-zeros = trie edges = n_nodes - 1        */
    uint32_t min_len;        /* shortest pattern (0 if none)                    */
    uint32_t max_len;        /* longest pattern = trie depth                    */
    uint32_t alphabet;       /* byte classes C: bytes used by patterns, +1 for  */
                             /* "any other byte" unless all 256 are used        */
    uint32_t dense_k_max;    /* deepest level with shared-memory tables         */
    uint64_t crs_elements;   /* 2*nnz + n + 1 (Section III's storage count)     */
    uint64_t csr_bytes;      /* row_ptr u32[n+1] + col u8[nnz] + next i32[nnz]  */
                             /* + final_id i32[n]                               */
    uint64_t dense256_bytes; /* uncompressed 256-wide state table: 256*4*n      */
    uint64_t bitmap36_bytes; /* 256-bit bitmap + 4-byte offset per node: 36*n   */
    uint64_t device_bytes;   /* everything the handle holds on the device      */
    uint64_t deep_bytes;     /* deep level table (0 if none)                    */
    uint32_t deep_k;         /* depth of the deep level read from L2: the root  */
                             /* paths of that depth as a bitmap with ranks;     */
                             /* byte-class tries only, 0 if none               */
} pm_trie_stats;

/* Launch configuration of the scan kernel (picked by an autotuner). Every
 * warp of a CTA is an independent pipeline over its own text tiles: it
 * stages them, tests each start position in the shared-memory filter, and
 * walks the positions that remain in rounds of 32 (one per lane) from its
 * own queue. */
typedef struct {
    int32_t threads;      /* threads per CTA: a multiple of 32, 128 .. 1024   */
    int32_t tile;         /* text bytes per warp tile: a multiple of          */
                          /* 32 * positions, 256 .. 32768                     */
    int32_t dense_k;      /* byte alphabet: trie levels resolved before a     */
                          /* walk, 0 .. dense_k_max (< shortest pattern);     */
                          /* byte classes: depth F of the filter's grams,     */
                          /* 0 (none) .. dense_k_max (<= shortest pattern)    */
    int32_t filter_bits;  /* byte alphabet: filter width per k-gram, 8, 16 or */
                          /* 32; byte classes: 8                              */
    int32_t row_search;   /* 0: linear, 1: binary search of the byte column   */
    int32_t ctas_per_sm;  /* persistent grid = SMs * ctas_per_sm (0: maximum) */
    int32_t stages;       /* tiles in flight per warp (TMA), 2..4             */
    int32_t checked;      /* 1: bounds-checked scan (PM_ERR_BOUNDS on error)  */
    int32_t positions;    /* start positions per lane and group: 4 or 8, or   */
                          /* 16 for the byte alphabet at dense_k 2 and for    */
                          /* 2-bit classes at dense_k 10 with the deep level  */
                          /* of depth 13                                      */
    int32_t deep;         /* byte classes: 1: positions passing the filter    */
                          /* look up the deep level before walking, 0: they  */
                          /* walk from the root; byte alphabet: 0             */
    int32_t layout;       /* trie form the walks read: 0 CRS row records (16  */
                          /* bytes a node), 1 the bitmapped node of Section  */
                          /* III (256-bit child bitmap + first child, 36 B)  */
    int32_t wait_clocks;  /* bound of each wait for a staged tile, in SM      */
                          /* clocks; 0: the default, about 2 s. A wait that  */
                          /* runs out records PM_ERR_TIMEOUT (pm_device_error) */
                          /* and ends the scan early                          */
    int32_t light_max;    /* single texts of at most this many bytes take the */
                          /* light launch form (small CTAs, no shared tables, */
                          /* four positions per thread, walks in place); 0:   */
                          /* never                                            */
    int32_t schedule;     /* which tiles a warp scans: PM_SCHED_AUTO, _STATIC */
                          /* or _DYNAMIC (below)                              */
} pm_config;

/* pm_config.schedule. STATIC: warp w of the grid scans tiles w, w + W,
 * w + 2W, ... (W warps). DYNAMIC: CTAs take runs of PM_CHUNK_TILES
 * consecutive tiles from a global counter, in text order, and their warps
 * take the run's tiles one at a time as they finish one; the whole grid then
 * sweeps the text as one front and a warp slowed by walks takes fewer tiles.
 * The counter is 4 bytes of stream-ordered device memory per launch (from a
 * pool the library keeps); a stream being captured into a graph always
 * takes STATIC. AUTO: STATIC, which measured as fast or faster on the
 * workloads this library is tuned on. */
#define PM_SCHED_AUTO    0
#define PM_SCHED_STATIC  1
#define PM_SCHED_DYNAMIC 2
#define PM_CHUNK_TILES   32u

/* ---- trie construction (Section III, steps I, II, VI and the CRS step) --
 * Builds the trie of patterns[0..n) (lengths[j] bytes each; any byte value,
 * NUL included) breadth-first with children in ascending byte order,
 * compresses it to CRS, derives the dense prefix tables of the top levels,
 * and copies everything to the current CUDA device. Inputs are copied; the
 * caller may free them on return. n == 0 is allowed (nothing ever matches).
 * *footprint_bytes (optional) receives csr_bytes.
 * Errors: PM_ERR_INVAL (null pointers with n > 0, out == NULL),
 *         PM_ERR_EMPTY_PATTERN, PM_ERR_PATTERN_TOO_LONG, PM_ERR_NOMEM,
 *         PM_ERR_CUDA (no device, copy failed). *out is NULL on error. */
int pm_build(const uint8_t *const *patterns, const uint32_t *lengths, uint32_t n,
             pm_trie **out, uint64_t *footprint_bytes);

/* As pm_build, but keeps the trie on the host only (no CUDA call is made):
 * for footprint reports and host-side checks. Scans on such a handle fail
 * with PM_ERR_HOST_ONLY. */
int pm_build_host(const uint8_t *const *patterns, const uint32_t *lengths,
                  uint32_t n, pm_trie **out, uint64_t *footprint_bytes);

/* Frees the handle and its device memory. NULL is ignored. The caller must
 * ensure no scan on it is still running, and destroy or close the servers
 * and scanners made from it first (they keep a pointer to it). */
void pm_free(pm_trie *h);

/* Sizes of the trie. Errors: PM_ERR_INVAL. */
int pm_stats(const pm_trie *h, pm_trie_stats *s);

/* Host copies of the CRS arrays (Section III): row_ptr u32[n+1], col
 * u8[nnz] (ascending within each row), next i32[nnz] (child node), final_id
 * i32[n] (-1 if no pattern ends at the node). Any output may be NULL.
 * Sizes come from pm_stats. Errors: PM_ERR_INVAL. */
int pm_export_csr(const pm_trie *h, uint32_t *row_ptr, uint8_t *col,
                  int32_t *next, int32_t *final_id);

/* The handle's current launch configuration / replace it after validation.
 * pm_set_config must not run concurrently with scans on the handle.
 * Errors: PM_ERR_INVAL (a field out of range). */
int pm_get_config(const pm_trie *h, pm_config *cfg);
int pm_set_config(pm_trie *h, const pm_config *cfg);

/* ---- scans (Section II-C) ----------------------------------------------
 * pm_scan: one text d_text[0..len) (device memory, any alignment). Writes
 * out.ids[0..len) and *out.count, asynchronously on `stream`. len == 0 is
 * legal (count 0). The handle is read-only during scans, so concurrent scans
 * on different streams are safe; out.ids must not alias the text. A text
 * (and a batch's total) is below 2^40 bytes.
 * Errors: PM_ERR_INVAL (null pointers with len > 0, len >= 2^40), PM_ERR_HOST_ONLY,
 *         PM_ERR_CUDA (launch failed). */
int pm_scan(const pm_trie *h, const uint8_t *d_text, uint64_t len,
            pm_result out, pm_stream stream);

/* pm_scan_range: the start positions [start, end) of a device text of which
 * the bytes d_text[0 .. limit) may be read (end <= limit). Walks from those
 * positions stop at `limit`, not at `end`: with limit = end + longest
 * pattern - 1 (clipped to the text), a range of a long text scanned on its
 * own gives exactly the ids and count that a scan of the whole text gives
 * for those positions (the overlap rule of Section II-B). That is how a text
 * is sharded over several GPUs: each rank holds its range plus that halo.
 * Writes out.ids[0 .. end - start) and *out.count (the occurrences starting
 * in the range), asynchronously on `stream`. start == end is legal.
 * Errors: PM_ERR_INVAL (start > end, end > limit, null pointers with
 * end > start, limit - start >= 2^40), PM_ERR_HOST_ONLY, PM_ERR_CUDA. */
int pm_scan_range(const pm_trie *h, const uint8_t *d_text, uint64_t start, uint64_t end,
                  uint64_t limit, pm_result out, pm_stream stream);

/* pm_scan_batch: ntexts texts stored back to back in d_texts; text t is
 * d_texts[d_offsets[t] .. d_offsets[t+1]) with d_offsets a DEVICE array of
 * ntexts+1 non-decreasing u64 starting at 0. Writes d_ids[0 .. total)
 * (same offsets as the texts) and d_counts[0..ntexts) (overwritten). One
 * persistent launch, no host synchronisation; can be captured in a CUDA
 * graph. Matches never cross a text boundary.
 * Errors: PM_ERR_INVAL, PM_ERR_HOST_ONLY, PM_ERR_CUDA. */
int pm_scan_batch(const pm_trie *h, const uint8_t *d_texts,
                  const uint64_t *d_offsets, uint32_t ntexts,
                  int32_t *d_ids, int64_t *d_counts, pm_stream stream);

/* As pm_scan_batch with an explicit configuration (NULL: the handle's) and
 * an optional DEVICE u64 d_lookups that receives the number of trie
 * transitions attempted (slower instrumented kernel; for the roofline's
 * trie term). With d_offsets == NULL the input is one text of `len` bytes
 * and d_counts has one entry; otherwise `len` is ignored. */
int pm_scan_ex(const pm_trie *h, const uint8_t *d_texts,
               const uint64_t *d_offsets, uint32_t ntexts, uint64_t len,
               int32_t *d_ids, int64_t *d_counts, uint64_t *d_lookups,
               const pm_config *cfg, pm_stream stream);

/* pm_scan_walks: pm_scan of one device text with an explicit configuration
 * (NULL: the handle's) that also counts, into the DEVICE u64 *d_walks
 * (overwritten), the walks it queued: the start positions the truncated
 * levels (filter, dense tables, deep level) could not settle. Every other
 * position was decided without a CRS walk.
 * Errors: as pm_scan_ex. */
int pm_scan_walks(const pm_trie *h, const uint8_t *d_text, uint64_t len, int32_t *d_ids,
                  int64_t *d_count, uint64_t *d_walks, const pm_config *cfg,
                  pm_stream stream);

/* ---- all matches (Sections II-B and II-C: every occurrence) --------------
 * One occurrence: pattern `id` (the index of its first occurrence in the
 * pattern list) of `len` bytes occurs at text position `pos`. */
typedef struct {
    uint64_t pos;
    int32_t id;
    int32_t len;
} pm_match;

/* Bytes of device workspace pm_scan_all needs for a text of len bytes
 * (a match count per 1024 positions, a bit per position, plus two counts
 * per 1 Mi positions). */
uint64_t pm_scan_all_work_bytes(uint64_t len);

/* pm_scan_all: pm_scan of one device text (out.ids and *out.count as
 * there) plus every occurrence, written to d_matches[0 .. min(count,
 * capacity)) ordered by position and, at one position, longer pattern first
 * (the patterns occurring at a position are all prefixes of the longest).
 * *out.count is the total; when it exceeds capacity the list stops after
 * `capacity` entries (scan again with a larger buffer). d_work: caller-owned
 * DEVICE workspace of at least pm_scan_all_work_bytes(len) bytes, 256-byte
 * aligned, overwritten. Asynchronous on `stream`, no host synchronisation.
 * Errors: PM_ERR_INVAL (null pointers, workspace too small or unaligned,
 * len >= 2^40), PM_ERR_HOST_ONLY, PM_ERR_CUDA. */
int pm_scan_all(const pm_trie *h, const uint8_t *d_text, uint64_t len, pm_result out,
                pm_match *d_matches, uint64_t capacity, void *d_work, uint64_t work_bytes,
                pm_stream stream);

/* pm_scan_all_host: every occurrence in a HOST text h_text[0..len), listed in
 * HOST memory: h_matches[0 .. min(count, capacity)) in the order of
 * pm_scan_all (position, then the longer pattern first) and *h_count = the
 * total. Only the list comes back (16 bytes per occurrence), not the 4 bytes
 * per position that pm_scan_host returns. The text is cut into chunks that
 * overlap by max_len - 1 bytes (Section II-B's overlap rule); copies in,
 * scans, listings and copies out are pipelined over the handle's two
 * internal streams with device buffers owned by the handle (shared with
 * pm_scan_host; the list buffers grow to the largest chunk's list). Pinned
 * host memory gives full copy speed. Blocks until the list is on the host.
 * Not reentrant per handle.
 * Errors: PM_ERR_INVAL, PM_ERR_HOST_ONLY, PM_ERR_NOMEM, PM_ERR_CUDA. */
int pm_scan_all_host(pm_trie *h, const uint8_t *h_text, uint64_t len, pm_match *h_matches,
                     uint64_t capacity, uint64_t *h_count);

/* ---- streams of chunks (Section II-B's overlap rule) ---------------------
 * A scanner scans one long text that arrives in chunks (a packet or file
 * stream) as if it were scanned whole. It holds back the last max_len - 1
 * bytes of what it has seen (the carry) together with the start positions
 * whose walks could still reach bytes not yet pushed.
 *
 * pm_scanner_push appends the DEVICE chunk d_chunk[0 .. len) and resolves
 * every start position whose walk lies inside the bytes seen so far: all
 * positions below (bytes pushed) - (max_len - 1), in stream order, starting
 * with the held ones. Their ids go to d_ids[0 .. *n_ids) (d_ids holds at
 * least len + max_len - 1 entries). *d_count is the number of occurrences
 * among them, overwritten. *n_ids (HOST) is set before the call returns.
 * The positions before a chunk boundary are scanned on a small copy of the
 * carry and the chunk's first max_len - 1 bytes; the chunk's own positions
 * are scanned in place.
 * pm_scanner_finish ends the stream: the held positions are resolved with
 * the stream's true end, and the scanner is ready for a new stream.
 * Calls are asynchronous on `stream`. A scanner is used from one stream and
 * one thread at a time; the chunk must stay valid until the push's work on
 * the stream is done. Chunks up to 16 MiB are copied behind the carry into
 * a scanner buffer and scanned in one launch; that buffer grows, stream
 * ordered, to the largest such chunk. pm_scanner_close waits for the
 * scanner's work on its last stream, then frees it.
 * Errors: PM_ERR_INVAL, PM_ERR_HOST_ONLY (open), PM_ERR_NOMEM, PM_ERR_CUDA. */
typedef struct pm_scanner pm_scanner;
int pm_scanner_open(const pm_trie *h, pm_scanner **out);
int pm_scanner_push(pm_scanner *s, const uint8_t *d_chunk, uint64_t len, int32_t *d_ids,
                    int64_t *d_count, uint64_t *n_ids, pm_stream stream);
int pm_scanner_finish(pm_scanner *s, int32_t *d_ids, int64_t *d_count, uint64_t *n_ids,
                      pm_stream stream);
int pm_scanner_close(pm_scanner *s);

/* ---- host buffers ---------------------------------------------------------
 * pm_scan_host: scans a HOST text h_text[0..len) and returns the results in
 * host memory (h_ids int32[len], *h_count). The text is cut into chunks
 * that overlap by max_len-1 bytes (Section II-B's overlap rule); copies in,
 * scans and copies out are pipelined over two internal streams using device
 * buffers owned by the handle. Pinned host memory gives full copy speed.
 * Blocks until the results are on the host. Not reentrant per handle.
 * Errors: PM_ERR_INVAL, PM_ERR_HOST_ONLY, PM_ERR_NOMEM, PM_ERR_CUDA. */
int pm_scan_host(pm_trie *h, const uint8_t *h_text, uint64_t len,
                 int32_t *h_ids, int64_t *h_count);

/* ---- host buffers, no device allocation ----------------------------------
 * pm_scan_host_static: pm_scan_host for callers that cannot let a library
 * allocate device memory: processes whose device memory belongs to one
 * allocator (a framework's caching allocator, or an arena reserved up front)
 * where a raw cudaMalloc/cudaFree would bypass or exceed it, and
 * latency-sensitive callers for whom cudaMalloc/cudaFree add long, often
 * device-synchronising stalls on the request path. The paper has no
 * counterpart: this is a service of the library, not part of the method.
 * The text (at most PM_STATIC_MAX_LEN bytes), its ids and its count are
 * staged in one statically sized device array inside libpm (about 5 MiB).
 * CUDA places the array on a GPU when the library's module that holds it is
 * loaded there: at the first pm_scan_host_static call on that GPU under the
 * default lazy module loading, at context creation when modules are loaded
 * eagerly. It stays until the process exits. No cudaMalloc, cudaFree or
 * allocating library routine is called. The caller
 * passes the host text h_text[0..len) and receives h_ids int32[len] and
 * *h_count; the copies and the scan run on `stream` (NULL: the legacy
 * default stream) and the call returns once the results are on the host.
 * The first call on a device looks up the array's device address for that
 * device (cudaGetSymbolAddress, with that device current) and keeps it for
 * the life of the process; make that first call before any stream capture
 * on the device. cudaDeviceReset after that first call is not supported:
 * the kept address would belong to the destroyed context.
 * Every call uses the same array, which keeps the last call's contents;
 * each call overwrites all its ids and zeroes the count first. Calls whose
 * work overlaps on the GPU (other streams, other host threads) race on the
 * array: serialise them.
 * Errors: PM_ERR_INVAL (null pointers, len > PM_STATIC_MAX_LEN, current
 * device is not the handle's), PM_ERR_HOST_ONLY, PM_ERR_CUDA. */
#define PM_STATIC_MAX_LEN (1ull << 20)
int pm_scan_host_static(const pm_trie *h, const uint8_t *h_text, uint64_t len,
                        int32_t *h_ids, int64_t *h_count, pm_stream stream);

/* ---- serving: continuous batching (a service of the library; the paper has
 * a single batch-free scan, Section II-C) ----------------------------------
 * A server keeps the trie resident and runs a scheduler thread that
 *  - admits submitted requests in arrival order as batch slots and device
 *    memory (a first-fit arena for request texts) free up,
 *  - launches everything admitted at that moment as one batched scan (one
 *    persistent kernel over a device offset table) whose ids and counts go
 *    straight to each request's own device buffers,
 *  - runs up to max_inflight batches at once, each on its own stream, so new
 *    requests overlap with those already on the GPU,
 *  - marks requests done when their batch's event completes.
 * Results are bit-identical to scanning each request alone with pm_scan. */
typedef struct pm_server pm_server;

typedef struct {
    uint64_t arena_bytes;     /* device bytes for texts in flight (0: 256 MiB)  */
    uint32_t max_inflight;    /* batches on the GPU at once, 1..64 (0: 4)       */
    uint32_t max_batch;       /* requests per batch (0: 1024)                   */
    uint64_t max_batch_bytes; /* text bytes per batch, a larger single request  */
                              /* still runs alone (0: 64 MiB)                   */
    uint32_t max_queue;       /* submitted, not yet admitted (0: 65536)         */
} pm_server_config;

typedef struct {
    uint64_t submitted, completed, batches, bytes;
    uint64_t max_batch_seen;     /* most requests in one batch                 */
    uint64_t max_inflight_seen;  /* most batches on the GPU at once            */
    uint64_t admission_waits;    /* times a request waited for arena memory    */
} pm_server_stats;

/* Creates a server for a built trie (device handle) on the current device,
 * which must be the trie's. cfg may be NULL (defaults). The handle must
 * outlive the server. Errors: PM_ERR_INVAL, PM_ERR_HOST_ONLY, PM_ERR_NOMEM. */
int pm_server_create(const pm_trie *h, const pm_server_config *cfg, pm_server **out);

/* Queues a scan of the HOST text h_text[0..len) (it must stay valid and
 * unchanged until the request is done; pinned memory copies fastest) with
 * results to caller-owned DEVICE buffers out.ids int32[len] and out.count
 * int64[1]. Returns at once with *req_id. Thread-safe.
 * Errors: PM_ERR_INVAL (NULLs, len > arena_bytes), PM_ERR_BUSY (queue full),
 * PM_ERR_CUDA (the server failed). */
int pm_submit(pm_server *s, const uint8_t *h_text, uint64_t len, pm_result out,
              uint64_t *req_id);

/* *done = 1 once the request's results are in its buffers; a done request
 * is reported once and then forgotten. Errors: PM_ERR_NOT_FOUND, or the
 * request's own error (PM_ERR_CUDA). */
int pm_poll(pm_server *s, uint64_t req_id, int *done);

/* Blocks until the request is done or timeout_ms passes (PM_ERR_TIMEOUT);
 * then as pm_poll with done = 1. */
int pm_wait(pm_server *s, uint64_t req_id, uint32_t timeout_ms);

int pm_server_get_stats(pm_server *s, pm_server_stats *st);

/* Finishes every submitted request, stops the scheduler and frees the
 * server's memory. Returns PM_ERR_CUDA if the server had failed. */
int pm_server_destroy(pm_server *s);

/* Trace replay for benchmarks, timed natively: request i (host text
 * h_texts[i], lens[i] bytes, outputs d_ids[i], d_counts[i]) is submitted at
 * arrival_ns[i] after the start; latency_ns[i] = completion seen on the host
 * minus that scheduled arrival; *wall_ns = start to the last completion. */
int pm_server_replay(pm_server *s, uint32_t n, const uint8_t *const *h_texts,
                     const uint64_t *lens, const uint64_t *arrival_ns,
                     int32_t *const *d_ids, int64_t *const *d_counts,
                     uint64_t *latency_ns, uint64_t *wall_ns);

/* The same trace served plainly: each request, at its arrival, is copied to
 * its own device buffer d_texts[i] and scanned by its own pm_scan launch on
 * `stream` (no batching, no overlap beyond one stream). */
int pm_replay_plain(const pm_trie *h, uint32_t n, const uint8_t *const *h_texts,
                    const uint64_t *lens, const uint64_t *arrival_ns,
                    uint8_t *const *d_texts, int32_t *const *d_ids,
                    int64_t *const *d_counts, uint64_t *latency_ns,
                    uint64_t *wall_ns, pm_stream stream);

/* ---- errors ------------------------------------------------------------ */
/* Reads and clears the device-side error word (synchronises the device):
 * *code = PM_OK, PM_ERR_TIMEOUT or PM_ERR_BOUNDS. Errors: PM_ERR_CUDA. */
int pm_device_error(int *code);
const char *pm_strerror(int code);   /* static string, never NULL          */
int pm_last_error(void);             /* last code returned on this thread  */
const char *pm_last_error_msg(void); /* detail for it, thread-local string */

#ifdef __cplusplus
}
#endif
#endif /* PM_H */

/*
 * psort.h -- C ABI of libpsort, a GB300 (sm_103a) parallel samplesort.
 *
 * The library implements the four-step parallel samplesort of Tokuue &
 * Ishiyama, "Performance Evaluation of Parallel Sortings on the Supercomputer
 * Fugaku" (arXiv 2305.05245), Sec. 2:
 *   1. sort each of n_B contiguous blocks of length ceil(N/n_B);
 *   2. select n_P-1 pivots, by regular sampling (PSRS, Sec. 2.3) or by
 *      exact splitting (PSES, Sec. 2.3, Eq. 1 and Eq. 2);
 *   3. partition every sorted block by the pivots (the split table);
 *   4. merge the k-th partition of all blocks into the output at offset O_k,
 *      the exclusive scan of the partition sizes.
 * Every step runs in CUDA kernels on the caller's stream; there is no CPU
 * fallback.  The paper poses only the problem of putting N elements in
 * ascending order (Sec. 2); the argument conventions below are this
 * library's own.
 *
 * Order.  Keys compare by an order key kappa: signed integers by value,
 * unsigned integers by value, floats by IEEE 754 totalOrder (so -0.0 sorts
 * before +0.0; NaN inputs are not supported and sort to the ends by their
 * bit pattern).  Records (uint64 key, uint32 payload) compare by
 * (key, payload).  Equal keys have equal bits, so the output is unique.
 *
 * Memory.  All key, payload and trace pointers are DEVICE pointers unless a
 * function says otherwise.  The caller owns them and must keep them valid
 * until the work queued on `stream` has finished.  The library owns its
 * workspace: it is taken from a library-private stream-ordered memory pool
 * (cudaMallocFromPoolAsync) on `stream` and returned to it on `stream`.
 *
 * Errors.  Every function returns PS_OK (0) or a negative ps_status.  Argument
 * errors are detected before any work is queued.  Errors of kernels already
 * queued surface at the caller's next synchronisation, as for any CUDA call.
 * No function throws, aborts or prints.
 *
 * Threads.  Functions may be called from several host threads at once; calls
 * on the same stream are ordered by the stream.
 */
#ifndef PSORT_H
#define PSORT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; NULL means the legacy default stream. */
typedef struct CUstream_st* ps_stream_t;

typedef enum {
    PS_OK = 0,
    PS_ERR_INVALID_ARG = -1,  /* null pointer, negative size, parameter out of range */
    PS_ERR_UNSUPPORTED = -2,  /* unknown dtype or pivot mode */
    PS_ERR_NO_MEMORY = -3,    /* workspace allocation failed */
    PS_ERR_CUDA = -4,         /* a CUDA runtime call failed (see ps_last_cuda_error) */
    PS_ERR_BUSY = -5,         /* server: admission budget or in-flight limit reached */
    PS_ERR_TIMEOUT = -6,      /* a bounded wait expired */
    PS_ERR_NOT_FOUND = -7     /* server: unknown request id */
} ps_status;

typedef enum {
    PS_I32 = 0, PS_I64 = 1, PS_F32 = 2, PS_F64 = 3, PS_U32 = 4, PS_U64 = 5
} ps_dtype;

typedef enum {
    PS_PIVOT_REGULAR = 0, /* PSRS: regular sampling (Sec. 2.3) */
    PS_PIVOT_EXACT = 1    /* PSES: exact splitting (Sec. 2.3, Eq. 1, Eq. 2) */
} ps_pivot_mode;

/* Tuning parameters.  0 in a field means "choose automatically" (a tuned
 * entry from ps_autotune, else the library's size-binned default).
 * n_blocks = n_B and n_parts = n_P of Sec. 2; both may exceed n (empty blocks
 * or partitions are legal).  Limits: 1 <= n_blocks <= 4096,
 * 1 <= n_parts <= 1048576.
 * items_per_thread and block_threads fix the launch shape of the two data
 * passes of the GPU design, the tile sort of step 1 and the chunk merges of
 * the in-block passes and of step 4: every CTA holds block_threads *
 * items_per_thread keys in shared memory (the tile and the chunk capacity).
 * They are an implementation choice, not part of the paper's method, and do
 * not change the result.  Supported: items_per_thread in {16, 32} and
 * block_threads in {128, 256, 512} for keys-only sorts (a 0 in one of the
 * two fields takes 32 items or 256 threads); records (ps_sort_pairs,
 * ps_sort_struct) take only the automatic shape (0, 0) or (16, 256).  Any
 * other value is PS_ERR_INVALID_ARG; a shape not offered for the dtype is
 * PS_ERR_UNSUPPORTED.  Batched sorts (and the server's rounds, which are
 * batched sorts) take, per size bin, the shape of the bin's entry in the
 * batched autotune table, else the automatic one. */
typedef struct {
    int64_t n_blocks;
    int64_t n_parts;
    int64_t merge_variant;    /* step 4 (Sec. 2.2), one of ps_merge_variant */
    int32_t items_per_thread; /* 0 = automatic, 16 or 32 */
    int32_t block_threads;    /* 0 = automatic, 128, 256 or 512 */
} ps_params;

/* How step 4 merges the pieces of one chunk of a partition (Sec. 2.2 and the
 * comparison of multiway merging algorithms in Sec. 4).  All three give the
 * same output; the default is the fast one, the others are for comparison.
 *   PS_MERGE_TREE  0: the pieces are merged pairwise, level by level
 *                     (ceil(log2 n_B) merge-path levels in shared memory)
 *   PS_MERGE_SORT  1: the pieces are copied next to each other and the chunk
 *                     is sorted as a whole (Sec. 2.2, "copying them into an
 *                     output array and sorting it")
 *   PS_MERGE_SELECT 2: one thread per chunk pops the chunk's smallest head
 *                     from a selection (loser) tree over the n_B run heads
 *                     (Sec. 2.2, Knuth's selection tree), reading the runs
 *                     straight from device memory */
typedef enum { PS_MERGE_TREE = 0, PS_MERGE_SORT = 1, PS_MERGE_SELECT = 2 } ps_merge_variant;

/* Optional record of the method's intermediates, for checking.  Each pointer
 * may be NULL (that intermediate is not reported).  All are device pointers
 * sized by the caller:
 *   pivots         n_P-1 pivots P_1..P_{n_P-1} in the key's own dtype
 *                  (for records: the uint64 key half)
 *   pivot_payload  n_P-1 uint32 payload halves of the pivots (records only)
 *   c              n_P-1 int64 tie counts c_k of Eq. 2 (exact splitting;
 *                  zeros under regular sampling)
 *   splits         n_B x (n_P+1) int64, row-major; splits[b*(n_P+1)+k] is the
 *                  number of elements of sorted block b that lie in
 *                  partitions 0..k-1
 *   offsets        n_P+1 int64 partition offsets O_0 = 0 .. O_{n_P} = n
 * The trace is written only when n >= 2. */
typedef struct {
    void* pivots;
    uint32_t* pivot_payload;
    int64_t* c;
    int64_t* splits;
    int64_t* offsets;
} ps_trace;

/* Sort n keys of `dtype` in place at `keys` (device memory, naturally
 * aligned for the dtype), with automatic parameters.  n = 0 or 1 is a no-op.
 * Returns PS_OK once all kernels are queued on `stream`. */
int ps_sort(void* keys, int64_t n, int dtype, int pivot_mode, ps_stream_t stream);

/* As ps_sort, with explicit parameters (NULL = automatic) and an optional
 * trace (NULL = none). */
int ps_sort_ex(void* keys, int64_t n, int dtype, int pivot_mode, const ps_params* params,
               const ps_trace* trace, ps_stream_t stream);

/* Sort n records in place, ordered by (key, payload): keys[i] and payload[i]
 * form record i (structure of arrays, device memory). */
int ps_sort_pairs(uint64_t* keys, uint32_t* payload, int64_t n, int pivot_mode,
                  const ps_params* params, const ps_trace* trace, ps_stream_t stream);

/* Sort n fixed-size records in place by the uint64 key stored inside each
 * record (Table 1's Pair, 16 B = key + index, and Particle, 96 B = key + 88 B
 * of particle data, both of which the paper orders by their uint64 key).
 *   records       n * record_bytes bytes of device memory, array of
 *                 structures, 8-byte aligned
 *   record_bytes  multiple of 8, 8 .. PS_STRUCT_MAX_BYTES
 *   key_offset    byte offset of the key inside a record: multiple of 8,
 *                 at most record_bytes - 8; the key is read as unsigned
 * Records with equal keys keep their input order (the order is (key, input
 * position)), so the result is unique.  n must be below 2^32.  The four steps
 * run on (key, position) pairs (as ps_sort_pairs); the records then move once,
 * by a gather.  Workspace from the pool: n * record_bytes bytes for a copy of
 * the records plus 12 * n bytes of pairs and the pair sort's own.  Argument
 * errors return PS_ERR_INVALID_ARG before anything is queued. */
#define PS_STRUCT_MAX_BYTES 4096
int ps_sort_struct(void* records, int64_t n, int64_t record_bytes, int64_t key_offset, int pivot_mode,
                   const ps_params* params, ps_stream_t stream);

/* Sort many independent segments of one key array in place: segment i is
 * keys[seg_offsets[i], seg_offsets[i+1]) (seg_offsets: n_segs+1 non-decreasing
 * DEVICE int64 offsets).  Segments are binned by length.  Every segment of at
 * most one shared-memory tile (8192 keys) is sorted by one persistent launch
 * (a grid sized to the GPU whose CTAs take work items from a device counter:
 * a CTA per segment above 1024 keys, a warp per segment up to 1024 keys);
 * every longer bin runs the four-step method on all of its segments at once.
 * So the number of kernel launches depends on the number of size bins, not
 * on the number of segments.  Each segment's result equals ps_sort on it alone.
 * The call reads seg_offsets back to the host (it waits for `stream` once,
 * before queuing the sort); it returns once the sort is queued. */
int ps_sort_batch(const int64_t* seg_offsets, int64_t n_segs, void* keys, int dtype, int pivot_mode,
                  ps_stream_t stream);

/* Batch plans for repeated batches of one shape.  ps_batch_plan_create reads
 * n_segs+1 HOST offsets once, bins the segments as ps_sort_batch does, and
 * allocates (cudaMalloc) the device instance table and the workspace of the
 * largest bin; it waits for those copies.  ps_batch_run then queues the sort
 * of every segment of `keys` (device memory laid out as the offsets say, the
 * dtype and pivot mode of the plan) on `stream` with no host synchronisation
 * and no allocation, so a caller can capture it in a CUDA graph and replay it.
 * Runs of one plan share its workspace: they must not overlap on the GPU.
 * Results equal ps_sort on each segment alone. */
typedef struct ps_batch_plan ps_batch_plan;
int ps_batch_plan_create(const int64_t* host_seg_offsets, int64_t n_segs, int dtype, int pivot_mode,
                         ps_batch_plan** out);
int ps_batch_run(const ps_batch_plan* plan, void* keys, ps_stream_t stream);
int ps_batch_plan_destroy(ps_batch_plan* plan);

/* End-to-end form for callers whose keys live in HOST memory (pinned or
 * pageable; naturally aligned for the dtype): sorts them as ps_sort_ex does,
 * leaves the result in `host_keys`, and waits for `stream` to finish before
 * returning.  Page-locked memory the device can address (cudaHostAlloc, or
 * cudaHostRegister with mapping, e.g. a pinned torch tensor): below 2^24 keys
 * (or with one block) the first pass reads it and the last pass writes it
 * directly, with no separate copies; from 2^24 keys the blocks are copied in
 * groups on a library-created copy stream while earlier groups are
 * block-sorted, and with exact splitting the result is copied back in
 * partition ranges while later ranges merge (regular sampling: the final
 * merge writes the host buffer directly).  Other memory is copied to a
 * device buffer and back.  Device buffers come from the library's pool. */
int ps_sort_host(void* host_keys, int64_t n, int dtype, int pivot_mode,
                 const ps_params* params, ps_stream_t stream);

/* Autotuner.  Times candidate (n_blocks, n_parts) pairs around the size
 * heuristic (n_B in {d/2, d, 2d, 4d}, n_P in {n_B/2, n_B, 2 n_B}) on seeded
 * uniform keys of `dtype`'s width for every power-of-two size 2^b in
 * [max(n_min, 2^14), n_max], and records the fastest pair per (key width, b)
 * in a process-wide table that automatic parameters then use for sorts of
 * round(log2 n) = b.  batched = 0 tunes single sorts; batched = 1 tunes the
 * size bins of ps_sort_batch (batches of about 2^26 keys in segments of
 * (2^(b-1), 2^b] keys) and fills a separate table.  Each size then also
 * times every launch shape (items_per_thread x block_threads) the dtype
 * offers at the fastest (n_B, n_P) and records the fastest shape with them
 * (for batches: per size bin).  Allocates
 * 2 * max(n_max, 2^26) keys of workspace; waits for `stream` (each candidate
 * is timed with CUDA events: one untimed run, median of three).  n_max at
 * most 2^34. */
int ps_autotune(int dtype, int pivot_mode, int64_t n_min, int64_t n_max, int batched, ps_stream_t stream);

/* Read (PS_ERR_NOT_FOUND when untuned) or write one entry of the tuned table:
 * out/p->n_blocks, n_parts, items_per_thread and block_threads for sorts of
 * round(log2 n) = log2_n keys of dtype's width (a shape of 0, 0 = the
 * automatic one).  ps_autotune_set with p NULL (or n_blocks and n_parts 0)
 * clears the entry; it lets a caller restore a table saved from an earlier
 * run. */
int ps_autotune_get(int dtype, int batched, int log2_n, ps_params* out);
int ps_autotune_set(int dtype, int batched, int log2_n, const ps_params* p);

/* The parameters a sort of n keys of `dtype` would use: copies `in` (or
 * zeros when NULL) to `out` with every automatic field resolved (tuned
 * entries first, then the size heuristic). */
int ps_resolve_params(int64_t n, int dtype, const ps_params* in, ps_params* out);

/* Bytes of workspace one sort of n keys of `dtype` takes from the pool
 * (dtype -1 = records). */
int ps_workspace_bytes(int64_t n, int dtype, const ps_params* params, size_t* out);

/* Static, human-readable text for a ps_status value. */
const char* ps_status_string(int status);

/* The cudaError_t of the last CUDA failure seen by this host thread (0 if
 * none). */
int ps_last_cuda_error(void);

/* ---- sort server (continuous batching) ------------------------------------
 * A server sorts device buffers submitted from any host thread.  Requests
 * queue in arrival order; a worker thread admits the queue's head whenever a
 * stream slot is free, fewer than max_inflight requests are on the GPU and the
 * memory budget holds the request's cost (scratch for a copy of its keys plus
 * the sort's workspace).  Each admission round runs as one batched sort per
 * (dtype, pivot mode) that reads every request from its own buffer and writes
 * the result back there (no gather or scatter copies), on one of several
 * server streams, so rounds admitted while others run overlap on the GPU.
 * Results are bit-identical to ps_sort on each buffer alone.  A round that
 * fails on the device may leave its requests' keys partly rewritten.
 *   ps_server_open    budget in bytes (> 0), max_inflight >= 1; the server
 *                     uses the device current at open.
 *   ps_server_submit  dev_keys must hold the n keys when submitted (ordered
 *                     before the call on the caller's side) and stay untouched
 *                     until the request completes; writes a request id.
 *                     PS_ERR_BUSY if the request alone exceeds the budget;
 *                     PS_ERR_INVALID_ARG after ps_server_close started.
 *   ps_server_poll    non-blocking: moves up to cap completed (id, status)
 *                     pairs out, in completion order, and sets *n_done.
 *   ps_server_close   stops accepting, waits for every admitted and queued
 *                     request to finish, frees the server. */
typedef struct ps_server ps_server;
int ps_server_open(size_t mem_budget_bytes, int max_inflight, ps_server** out);
int ps_server_submit(ps_server* server, void* dev_keys, int64_t n, int dtype, int pivot_mode, uint64_t* req_id);
int ps_server_poll(ps_server* server, uint64_t* done_ids, int* statuses, int cap, int* n_done);
int ps_server_close(ps_server* server);

/* Failure injection for tests, on the host (no device fault): what = 0 makes
 * the next `count` admitted rounds fail at launch (their requests complete
 * with PS_ERR_CUDA, nothing is queued on the GPU); what = 1 retires the next
 * `count` idle stream slots as if their streams had failed (the server keeps
 * serving on the others; with none left, queued and new requests complete
 * with PS_ERR_CUDA).  PS_ERR_INVALID_ARG for other values. */
int ps_server_debug_fail(ps_server* server, int what, int count);

/* ---- allocation-free variant -------------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers
 * that must not allocate device memory: code running while a CUDA graph is
 * being captured by someone else, real-time loops that forbid allocator
 * calls, and hosts whose memory pools are owned and capped by another
 * runtime.  ps_sort_noalloc sorts like ps_sort (same dtypes and pivot modes,
 * result bit-identical) but takes all of its workspace from one static device
 * array of PS_NOALLOC_SCRATCH_BYTES that the library reserves on every GPU it
 * is loaded on, for the life of the process.  Its n_B and n_P always come from
 * the size heuristic (not from tuned or measured table entries, which
 * ps_sort prefers): the array is sized for the heuristic's shapes, so the
 * speed may differ from ps_sort's, the result does not.
 *   - n above PS_NOALLOC_MAX_KEYS (or a shape whose workspace would not fit
 *     the array) is rejected with PS_ERR_INVALID_ARG before any work is queued.
 *   - It calls no cudaMalloc, cudaFree or pool allocation.  (Keep profiling
 *     off: ps_profile_enable makes every launch create CUDA events.)
 *   - The first call in each CUDA context (per device: its primary context,
 *     or a context the caller made current) looks up the array's device
 *     address there (cudaGetSymbolAddress) and caches it under the context's
 *     unique ID; make that first call outside any stream capture.
 *   - All calls on a device share the one array and the kernels overwrite
 *     whatever a previous call left there (the counters they need are zeroed
 *     on the stream before use).  Two calls whose work overlaps on the GPU --
 *     on different streams, or from different threads without ordering --
 *     race on the array and corrupt each other's results: serialise them. */
#define PS_NOALLOC_MAX_KEYS ((int64_t)1 << 20)
#define PS_NOALLOC_SCRATCH_BYTES ((size_t)12 << 20)
int ps_sort_noalloc(void* keys, int64_t n, int dtype, int pivot_mode, ps_stream_t stream);

/* Failure injection for tests, on the host: the next `count` workspace
 * allocations of the library fail with PS_ERR_NO_MEMORY before any CUDA call
 * (0 turns it off).  Sorts then return PS_ERR_NO_MEMORY with nothing queued. */
int ps_debug_fail_alloc(int count);

/* ---- checked builds -------------------------------------------------------
 * A build compiled with -DPS_CHECKED (libpsort_checked.so) validates every
 * global and shared-memory index in its kernels; the first out-of-range
 * access is not performed but recorded.  ps_debug_violation waits for
 * nothing, reads and clears that record: it returns 1 and fills out[0..3]
 * with (site + 100 * key family, index, bound, CTA) if a violation was seen,
 * 0 if none (always 0 in an ordinary build), or a negative status. */
int ps_debug_violation(uint64_t* out);

/* ---- profiling (library-wide, off by default) ---------------------------
 * While enabled, every kernel the library launches is bracketed by two CUDA
 * events recorded on the launch stream, so that per-kernel device time can be
 * read back without an external profiler.  Recording adds two event records
 * per launch; it does not synchronise. */
typedef struct {
    char name[32];     /* kernel label, e.g. "tile_sort", "merge_final" */
    int64_t launches;  /* launches recorded since the last reset */
    double total_ms;   /* summed device time of those launches */
} ps_kernel_stat;

/* Turn recording on (1) or off (0).  Returns the previous state. */
int ps_profile_enable(int on);

/* Wait for every recorded launch to finish, then write at most `cap`
 * per-kernel aggregates to `out` and their count to *n (kernels in first-seen
 * order).  Returns PS_ERR_CUDA if an event cannot be read. */
int ps_profile_read(ps_kernel_stat* out, int cap, int* n);

/* Forget all recorded launches. */
int ps_profile_reset(void);

#ifdef __cplusplus
}
#endif

#endif /* PSORT_H */

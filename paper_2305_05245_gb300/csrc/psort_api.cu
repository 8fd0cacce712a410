// psort_api.cu -- the C ABI declared in include/psort.h: argument checks,
// automatic parameters, the workspace pool, and dispatch to the key families.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "psort_internal.h"

namespace ps {

static thread_local int g_last_cuda = 0;

int fail_cuda(cudaError_t e)
{
    g_last_cuda = (int)e;
    if (e == cudaErrorMemoryAllocation) return PS_ERR_NO_MEMORY;
    return PS_ERR_CUDA;
}

// One stream-ordered memory pool per device, created on first use and kept
// for the life of the process; freed blocks stay cached in the pool.
static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[64];

static int get_pool(cudaMemPool_t* out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail_cuda(e);
    if (dev < 0 || dev >= 64) return PS_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p;
        e = cudaMemPoolCreate(&p, &props);
        if (e != cudaSuccess) return fail_cuda(e);
        uint64_t keep = ~0ull;
        e = cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) return fail_cuda(e);
        g_pool[dev] = p;
    }
    *out = g_pool[dev];
    return PS_OK;
}

// Host-side failure injection (ps_debug_fail_alloc): the next n workspace
// allocations fail with PS_ERR_NO_MEMORY before any CUDA call.
static std::atomic<int> g_fail_alloc{0};

int ws_alloc(void** p, size_t bytes, cudaStream_t s)
{
    for (int k = g_fail_alloc.load(); k > 0;)
        if (g_fail_alloc.compare_exchange_weak(k, k - 1)) return PS_ERR_NO_MEMORY;
    cudaMemPool_t pool;
    int rc = get_pool(&pool);
    if (rc != PS_OK) return rc;
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes ? bytes : 256, pool, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail_cuda(e);
    }
    return PS_OK;
}

void ws_free(void* p, cudaStream_t s)
{
    if (p) cudaFreeAsync(p, s);
}

// ---- profiling records
struct ProfRec {
    std::string name;
    cudaEvent_t a, b;
};
static std::atomic<bool> g_prof{false};
static std::mutex g_prof_mu;
static std::vector<ProfRec> g_prof_recs;

bool prof_on() { return g_prof.load(std::memory_order_relaxed); }

int prof_begin(const char* name, cudaStream_t s)
{
    ProfRec r;
    r.name = name;
    if (cudaEventCreate(&r.a) != cudaSuccess) return -1;
    if (cudaEventCreate(&r.b) != cudaSuccess) {
        cudaEventDestroy(r.a);
        return -1;
    }
    cudaEventRecord(r.a, s);
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_recs.push_back(r);
    return (int)g_prof_recs.size() - 1;
}

void prof_end(int rec, cudaStream_t s)
{
    cudaEvent_t b;
    {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        if (rec < 0 || rec >= (int)g_prof_recs.size()) return;
        b = g_prof_recs[rec].b;
    }
    cudaEventRecord(b, s);
}

static void prof_clear()
{
    for (auto& r : g_prof_recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    g_prof_recs.clear();
}

static const int64_t MAX_BLOCKS = 4096;
static const int64_t MAX_PARTS = 1 << 20;

static int64_t pow2_floor(int64_t x)
{
    int64_t p = 1;
    while (p * 2 <= x) p *= 2;
    return p;
}

// Size-binned defaults.  The block sort makes in-block merge passes of
// fan-in <= 256 over tiles of T keys and the final merge has fan-in n_B; on
// GB300 the measured optimum sits near n_B = 0.35 * sqrt(N / T) (64 blocks at
// 2^28 keys, 128 at 2^30).  Exact splitting costs O(n_P * n_B * log^2 L)
// probes (Sec. 2.3), so n_P stays <= min(n_B, 256); the final merge cuts
// partitions into chunks on its own.
//
// Autotuned parameters (ps_autotune) take precedence over these defaults for
// automatic fields: g_tune[context][family][round(log2 n)] holds (n_B, n_P)
// and the launch shape (items per thread, threads per CTA; 0, 0 = automatic)
// measured fastest for sorts of about n keys, context 0 for single sorts and
// 1 for the size bins of batched sorts; family 0 = 32-bit keys, 1 = 64-bit.
struct TuneEntry {
    int32_t nb, np, items, threads;
};
static std::mutex g_tune_mu;
static TuneEntry g_tune[2][2][64];

static int tune_family(int dtype)
{
    if (dtype == PS_I32 || dtype == PS_F32 || dtype == PS_U32) return 0;
    if (dtype == PS_I64 || dtype == PS_F64 || dtype == PS_U64) return 1;
    return -1;
}

static int tune_bin(int64_t n)
{
    int b = 0;
    while (b < 62 && (int64_t(1) << (b + 1)) <= n) b++;  // floor(log2 n)
    // round to the nearer power of two
    if (b < 62 && (double)n >= 1.41421356 * (double)(int64_t(1) << b)) b++;
    return b;
}

static bool tuned(int ctx, int dtype, int64_t n, int32_t* nb, int32_t* np, int32_t* items = nullptr,
                  int32_t* threads = nullptr)
{
    const int f = tune_family(dtype);
    if (f < 0 || n < 2) return false;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const TuneEntry& e = g_tune[ctx][f][tune_bin(n)];
    if (e.nb <= 0) return false;
    *nb = e.nb;
    *np = e.np;
    if (items) *items = e.items;
    if (threads) *threads = e.threads;
    return true;
}

static void resolve_heuristic(int64_t n, int dtype, const ps_params* in, ps_params* out)
{
    ps_params r;
    memset(&r, 0, sizeof(r));
    if (in) r = *in;
    const double tile = dtype < 0 ? 4096.0 : 8192.0;
    const double want = 0.35 * std::sqrt((double)n / tile);
    int64_t nb = 1;
    while (nb < 1024 && (double)nb * 1.41421356 < want) nb *= 2;
    if (r.n_blocks <= 0) r.n_blocks = nb;
    if (r.n_parts <= 0) r.n_parts = std::min<int64_t>(256, std::max<int64_t>(1, r.n_blocks));
    *out = r;
}

void resolve_default(int64_t n, int dtype, ps_params* out) { resolve_heuristic(n, dtype, nullptr, out); }

// Defaults measured on GB300 with ps_autotune (exact splitting, uniform keys):
// (n_B, n_P) per round(log2 n) from 2^14 on, for single sorts and for the size
// bins of batched sorts, 32-bit and 64-bit keys.  Up to 2^19-2^20 keys one
// block and one partition win (the block sort is the whole sort).
struct DefaultTune {
    int lo, hi;              // log2 sizes covered
    const int32_t (*e)[2];   // e[b - lo] = {n_B, n_P}
};
static const int32_t kTuneU32[][2] = {{1, 1}, {1, 1}, {1, 1}, {1, 1}, {1, 1}, {1, 1}, {2, 1}, {8, 8}, {16, 32},
                                      {32, 32}, {64, 64}, {64, 128}, {128, 128}, {16, 32}, {32, 64}, {64, 128},
                                      {64, 128}, {64, 64}};                                 // 2^14 .. 2^31
static const int32_t kTuneU64[][2] = {{1, 1}, {1, 1}, {1, 1}, {1, 1}, {1, 1}, {1, 1}, {16, 32}, {16, 16},
                                      {32, 64}, {32, 64}, {64, 128}, {64, 128}, {16, 16}, {16, 16}, {32, 64},
                                      {32, 64}, {64, 128}};                                 // 2^14 .. 2^30
static const int32_t kTuneU32Batch[][2] = {{2, 1}, {1, 1}, {1, 1}, {1, 1}, {1, 1}, {1, 1}, {2, 1}, {8, 4},
                                           {8, 8}, {16, 16}, {32, 16}};                    // 2^14 .. 2^24
static const int32_t kTuneU64Batch[][2] = {{2, 1}, {1, 1}, {1, 1}, {1, 1}, {1, 1}, {1, 1}, {4, 2}, {8, 4},
                                           {16, 8}, {32, 16}, {32, 16}};                   // 2^14 .. 2^24
static const DefaultTune kDefaults[2][2] = {{{14, 31, kTuneU32}, {14, 30, kTuneU64}},
                                            {{14, 24, kTuneU32Batch}, {14, 24, kTuneU64Batch}}};

static bool measured_default(int ctx, int dtype, int64_t n, int32_t* nb, int32_t* np)
{
    const int f = tune_family(dtype);
    if (f < 0 || n < 2) return false;
    const DefaultTune& d = kDefaults[ctx][f];
    const int b = tune_bin(n);
    if (b < d.lo || b > d.hi) return false;
    *nb = d.e[b - d.lo][0];
    *np = d.e[b - d.lo][1];
    return true;
}

// Automatic fields: a tuned entry for this size (context ctx) when there is
// one, else the measured default, else the heuristic.  Explicit fields are
// kept.  A tuned entry supplies its launch shape too when n_blocks and both
// shape fields are automatic; otherwise (0, 0) stays the family's automatic
// shape.
static void resolve(int64_t n, int dtype, const ps_params* in, ps_params* out, int ctx = 0)
{
    ps_params r;
    memset(&r, 0, sizeof(r));
    if (in) r = *in;
    int32_t nb = 0, np = 0, it = 0, th = 0;
    const bool auto_shape = r.items_per_thread == 0 && r.block_threads == 0;
    if ((r.n_blocks <= 0 || r.n_parts <= 0) && tuned(ctx, dtype, n, &nb, &np, &it, &th)) {
        if (r.n_blocks <= 0) {
            r.n_blocks = nb;
            if (r.n_parts <= 0) r.n_parts = np;
            if (auto_shape) {
                r.items_per_thread = it;
                r.block_threads = th;
            }
        }
    } else if ((r.n_blocks <= 0 || r.n_parts <= 0) && measured_default(ctx, dtype, n, &nb, &np)) {
        if (r.n_blocks <= 0) {
            r.n_blocks = nb;
            if (r.n_parts <= 0) r.n_parts = np;
        }
    }
    resolve_heuristic(n, dtype, &r, out);
}

static int check_params(const ps_params* p)
{
    if (!p) return PS_OK;
    if (p->n_blocks < 0 || p->n_blocks > MAX_BLOCKS) return PS_ERR_INVALID_ARG;
    if (p->n_parts < 0 || p->n_parts > MAX_PARTS) return PS_ERR_INVALID_ARG;
    if (p->merge_variant < PS_MERGE_TREE || p->merge_variant > PS_MERGE_SELECT) return PS_ERR_INVALID_ARG;
    if (p->items_per_thread != 0 && p->items_per_thread != 16 && p->items_per_thread != 32) return PS_ERR_INVALID_ARG;
    if (p->block_threads != 0 && p->block_threads != 128 && p->block_threads != 256 && p->block_threads != 512)
        return PS_ERR_INVALID_ARG;
    return PS_OK;
}

// The launch shape a sort runs with: nullptr for the family's automatic
// shape, else the compiled shape; PS_ERR_UNSUPPORTED in *rc when the shape is
// not offered for the dtype.
static const ShapeEntry* shape_of(int dtype, int items, int threads, int* rc)
{
    *rc = PS_OK;
    if (items == 0 && threads == 0) return nullptr;
    const int it = items ? items : 32, th = threads ? threads : 256;
    if (dtype == -1) {
        if (it != 16 || th != 256) *rc = PS_ERR_UNSUPPORTED;
        return nullptr;
    }
    const int bits = (dtype == PS_I32 || dtype == PS_F32 || dtype == PS_U32) ? 32 : 64;
    if (bits == 64 && it == 32 && th == 256) return nullptr;  // the automatic 64-bit shape
    const ShapeEntry* e = find_shape(bits, it, th);
    if (!e) *rc = PS_ERR_UNSUPPORTED;
    return e;
}

// PS_LOG=1 in the environment: one line per sort on stderr with the
// resolved parameters (read once).
static int log_level()
{
    static const int lvl = [] {
        const char* v = getenv("PS_LOG");
        return v ? atoi(v) : 0;
    }();
    return lvl;
}

static int dispatch(SortArgs& a)
{
    if (log_level() >= 1)
        fprintf(stderr, "psort: n=%lld dtype=%d mode=%d n_B=%lld n_P=%lld instances=%lld merge_variant=%d shape=%dx%d\n",
                (long long)a.n, a.dtype, a.mode, (long long)a.n_B, (long long)a.n_P, (long long)a.n_inst,
                a.merge_variant, a.items, a.threads);
    int rc = PS_OK;
    const ShapeEntry* sh = shape_of(a.dtype, a.items, a.threads, &rc);
    if (rc != PS_OK) return rc;
    if (sh) return sh->run(a);
    switch (a.dtype) {
    case PS_I32: case PS_F32: case PS_U32: return run_sort_u32(a);
    case PS_I64: case PS_F64: case PS_U64: return run_sort_u64(a);
    case -1: return run_sort_rec(a);
    default: return PS_ERR_UNSUPPORTED;
    }
}

static int sort_common(void* keys, uint32_t* payload, int64_t n, int dtype, int mode, const ps_params* params,
                       const ps_trace* trace, ps_stream_t stream)
{
    if (n < 0) return PS_ERR_INVALID_ARG;
    if (dtype < -1 || dtype > PS_U64) return PS_ERR_UNSUPPORTED;
    if (mode != PS_PIVOT_REGULAR && mode != PS_PIVOT_EXACT) return PS_ERR_UNSUPPORTED;
    int rc = check_params(params);
    if (rc != PS_OK) return rc;
    if (n <= 1) return PS_OK;
    if (!keys || (dtype == -1 && !payload)) return PS_ERR_INVALID_ARG;
    const size_t align = (dtype == PS_I32 || dtype == PS_F32 || dtype == PS_U32) ? 4 : 8;
    if ((uintptr_t)keys % align != 0 || (payload && (uintptr_t)payload % 4 != 0)) return PS_ERR_INVALID_ARG;
    ps_params r;
    resolve(n, dtype, params, &r);
    SortArgs a;
    a.keys = keys;
    a.payload = payload;
    a.n = n;
    a.dtype = dtype;
    a.mode = mode;
    a.n_B = r.n_blocks;
    a.n_P = r.n_parts;
    a.merge_variant = (int)r.merge_variant;
    a.items = r.items_per_thread;
    a.threads = r.block_threads;
    a.trace = trace;
    a.stream = (cudaStream_t)stream;
    return dispatch(a);
}

int sort_records(uint64_t* keys, uint32_t* payload, int64_t n, int mode, const ps_params* params, cudaStream_t s)
{
    return sort_common(keys, payload, n, -1, mode, params, nullptr, s);
}

static size_t dtype_size(int dtype)
{
    return (dtype == PS_I32 || dtype == PS_F32 || dtype == PS_U32) ? 4 : 8;
}

size_t sort_ws_bytes(int64_t n, int dtype)
{
    ps_params r;
    resolve(n, dtype, nullptr, &r);
    switch (dtype) {
    case PS_I32: case PS_F32: case PS_U32: return ws_bytes_u32(n, r.n_blocks, r.n_parts);
    case -1: return ws_bytes_rec(n, r.n_blocks, r.n_parts);
    default: return ws_bytes_u64(n, r.n_blocks, r.n_parts);
    }
}

// Batched sorts.  A batch plan bins the segments [off[i], off[i+1]) by length
// and fixes each bin's parameters and its part of the instance table (per
// bin: all starts, then all lengths); launching a plan queues one persistent
// launch for the segments of at most one tile (both short bins together) and
// one multi-instance pipeline per longer bin.
struct BatchBin {
    size_t at;                // offset of the bin's starts in the instance table
    int64_t cnt, nmax, nsum;  // instances, longest, total keys
    int64_t n_B, n_P;
    int items, threads;       // launch shape (0, 0: automatic)
    bool small;               // at most SMALL_SEG keys each (one warp each)
    bool front;               // at most one tile each: sorted by the persistent front kernel
};
struct BatchPlan {
    int dtype = 0, mode = 0;
    int64_t extent = 0;
    bool own = false;            // segments in buffers of their own (per bin: starts, lengths, pointers)
    std::vector<int64_t> table;  // host copy of the instance table
    std::vector<BatchBin> bins;
    size_t counter_at = 0;       // the front kernel's work counter (last table slot), if a front bin exists
};

// own (optional): one device pointer per segment; segment i then lives in its
// own buffer, and off only lays the segments out for the workspace.
static int batch_make_plan(const std::vector<int64_t>& off, int dtype, int mode, const ps_params* force,
                           BatchPlan* bp, const std::vector<void*>* own = nullptr)
{
    const int64_t n_segs = (int64_t)off.size() - 1;
    if (dtype < PS_I32 || dtype > PS_U64) return PS_ERR_UNSUPPORTED;
    if (n_segs < 0 || off.empty() || off[0] < 0) return PS_ERR_INVALID_ARG;
    for (int64_t i = 0; i < n_segs; i++)
        if (off[i + 1] < off[i]) return PS_ERR_INVALID_ARG;
    bp->dtype = dtype;
    bp->mode = mode;
    bp->extent = off[(size_t)n_segs];
    bp->own = own != nullptr;
    if (own && own->size() < (size_t)n_segs) return PS_ERR_INVALID_ARG;
    bp->table.clear();
    bp->bins.clear();
    // bins: 0 = at most SMALL_SEG keys (a warp each); 1 = fits one tile (a
    // CTA each); b >= 2 = lengths in (T*2^(b-2), T*2^(b-1)]
    const int64_t tile = 8192;
    std::vector<std::vector<int64_t>> bins(48);
    for (int64_t i = 0; i < n_segs; i++) {
        const int64_t len = off[i + 1] - off[i];
        if (len <= 1) continue;
        int b = 1;
        if (len <= SMALL_SEG) b = 0;
        while (len > (tile << (b - 1)) && b > 0) b++;
        bins[b].push_back(i);
    }
    for (size_t b = 0; b < bins.size(); b++) {
        if (bins[b].empty()) continue;
        BatchBin bb;
        bb.at = bp->table.size();
        bb.cnt = (int64_t)bins[b].size();
        bb.nmax = bb.nsum = 0;
        for (int64_t i : bins[b]) bp->table.push_back(off[i]);
        for (int64_t i : bins[b]) {
            const int64_t len = off[i + 1] - off[i];
            bp->table.push_back(len);
            bb.nmax = std::max<int64_t>(bb.nmax, len);
            bb.nsum += len;
        }
        if (own)
            for (int64_t i : bins[b]) bp->table.push_back((int64_t)(uintptr_t)(*own)[(size_t)i]);
        ps_params r;
        memset(&r, 0, sizeof(r));
        if (b <= 1) {
            r.n_blocks = r.n_parts = 1;  // one tile: the block sort is the whole sort
        } else if (force) {
            r = *force;
        } else {
            resolve(bb.nmax, dtype, nullptr, &r, 1);
        }
        bb.n_B = r.n_blocks;
        bb.n_P = r.n_parts;
        bb.items = b <= 1 ? 0 : r.items_per_thread;
        bb.threads = b <= 1 ? 0 : r.block_threads;
        bb.small = b == 0;
        bb.front = b <= 1;
        bp->bins.push_back(bb);
    }
    for (const BatchBin& bb : bp->bins)
        if (bb.front) {
            bp->counter_at = bp->table.size();
            bp->table.push_back(0);
            break;
        }
    return PS_OK;
}

static SortArgs batch_bin_args(const BatchPlan& bp, const BatchBin& bb, const int64_t* dev_table, void* keys,
                               cudaStream_t s)
{
    SortArgs a;
    a.keys = keys;
    a.payload = nullptr;
    a.n = bb.nmax;
    a.dtype = bp.dtype;
    a.mode = bp.mode;
    a.n_B = bb.n_B;
    a.n_P = bb.n_P;
    a.items = bb.items;
    a.threads = bb.threads;
    a.trace = nullptr;
    a.stream = s;
    a.inst_base = dev_table + bb.at;
    a.inst_n = dev_table + bb.at + bb.cnt;
    if (bp.own && dev_table) a.inst_ptrs = (void* const*)(dev_table + bb.at + 2 * bb.cnt);
    a.n_inst = bb.cnt;
    a.n_max = bb.nmax;
    a.n_sum = bb.nsum;
    a.extent = bp.extent;
    return a;
}

static bool narrow_dtype(int dtype) { return dtype == PS_I32 || dtype == PS_F32 || dtype == PS_U32; }

// Queue every bin of a plan on s: the short bins in one persistent launch,
// then one pipeline per longer bin.  ws == nullptr: each pipeline takes its
// workspace from the pool; otherwise every one runs on ws (cap bytes) and
// nothing is allocated.
static int batch_launch(const BatchPlan& bp, const int64_t* dev_table, void* keys, cudaStream_t s, char* ws,
                        size_t cap)
{
    const bool narrow = narrow_dtype(bp.dtype);
    int rc = PS_OK;
    SortArgs ft, fs;
    const SortArgs *pt = nullptr, *psm = nullptr;
    for (const BatchBin& bb : bp.bins) {
        if (!bb.front) continue;
        if (bb.small) {
            fs = batch_bin_args(bp, bb, dev_table, keys, s);
            psm = &fs;
        } else {
            ft = batch_bin_args(bp, bb, dev_table, keys, s);
            pt = &ft;
        }
    }
    if (pt || psm) {
        // the counter is a slot of the device instance table, which the
        // plan owns (const only as the table's view)
        unsigned long long* next = (unsigned long long*)const_cast<int64_t*>(dev_table + bp.counter_at);
        rc = narrow ? run_front_u32(pt, psm, next) : run_front_u64(pt, psm, next);
    }
    for (size_t i = 0; i < bp.bins.size() && rc == PS_OK; i++) {
        if (bp.bins[i].front) continue;
        SortArgs a = batch_bin_args(bp, bp.bins[i], dev_table, keys, s);
        if (ws) {
            const ShapeEntry* sh = shape_of(a.dtype, a.items, a.threads, &rc);
            if (rc == PS_OK)
                rc = sh ? sh->run_on(a, ws, cap) : narrow ? run_sort_u32_on(a, ws, cap) : run_sort_u64_on(a, ws, cap);
        } else {
            rc = dispatch(a);
        }
    }
    return rc;
}

// Batched sort of the segments [off[i], off[i+1]) of `keys` (host offsets):
// bins by length, one multi-instance pipeline per bin, queued on s.
int batch_sort(const std::vector<int64_t>& off, void* keys, int dtype, int mode, cudaStream_t s,
               int64_t* pinned, size_t pinned_cap, const ps_params* force, const std::vector<void*>* own)
{
    if ((int64_t)off.size() - 1 <= 0) return PS_OK;
    if (dtype < PS_I32 || dtype > PS_U64) return PS_ERR_UNSUPPORTED;
    if (!keys) return PS_ERR_INVALID_ARG;
    if ((uintptr_t)keys % (narrow_dtype(dtype) ? 4 : 8) != 0) return PS_ERR_INVALID_ARG;
    BatchPlan bp;
    int rc = batch_make_plan(off, dtype, mode, force, &bp, own);
    if (rc != PS_OK) return rc;
    const size_t total = bp.table.size();
    if (total == 0) return PS_OK;
    // the instance table is staged in the caller's pinned buffer when it is
    // large enough (the copy then stays asynchronous; the caller keeps the
    // buffer untouched until the stream has passed this point), else the
    // copy is waited for before the plan's host table goes away
    const int64_t* host = bp.table.data();
    if (pinned && pinned_cap >= total) {
        memcpy(pinned, bp.table.data(), total * 8);
        host = pinned;
    }
    void* dev = nullptr;
    rc = ws_alloc(&dev, total * 8, s);
    if (rc != PS_OK) return rc;
    cudaError_t e = cudaMemcpyAsync(dev, host, total * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && host != pinned) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        ws_free(dev, s);
        return fail_cuda(e);
    }
    rc = batch_launch(bp, (const int64_t*)dev, keys, s, nullptr, 0);
    ws_free(dev, s);
    return rc;
}

// ------------------------------------------------------------- autotuner
// Uniform 64-bit words from SplitMix64 (Steele, Lea & Flood 2014) for the
// tuning inputs: word i of stream s is mix(s + (i + 1) * golden gamma).
__global__ void k_tune_fill(uint64_t* w, int64_t nwords, uint64_t seed)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nwords;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t z = seed + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        w[i] = z ^ (z >> 31);
    }
}

// Median of `reps` timed runs of f() on stream s (after one untimed run);
// restore() runs before each, outside the timed events.
template <typename F, typename R>
static int time_median(F f, R restore, cudaStream_t s, int reps, float* ms)
{
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return fail_cuda(e);
    e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail_cuda(e);
    }
    std::vector<float> t;
    int rc = PS_OK;
    for (int i = 0; i <= reps && rc == PS_OK; i++) {
        if ((rc = restore()) != PS_OK) break;
        if ((e = cudaEventRecord(e0, s)) != cudaSuccess) { rc = fail_cuda(e); break; }
        if ((rc = f()) != PS_OK) break;
        if ((e = cudaEventRecord(e1, s)) != cudaSuccess) { rc = fail_cuda(e); break; }
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) { rc = fail_cuda(e); break; }
        float x = 0.f;
        cudaEventElapsedTime(&x, e0, e1);
        if (i > 0) t.push_back(x);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != PS_OK) return rc;
    std::sort(t.begin(), t.end());
    *ms = t[t.size() / 2];
    return PS_OK;
}

// Candidates around the heuristic d: n_B in {d/2, d, 2d, 4d}, n_P in
// {n_B/2, n_B, 2 n_B} (within the limits).
static std::vector<std::pair<int64_t, int64_t>> tune_candidates(int64_t n, int dtype)
{
    ps_params d;
    resolve_heuristic(n, dtype, nullptr, &d);
    std::vector<std::pair<int64_t, int64_t>> c;
    for (int64_t nb : {d.n_blocks / 2, d.n_blocks, d.n_blocks * 2, d.n_blocks * 4}) {
        if (nb < 1 || nb > MAX_BLOCKS) continue;
        for (int64_t np : {nb / 2, nb, nb * 2}) {
            if (np < 1 || np > 1024) continue;
            bool dup = false;
            for (auto& x : c) dup = dup || (x.first == nb && x.second == np);
            if (!dup) c.push_back({nb, np});
        }
    }
    return c;
}

static int autotune(int dtype, int mode, int64_t n_min, int64_t n_max, int batched, cudaStream_t s)
{
    const int f = tune_family(dtype);
    const size_t kb = f == 0 ? 4 : 8;
    int b0 = 14;
    while ((int64_t(1) << b0) < n_min) b0++;
    int b1 = b0;
    while (b1 < 62 && (int64_t(1) << (b1 + 1)) <= n_max) b1++;
    if ((int64_t(1) << b1) > n_max) return PS_OK;  // no power of two in range
    // batched bins: segments of about 2^b keys, 2^26 keys per batch (at least 2 segments)
    const int64_t nkeys = batched ? std::max<int64_t>(int64_t(1) << 26, int64_t(2) << b1) : int64_t(1) << b1;
    char* buf = nullptr;
    int rc = ws_alloc((void**)&buf, 2 * (size_t)nkeys * kb + 512, s);
    if (rc != PS_OK) return rc;
    char* keys = buf;
    char* pristine = buf + (((size_t)nkeys * kb + 255) & ~(size_t)255);
    k_tune_fill<<<1024, 256, 0, s>>>((uint64_t*)pristine, (int64_t)(nkeys * kb / 8), 0x5EED5EED5EEDull);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) rc = fail_cuda(e);
    for (int b = b0; b <= b1 && rc == PS_OK; b++) {
        const int64_t n = int64_t(1) << b;
        std::vector<int64_t> off;
        int64_t used = n;
        if (batched) {
            // lengths spread over (2^(b-1), 2^b], the batch bin of 2^b
            off.push_back(0);
            int64_t i = 0;
            while (off.back() + n <= nkeys) {
                const int64_t len = n / 2 + 1 + (int64_t)(((uint64_t)(i * 0x9E3779B97F4A7C15ull) >> 40) % (uint64_t)(n / 2));
                off.push_back(off.back() + len);
                i++;
            }
            used = off.back();
        }
        auto restore = [&]() {
            cudaError_t ce = cudaMemcpyAsync(keys, pristine, (size_t)used * kb, cudaMemcpyDeviceToDevice, s);
            return ce == cudaSuccess ? PS_OK : fail_cuda(ce);
        };
        float best = 1e30f;
        int64_t bnb = 0, bnp = 0;
        for (auto& cand : tune_candidates(n, dtype)) {
            ps_params p;
            memset(&p, 0, sizeof(p));
            p.n_blocks = cand.first;
            p.n_parts = cand.second;
            auto run = [&]() {
                if (batched) return batch_sort(off, keys, dtype, mode, s, nullptr, 0, &p);
                return sort_common(keys, nullptr, n, dtype, mode, &p, nullptr, s);
            };
            float ms = 0.f;
            rc = time_median(run, restore, s, 3, &ms);
            if (rc != PS_OK) break;
            if (ms < best) {
                best = ms;
                bnb = cand.first;
                bnp = cand.second;
            }
        }
        // every launch shape of the family at the fastest (n_B, n_P); the
        // automatic shape (0, 0) is the one timed above
        int32_t bit = 0, bth = 0;
        for (const ShapeEntry* const* sh = all_shapes(); rc == PS_OK && bnb > 0 && *sh; sh++) {
            if ((*sh)->bits != (f == 0 ? 32 : 64)) continue;
            ps_params p;
            memset(&p, 0, sizeof(p));
            p.n_blocks = bnb;
            p.n_parts = bnp;
            p.items_per_thread = (*sh)->items;
            p.block_threads = (*sh)->threads;
            auto run = [&]() {
                if (batched) return batch_sort(off, keys, dtype, mode, s, nullptr, 0, &p);
                return sort_common(keys, nullptr, n, dtype, mode, &p, nullptr, s);
            };
            float ms = 0.f;
            rc = time_median(run, restore, s, 3, &ms);
            if (rc == PS_OK && ms < best) {
                best = ms;
                bit = (*sh)->items;
                bth = (*sh)->threads;
            }
        }
        if (rc == PS_OK && bnb > 0) {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_tune[batched ? 1 : 0][f][b] = TuneEntry{(int32_t)bnb, (int32_t)bnp, bit, bth};
        }
    }
    ws_free(buf, s);
    return rc;
}

// ps_sort_host on page-locked host keys the device can address, for sorts
// of several blocks: the blocks of step 1 are independent, so the host keys
// travel to the device in groups of blocks on a copy stream while the blocks
// that have arrived are sorted (one batched block sort per group: every block
// an instance with one block and one partition, its result kept as order
// keys).  Steps 2 to 4 then run on the sorted blocks.  Exact splitting fixes
// every partition's offset in advance, so the final merge runs over ranges of
// partitions into device memory and each range is copied back while the next
// is merged; regular sampling's final merge writes straight into the host
// buffer.  The host link (about 0.2 TB/s each way on GB300) is the bound; this
// hides the block sort and the final merge behind the transfers.
static constexpr int64_t HOST_PIPE_MIN = int64_t(1) << 24;
#ifndef PS_HOST_GROUPS
#define PS_HOST_GROUPS 8   // block groups copied in while earlier ones sort
#endif
#ifndef PS_HOST_RANGES
#define PS_HOST_RANGES 8   // partition ranges copied out while later ones merge
#endif

static int host_pipelined(const void* host_keys, void* mapped, void* d, int64_t n, int dtype, int mode,
                          const ps_params& r, cudaStream_t s)
{
    const int64_t nb = r.n_blocks, L = (n + nb - 1) / nb;
    const size_t kb = dtype_size(dtype);
    // instance table of the blocks: all starts, then all lengths
    std::vector<int64_t> tab(2 * (size_t)nb);
    for (int64_t b = 0; b < nb; b++) {
        const int64_t bs = std::min(b * L, n), be = std::min(bs + L, n);
        tab[(size_t)b] = bs;
        tab[(size_t)(nb + b)] = be - bs;
    }
    int64_t* dtab = nullptr;
    int rc = ws_alloc((void**)&dtab, tab.size() * 8, s);
    if (rc != PS_OK) return rc;
    cudaError_t e = cudaMemcpyAsync(dtab, tab.data(), tab.size() * 8, cudaMemcpyHostToDevice, s);
    cudaStream_t sc = nullptr;
    const int64_t G = std::max<int64_t>(1, (nb + PS_HOST_GROUPS - 1) / PS_HOST_GROUPS);  // blocks per group
    const int64_t ng = (nb + G - 1) / G;
    std::vector<cudaEvent_t> ev((size_t)ng + 1, nullptr);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sc, cudaStreamNonBlocking);
    for (auto& x : ev)
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming);
    // the copies start once the device buffer exists on s
    if (e == cudaSuccess) e = cudaEventRecord(ev[(size_t)ng], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(sc, ev[(size_t)ng], 0);
    for (int64_t g = 0; g < ng && e == cudaSuccess && rc == PS_OK; g++) {
        const int64_t b0 = g * G, b1 = std::min(nb, b0 + G);
        const int64_t k0 = std::min(b0 * L, n), k1 = std::min(b1 * L, n);
        if (k1 > k0)
            e = cudaMemcpyAsync((char*)d + k0 * kb, (const char*)host_keys + k0 * kb, (size_t)(k1 - k0) * kb,
                                cudaMemcpyHostToDevice, sc);
        if (e == cudaSuccess) e = cudaEventRecord(ev[(size_t)g], sc);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev[(size_t)g], 0);
        if (e != cudaSuccess || k1 <= k0) continue;
        SortArgs a;
        a.keys = d;
        a.payload = nullptr;
        a.n = L;
        a.dtype = dtype;
        a.mode = mode;
        a.n_B = a.n_P = 1;
        a.items = r.items_per_thread;
        a.threads = r.block_threads;
        a.trace = nullptr;
        a.stream = s;
        a.inst_base = dtab + b0;
        a.inst_n = dtab + nb + b0;
        a.n_inst = b1 - b0;
        a.n_max = L;
        a.n_sum = k1 - k0;
        a.extent = n;
        a.keep_order_keys = true;
        rc = dispatch(a);
    }
    void* d2 = nullptr;  // the final merge's device output (exact splitting)
    if (e == cudaSuccess && rc == PS_OK && mode == PS_PIVOT_EXACT && PS_HOST_RANGES > 1)
        rc = ws_alloc(&d2, (size_t)n * kb, s);
    if (e == cudaSuccess && rc == PS_OK) {
        SortArgs a;  // steps 2 to 4 on the sorted blocks, result into the host buffer
        a.keys = d;
        a.payload = nullptr;
        a.n = n;
        a.dtype = dtype;
        a.mode = mode;
        a.n_B = nb;
        a.n_P = r.n_parts;
        a.merge_variant = (int)r.merge_variant;
        a.items = r.items_per_thread;
        a.threads = r.block_threads;
        a.trace = nullptr;
        a.stream = s;
        a.dst_keys = d2 ? d2 : mapped;
        a.host_out = d2 ? const_cast<void*>(host_keys) : nullptr;
        a.copy_stream = d2 ? sc : nullptr;
        a.out_ranges = PS_HOST_RANGES;
        a.presorted = true;
        rc = dispatch(a);
    }
    // the caller waits for s; the copy stream's work is ordered before s's
    // sorts by the events, so both are done once s is.  After a failure some
    // copy may not be ordered before s: wait for the copy stream before the
    // buffers it may still touch go back to the pool.
    if (sc && (e != cudaSuccess || rc != PS_OK)) cudaStreamSynchronize(sc);
    if (d2) ws_free(d2, s);
    if (sc) cudaStreamDestroy(sc);
    for (auto& x : ev)
        if (x) cudaEventDestroy(x);
    ws_free(dtab, s);
    if (e != cudaSuccess) return fail_cuda(e);
    return rc;
}

}  // namespace ps

using namespace ps;

struct ps_batch_plan {
    BatchPlan plan;
    int64_t* table = nullptr;  // device instance table
    char* ws = nullptr;        // device workspace for the largest bin
    size_t ws_bytes = 0;
};

extern "C" {

int ps_sort(void* keys, int64_t n, int dtype, int pivot_mode, ps_stream_t stream)
{
    if (dtype < 0) return PS_ERR_UNSUPPORTED;
    return sort_common(keys, nullptr, n, dtype, pivot_mode, nullptr, nullptr, stream);
}

int ps_sort_ex(void* keys, int64_t n, int dtype, int pivot_mode, const ps_params* params, const ps_trace* trace,
               ps_stream_t stream)
{
    if (dtype < 0) return PS_ERR_UNSUPPORTED;
    return sort_common(keys, nullptr, n, dtype, pivot_mode, params, trace, stream);
}

int ps_sort_pairs(uint64_t* keys, uint32_t* payload, int64_t n, int pivot_mode, const ps_params* params,
                  const ps_trace* trace, ps_stream_t stream)
{
    return sort_common(keys, payload, n, -1, pivot_mode, params, trace, stream);
}

int ps_sort_struct(void* records, int64_t n, int64_t record_bytes, int64_t key_offset, int pivot_mode,
                   const ps_params* params, ps_stream_t stream)
{
    if (n < 0 || n >= (int64_t(1) << 32)) return PS_ERR_INVALID_ARG;
    if (record_bytes < 8 || record_bytes > PS_STRUCT_MAX_BYTES || record_bytes % 8 != 0) return PS_ERR_INVALID_ARG;
    if (key_offset < 0 || key_offset % 8 != 0 || key_offset > record_bytes - 8) return PS_ERR_INVALID_ARG;
    if (pivot_mode != PS_PIVOT_REGULAR && pivot_mode != PS_PIVOT_EXACT) return PS_ERR_UNSUPPORTED;
    const int rc = check_params(params);
    if (rc != PS_OK) return rc;
    if (n <= 1) return PS_OK;
    if (!records || (uintptr_t)records % 8 != 0) return PS_ERR_INVALID_ARG;
    return struct_sort(records, n, record_bytes, key_offset, pivot_mode, params, (cudaStream_t)stream);
}

int ps_sort_batch(const int64_t* seg_offsets, int64_t n_segs, void* keys, int dtype, int pivot_mode,
                  ps_stream_t stream)
{
    if (n_segs < 0) return PS_ERR_INVALID_ARG;
    if (dtype < PS_I32 || dtype > PS_U64) return PS_ERR_UNSUPPORTED;
    if (pivot_mode != PS_PIVOT_REGULAR && pivot_mode != PS_PIVOT_EXACT) return PS_ERR_UNSUPPORTED;
    if (n_segs == 0) return PS_OK;
    if (!seg_offsets || !keys) return PS_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<int64_t> off((size_t)n_segs + 1);
    cudaError_t e = cudaMemcpyAsync(off.data(), seg_offsets, off.size() * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_cuda(e);
    return batch_sort(off, keys, dtype, pivot_mode, s, nullptr, 0);
}

int ps_batch_plan_create(const int64_t* host_seg_offsets, int64_t n_segs, int dtype, int pivot_mode,
                         ps_batch_plan** out)
{
    if (!out) return PS_ERR_INVALID_ARG;
    *out = nullptr;
    if (n_segs < 0 || (n_segs > 0 && !host_seg_offsets)) return PS_ERR_INVALID_ARG;
    if (dtype < PS_I32 || dtype > PS_U64) return PS_ERR_UNSUPPORTED;
    if (pivot_mode != PS_PIVOT_REGULAR && pivot_mode != PS_PIVOT_EXACT) return PS_ERR_UNSUPPORTED;
    std::vector<int64_t> off(host_seg_offsets, host_seg_offsets + (n_segs > 0 ? n_segs + 1 : 0));
    if (off.empty()) off.push_back(0);
    ps_batch_plan* p = new (std::nothrow) ps_batch_plan();
    if (!p) return PS_ERR_NO_MEMORY;
    int rc = batch_make_plan(off, dtype, pivot_mode, nullptr, &p->plan);
    size_t ws = 0;
    for (const BatchBin& bb : p->plan.bins) {
        if (bb.front) continue;
        SortArgs a = batch_bin_args(p->plan, bb, nullptr, nullptr, nullptr);
        int src = PS_OK;
        const ShapeEntry* sh = shape_of(dtype, a.items, a.threads, &src);
        if (src != PS_OK && rc == PS_OK) rc = src;
        ws = std::max(ws, sh ? sh->ws(a) : narrow_dtype(dtype) ? ws_bytes_args_u32(a) : ws_bytes_args_u64(a));
    }
    cudaError_t e = cudaSuccess;
    if (rc == PS_OK && !p->plan.table.empty()) {
        e = cudaMalloc((void**)&p->table, p->plan.table.size() * 8);
        if (e == cudaSuccess)
            e = cudaMemcpy(p->table, p->plan.table.data(), p->plan.table.size() * 8, cudaMemcpyHostToDevice);
        if (e == cudaSuccess && ws > 0) e = cudaMalloc((void**)&p->ws, ws);
        p->ws_bytes = ws;
    }
    if (rc == PS_OK && e != cudaSuccess) rc = fail_cuda(e);
    if (rc != PS_OK) {
        ps_batch_plan_destroy(p);
        return rc;
    }
    *out = p;
    return PS_OK;
}

int ps_batch_run(const ps_batch_plan* plan, void* keys, ps_stream_t stream)
{
    if (!plan) return PS_ERR_INVALID_ARG;
    if (plan->plan.table.empty()) return PS_OK;
    if (!keys || (uintptr_t)keys % (narrow_dtype(plan->plan.dtype) ? 4 : 8) != 0) return PS_ERR_INVALID_ARG;
    return batch_launch(plan->plan, plan->table, keys, (cudaStream_t)stream, plan->ws, plan->ws_bytes);
}

int ps_batch_plan_destroy(ps_batch_plan* plan)
{
    if (!plan) return PS_ERR_INVALID_ARG;
    if (plan->table) cudaFree(plan->table);
    if (plan->ws) cudaFree(plan->ws);
    delete plan;
    return PS_OK;
}

int ps_sort_host(void* host_keys, int64_t n, int dtype, int pivot_mode, const ps_params* params, ps_stream_t stream)
{
    if (dtype < 0 || dtype > PS_U64) return PS_ERR_UNSUPPORTED;
    if (pivot_mode != PS_PIVOT_REGULAR && pivot_mode != PS_PIVOT_EXACT) return PS_ERR_UNSUPPORTED;
    if (n < 0) return PS_ERR_INVALID_ARG;
    int rc = check_params(params);
    if (rc != PS_OK) return rc;
    if (n <= 1) return PS_OK;
    if (!host_keys) return PS_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = (size_t)n * dtype_size(dtype);
    if ((uintptr_t)host_keys % dtype_size(dtype) != 0) return PS_ERR_INVALID_ARG;
    // Page-locked host memory that the device can address directly (mapped
    // pinned memory; on GB300 it travels over NVLink-C2C): the first pass
    // reads the keys from it and the last pass writes the result back into
    // it, so the transfers ride inside the tile sort and the final merge
    // instead of two separate copies.  Other host memory is copied in and out.
    cudaPointerAttributes pa;
    void* mapped = nullptr;
    if (cudaPointerGetAttributes(&pa, host_keys) == cudaSuccess && pa.type == cudaMemoryTypeHost &&
        pa.devicePointer != nullptr)
        mapped = pa.devicePointer;
    cudaGetLastError();  // a pageable pointer may leave an error behind on older drivers
    void* d = nullptr;
    rc = ws_alloc(&d, bytes, s);
    if (rc != PS_OK) return rc;
    cudaError_t e = cudaSuccess;
    ps_params r;
    resolve(n, dtype, params, &r);
    if (mapped && r.n_blocks > 1 && n >= HOST_PIPE_MIN) {
        rc = host_pipelined(host_keys, mapped, d, n, dtype, pivot_mode, r, s);
    } else if (mapped) {
        SortArgs a;
        a.keys = d;
        a.payload = nullptr;
        a.n = n;
        a.dtype = dtype;
        a.mode = pivot_mode;
        a.n_B = r.n_blocks;
        a.n_P = r.n_parts;
        a.merge_variant = (int)r.merge_variant;
        a.items = r.items_per_thread;
        a.threads = r.block_threads;
        a.trace = nullptr;
        a.stream = s;
        a.src_keys = mapped;
        a.dst_keys = mapped;
        rc = dispatch(a);
    } else {
        e = cudaMemcpyAsync(d, host_keys, bytes, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) {
            rc = sort_common(d, nullptr, n, dtype, pivot_mode, params, nullptr, stream);
            if (rc == PS_OK) e = cudaMemcpyAsync(host_keys, d, bytes, cudaMemcpyDeviceToHost, s);
        }
    }
    ws_free(d, s);
    if (e != cudaSuccess) return fail_cuda(e);
    if (rc != PS_OK) return rc;
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_cuda(e);
    return PS_OK;
}

int ps_resolve_params(int64_t n, int dtype, const ps_params* in, ps_params* out)
{
    if (!out || n < 0) return PS_ERR_INVALID_ARG;
    if (dtype < -1 || dtype > PS_U64) return PS_ERR_UNSUPPORTED;
    int rc = check_params(in);
    if (rc != PS_OK) return rc;
    resolve(n, dtype, in, out);
    return PS_OK;
}

int ps_workspace_bytes(int64_t n, int dtype, const ps_params* params, size_t* out)
{
    if (!out || n < 0) return PS_ERR_INVALID_ARG;
    if (dtype < -1 || dtype > PS_U64) return PS_ERR_UNSUPPORTED;
    int rc = check_params(params);
    if (rc != PS_OK) return rc;
    if (n <= 1) {
        *out = 0;
        return PS_OK;
    }
    ps_params r;
    resolve(n, dtype, params, &r);
    const ShapeEntry* sh = shape_of(dtype, r.items_per_thread, r.block_threads, &rc);
    if (rc != PS_OK) return rc;
    if (sh) {
        SortArgs a;
        a.keys = nullptr;
        a.payload = nullptr;
        a.n = n;
        a.dtype = dtype;
        a.mode = PS_PIVOT_REGULAR;
        a.n_B = r.n_blocks;
        a.n_P = r.n_parts;
        a.trace = nullptr;
        a.stream = nullptr;
        *out = sh->ws(a);
        return PS_OK;
    }
    switch (dtype) {
    case PS_I32: case PS_F32: case PS_U32: *out = ws_bytes_u32(n, r.n_blocks, r.n_parts); break;
    case -1: *out = ws_bytes_rec(n, r.n_blocks, r.n_parts); break;
    default: *out = ws_bytes_u64(n, r.n_blocks, r.n_parts); break;
    }
    return PS_OK;
}

int ps_autotune(int dtype, int pivot_mode, int64_t n_min, int64_t n_max, int batched, ps_stream_t stream)
{
    if (tune_family(dtype) < 0) return PS_ERR_UNSUPPORTED;
    if (pivot_mode != PS_PIVOT_REGULAR && pivot_mode != PS_PIVOT_EXACT) return PS_ERR_UNSUPPORTED;
    if (n_min < 2 || n_max < n_min || n_max > (int64_t(1) << 34)) return PS_ERR_INVALID_ARG;
    if (batched != 0 && batched != 1) return PS_ERR_INVALID_ARG;
    return autotune(dtype, pivot_mode, n_min, n_max, batched, (cudaStream_t)stream);
}

int ps_autotune_get(int dtype, int batched, int log2_n, ps_params* out)
{
    const int f = tune_family(dtype);
    if (f < 0) return PS_ERR_UNSUPPORTED;
    if (!out || log2_n < 0 || log2_n > 63 || (batched != 0 && batched != 1)) return PS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const TuneEntry& e = g_tune[batched][f][log2_n];
    if (e.nb <= 0) return PS_ERR_NOT_FOUND;
    memset(out, 0, sizeof(*out));
    out->n_blocks = e.nb;
    out->n_parts = e.np;
    out->items_per_thread = e.items;
    out->block_threads = e.threads;
    return PS_OK;
}

int ps_autotune_set(int dtype, int batched, int log2_n, const ps_params* p)
{
    const int f = tune_family(dtype);
    if (f < 0) return PS_ERR_UNSUPPORTED;
    if (log2_n < 0 || log2_n > 63 || (batched != 0 && batched != 1)) return PS_ERR_INVALID_ARG;
    TuneEntry t{0, 0, 0, 0};
    if (p && (p->n_blocks != 0 || p->n_parts != 0)) {
        if (p->n_blocks < 1 || p->n_blocks > MAX_BLOCKS || p->n_parts < 1 || p->n_parts > MAX_PARTS)
            return PS_ERR_INVALID_ARG;
        if (check_params(p) != PS_OK) return PS_ERR_INVALID_ARG;
        int rc = PS_OK;
        shape_of(f == 0 ? PS_U32 : PS_U64, p->items_per_thread, p->block_threads, &rc);
        if (rc != PS_OK) return rc;
        t = TuneEntry{(int32_t)p->n_blocks, (int32_t)p->n_parts, p->items_per_thread, p->block_threads};
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[batched][f][log2_n] = t;
    return PS_OK;
}

const char* ps_status_string(int status)
{
    switch (status) {
    case PS_OK: return "ok";
    case PS_ERR_INVALID_ARG: return "invalid argument";
    case PS_ERR_UNSUPPORTED: return "unsupported dtype or pivot mode";
    case PS_ERR_NO_MEMORY: return "out of device memory";
    case PS_ERR_CUDA: return "CUDA runtime error";
    case PS_ERR_BUSY: return "busy: admission budget or in-flight limit reached";
    case PS_ERR_TIMEOUT: return "timed out";
    case PS_ERR_NOT_FOUND: return "unknown request id";
    default: return "unknown status";
    }
}

int ps_last_cuda_error(void) { return g_last_cuda; }

int ps_debug_fail_alloc(int count)
{
    if (count < 0) return PS_ERR_INVALID_ARG;
    g_fail_alloc.store(count);
    return PS_OK;
}

int ps_debug_violation(uint64_t* out)
{
    if (!out) return PS_ERR_INVALID_ARG;
    unsigned long long v[4];
    int (*readers[3])(unsigned long long*) = {viol_read_u32, viol_read_u64, viol_read_rec};
    int found = 0;
    for (int f = 0; f < 3; f++) {
        int rc = readers[f](v);
        if (rc < 0) return rc;
        if (rc == 1 && !found) {
            out[0] = v[0] + 100ull * (unsigned long long)f;
            out[1] = v[1];
            out[2] = v[2];
            out[3] = v[3];
            found = 1;
        }
    }
    if (!found)
        for (int i = 0; i < 4; i++) out[i] = 0;
    return found;
}

int ps_profile_enable(int on) { return g_prof.exchange(on != 0) ? 1 : 0; }

int ps_profile_read(ps_kernel_stat* out, int cap, int* n)
{
    if (!n || cap < 0 || (cap > 0 && !out)) return PS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    std::vector<ps_kernel_stat> agg;
    for (auto& r : g_prof_recs) {
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e != cudaSuccess) return fail_cuda(e);
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, r.a, r.b);
        if (e != cudaSuccess) return fail_cuda(e);
        size_t i = 0;
        for (; i < agg.size(); i++)
            if (r.name == agg[i].name) break;
        if (i == agg.size()) {
            ps_kernel_stat st;
            memset(&st, 0, sizeof(st));
            strncpy(st.name, r.name.c_str(), sizeof(st.name) - 1);
            agg.push_back(st);
        }
        agg[i].launches++;
        agg[i].total_ms += ms;
    }
    int k = 0;
    for (; k < (int)agg.size() && k < cap; k++) out[k] = agg[k];
    *n = (int)agg.size();
    return PS_OK;
}

int ps_profile_reset(void)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    prof_clear();
    return PS_OK;
}

}  // extern "C"

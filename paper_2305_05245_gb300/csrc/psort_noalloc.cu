// psort_noalloc.cu -- ps_sort_noalloc: the sort on a static device array, for
// callers that must not allocate device memory (see include/psort.h).
#include <cstring>
#include <mutex>
#include <vector>

#include "psort_internal.h"

namespace ps {

// The workspace of every ps_sort_noalloc call on a device.  Host code must not
// pass this name to a kernel (on the host it is only a stand-in symbol); it
// uses the device address that cudaGetSymbolAddress returns instead.
static __device__ __align__(256) unsigned char g_noalloc_scratch[PS_NOALLOC_SCRATCH_BYTES];

// Device address of the array in the current CUDA context, looked up once per
// context on the first call made in it.  The key is the context's unique ID
// (cuCtxGetId), not the device ordinal: a module-scope array has its own
// address in every context, a cudaDeviceReset replaces the primary context
// (and may move the array), and a caller may run in a context of its own on
// the same device.  IDs are never reused within a process, so a cached
// address is never handed to a context it does not belong to.  The two
// driver functions are fetched through the runtime, so the library does not
// link the driver library itself.
typedef int (*ctx_get_current_fn)(void**);
typedef int (*ctx_get_id_fn)(void*, unsigned long long*);

struct NoallocCache {
    std::mutex mu;
    ctx_get_current_fn get_current = nullptr;
    ctx_get_id_fn get_id = nullptr;
    struct Entry {
        unsigned long long ctx_id;
        void* addr;
    };
    std::vector<Entry> entries;
};
static NoallocCache& noalloc_cache()
{
    static NoallocCache c;
    return c;
}

static int noalloc_scratch(void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail_cuda(e);
    NoallocCache& c = noalloc_cache();
    std::lock_guard<std::mutex> lk(c.mu);
    if (!c.get_current || !c.get_id) {
        cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
        void* f1 = nullptr;
        void* f2 = nullptr;
        e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1);
        if (e == cudaSuccess)
            e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
        if (e != cudaSuccess) return fail_cuda(e);
        if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
            return PS_ERR_UNSUPPORTED;
        c.get_current = (ctx_get_current_fn)f1;
        c.get_id = (ctx_get_id_fn)f2;
    }
    void* ctx = nullptr;
    unsigned long long id = 0;
    if (c.get_current(&ctx) != 0) return fail_cuda(cudaErrorDeviceUninitialized);
    if (!ctx) {
        // no context bound to this thread yet: the runtime's first real call
        // (this lookup; it allocates nothing) creates the device's primary one
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return fail_cuda(e);
        if (c.get_current(&ctx) != 0 || !ctx) return fail_cuda(cudaErrorDeviceUninitialized);
    }
    if (c.get_id(ctx, &id) != 0) return fail_cuda(cudaErrorDeviceUninitialized);
    for (const auto& x : c.entries)
        if (x.ctx_id == id) {
            *out = x.addr;
            return PS_OK;
        }
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return fail_cuda(e != cudaSuccess ? e : cudaErrorInvalidSymbol);
    c.entries.push_back({id, p});
    *out = p;
    return PS_OK;
}

}  // namespace ps

using namespace ps;

extern "C" int ps_sort_noalloc(void* keys, int64_t n, int dtype, int pivot_mode, ps_stream_t stream)
{
    if (n < 0 || n > PS_NOALLOC_MAX_KEYS) return PS_ERR_INVALID_ARG;
    if (dtype < PS_I32 || dtype > PS_U64) return PS_ERR_UNSUPPORTED;
    if (pivot_mode != PS_PIVOT_REGULAR && pivot_mode != PS_PIVOT_EXACT) return PS_ERR_UNSUPPORTED;
    if (n <= 1) return PS_OK;
    const bool narrow = dtype == PS_I32 || dtype == PS_F32 || dtype == PS_U32;
    if (!keys || (uintptr_t)keys % (narrow ? 4 : 8) != 0) return PS_ERR_INVALID_ARG;
    // the size heuristic, not tuned entries: the scratch is sized for it
    ps_params r;
    resolve_default(n, dtype, &r);
    void* ws = nullptr;
    int rc = noalloc_scratch(&ws);
    if (rc != PS_OK) return rc;
    SortArgs a;
    a.keys = keys;
    a.payload = nullptr;
    a.n = n;
    a.dtype = dtype;
    a.mode = pivot_mode;
    a.n_B = r.n_blocks;
    a.n_P = r.n_parts;
    a.trace = nullptr;
    a.stream = (cudaStream_t)stream;
    return narrow ? run_sort_u32_on(a, (char*)ws, PS_NOALLOC_SCRATCH_BYTES)
                  : run_sort_u64_on(a, (char*)ws, PS_NOALLOC_SCRATCH_BYTES);
}

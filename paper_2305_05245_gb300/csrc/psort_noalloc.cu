// psort_noalloc.cu -- ps_sort_noalloc: the sort on a static device array, for
// callers that must not allocate device memory (see include/psort.h).
#include <cstring>
#include <mutex>

#include "psort_internal.h"

namespace ps {

// The workspace of every ps_sort_noalloc call on a device.  Host code must not
// pass this name to a kernel (on the host it is only a stand-in symbol); it
// uses the device address that cudaGetSymbolAddress returns instead.
static __device__ __align__(256) unsigned char g_noalloc_scratch[PS_NOALLOC_SCRATCH_BYTES];

static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[64];

// Device address of the array on the current device; looked up once per
// device, on the first call made with that device current.
static int noalloc_scratch(void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail_cuda(e);
    if (dev < 0 || dev >= 64) return PS_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return fail_cuda(e != cudaSuccess ? e : cudaErrorInvalidSymbol);
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
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

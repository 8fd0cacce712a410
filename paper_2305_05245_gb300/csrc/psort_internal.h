// psort_internal.h -- host-side declarations shared by the library's
// translation units (not part of the public ABI).
#pragma once

#include <cstddef>
#include <algorithm>
#include <cstdint>
#include <vector>
#include <cuda_runtime.h>

#include "../../include/psort.h"

namespace ps {

// One sort request after argument validation and parameter resolution.
struct SortArgs {
    void* keys;          // device keys (records: uint64 keys)
    uint32_t* payload;   // records only
    int64_t n;
    int dtype;           // ps_dtype, or -1 for records
    int mode;            // ps_pivot_mode
    int64_t n_B, n_P;    // resolved
    int merge_variant = 0;  // ps_merge_variant of step 4
    // Launch shape of the data passes (ps_params items_per_thread and
    // block_threads); 0, 0 = the family's automatic shape.
    int items = 0, threads = 0;
    const ps_trace* trace;
    cudaStream_t stream;
    // Batched sorts: n_inst independent instances sharing n_B and n_P, with
    // device arrays of their starts and lengths.  inst_base == nullptr means
    // one sort of n keys at offset 0.
    const int64_t* inst_base = nullptr;
    const int64_t* inst_n = nullptr;
    int64_t n_inst = 1;
    int64_t n_max = 0;   // longest instance
    int64_t n_sum = 0;   // keys over all instances
    int64_t extent = 0;  // extent of the key arrays (largest end offset)
    // Optional separate ends of a keys-only sort: the first pass reads src_keys
    // and the last pass writes dst_keys (n keys each, any memory the device
    // can address, e.g. mapped pinned host memory); `keys` is then device
    // scratch for the passes in between.  nullptr: both are `keys`.
    const void* src_keys = nullptr;
    void* dst_keys = nullptr;
    // The block sort's last pass keeps the order keys (no inverse transform):
    // used to sort the blocks of a larger sort ahead of its steps 2 to 4.
    bool keep_order_keys = false;
    // Step 1 is done already: `keys` holds every block of the sort sorted, as
    // order keys; the call runs steps 2 to 4 only (dst_keys must be given).
    bool presorted = false;
    // Exact splitting, one instance: step 4 runs over out_ranges ranges of
    // partitions into dst_keys (device), and each range's output is copied to
    // host_out on copy_stream as soon as it is merged (partition k starts at
    // floor(k*n/n_P), known on the host).  The caller's stream waits for the
    // copies.
    void* host_out = nullptr;
    cudaStream_t copy_stream = nullptr;
    int out_ranges = 0;
    // Batched keys-only sorts whose instances live in buffers of their own:
    // device table of one device pointer per instance (in instance-table
    // order).  The first pass reads each instance from its buffer and the
    // last pass writes it back there; `keys` (extent keys, laid out by
    // inst_base) only carries the passes in between.
    void* const* inst_ptrs = nullptr;
};

// Workspace from the library's stream-ordered pool.
int ws_alloc(void** p, size_t bytes, cudaStream_t s);
void ws_free(void* p, cudaStream_t s);
int fail_cuda(cudaError_t e);

// Profiling: when enabled (ps_profile_enable), a ProfScope records a CUDA
// event before and after the launch it brackets.
bool prof_on();
int prof_begin(const char* name, cudaStream_t s);  // returns a record index or -1
void prof_end(int rec, cudaStream_t s);
struct ProfScope {
    int rec;
    cudaStream_t s;
    ProfScope(const char* name, cudaStream_t st) : rec(prof_on() ? prof_begin(name, st) : -1), s(st) {}
    ~ProfScope()
    {
        if (rec >= 0) prof_end(rec, s);
    }
};

// Per key family (defined in psort_u32.cu, psort_u64.cu, psort_rec.cu).
int run_sort_u32(const SortArgs& a);
int run_sort_u64(const SortArgs& a);
int run_sort_rec(const SortArgs& a);
size_t ws_bytes_u32(int64_t n, int64_t n_B, int64_t n_P);
size_t ws_bytes_u64(int64_t n, int64_t n_B, int64_t n_P);
size_t ws_bytes_rec(int64_t n, int64_t n_B, int64_t n_P);
// Index-violation records of the checked build (one per key family).
int viol_read_u32(unsigned long long* out);
int viol_read_u64(unsigned long long* out);
int viol_read_rec(unsigned long long* out);
// Batched sort of the segments [off[i], off[i+1]) of keys (host offsets).
// pinned (optional): page-locked host scratch of pinned_cap int64 for the
// instance table; when given, the call does not wait for the stream.
// force (optional): n_B/n_P for every bin above the one-tile bin (tuning).
// own (optional, keys-only): one device pointer per segment; each segment is
// then read from and written back to its own buffer, and keys only carries
// the passes in between (off lays the segments out in it).  The instance
// table then holds 3 int64 per segment instead of 2.
int batch_sort(const std::vector<int64_t>& off, void* keys, int dtype, int mode, cudaStream_t s,
               int64_t* pinned, size_t pinned_cap, const ps_params* force = nullptr,
               const std::vector<void*>* own = nullptr);
// The size heuristic alone (no tuned entries), with every field automatic.
void resolve_default(int64_t n, int dtype, ps_params* out);
// Records (uint64 key, uint32 payload) through the validated record path.
int sort_records(uint64_t* keys, uint32_t* payload, int64_t n, int mode, const ps_params* params, cudaStream_t s);
// Fixed-size records sorted by an embedded uint64 key (arguments validated).
int struct_sort(void* records, int64_t n, int64_t rb, int64_t ko, int mode, const ps_params* params,
                cudaStream_t s);
// Workspace bytes of a single sort of n keys with automatic parameters.
size_t sort_ws_bytes(int64_t n, int dtype);
// The same sorts on a caller-provided workspace (allocation-free entry point).
int run_sort_u32_on(const SortArgs& a, char* ws, size_t cap);
int run_sort_u64_on(const SortArgs& a, char* ws, size_t cap);
// The short instances of a batch in one persistent launch: t (optional)
// instances of at most one tile, sm (optional) instances of at most
// SMALL_SEG keys; next: a device counter the call zeroes on the stream.
int run_front_u32(const SortArgs* t, const SortArgs* sm, unsigned long long* next);
int run_front_u64(const SortArgs* t, const SortArgs* sm, unsigned long long* next);
constexpr int64_t SMALL_SEG = 1024;
// Workspace bytes of the sort a describes (batched instances included).
size_t ws_bytes_args_u32(const SortArgs& a);
size_t ws_bytes_args_u64(const SortArgs& a);

// Keys-only pipelines compiled for other launch shapes than the automatic one
// (one translation unit per shape: psort_shape.cu built with -D flags).
struct ShapeEntry {
    int bits;     // key width: 32 or 64
    int items;    // keys per thread of the tile sort and the chunk merge
    int threads;  // threads per CTA of both
    int (*run)(const SortArgs&);
    size_t (*ws)(const SortArgs&);
    int (*run_on)(const SortArgs&, char* ws, size_t cap);  // on a caller's workspace
};
// The entry for (bits, items, threads), or nullptr if none was compiled.
const ShapeEntry* find_shape(int bits, int items, int threads);
// Every compiled shape (for the autotuner), terminated by a null entry.
const ShapeEntry* const* all_shapes();

}  // namespace ps

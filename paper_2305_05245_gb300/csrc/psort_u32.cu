// psort_u32.cu -- kernels and pipeline instantiated for the uint32_t key family.
#include "psort_pipeline.cuh"

namespace ps {
int run_sort_u32(const SortArgs& a) { return Pipeline<uint32_t>::run(a); }
size_t ws_bytes_u32(int64_t n, int64_t n_B, int64_t n_P) { return Pipeline<uint32_t>::ws_bytes(n, n_B, n_P); }
int run_sort_u32_on(const SortArgs& a, char* ws, size_t cap) { return Pipeline<uint32_t>::run_on(a, ws, cap); }
}  // namespace ps

// psort_rec.cu -- kernels and pipeline instantiated for the Rec key family.
#include "psort_pipeline.cuh"

namespace ps {
int run_sort_rec(const SortArgs& a) { return Pipeline<Rec>::run(a); }
size_t ws_bytes_rec(int64_t n, int64_t n_B, int64_t n_P) { return Pipeline<Rec>::ws_bytes(n, n_B, n_P); }
}  // namespace ps

// psort_rec.cu -- kernels and pipeline instantiated for the Rec key family.
#include "psort_pipeline.cuh"

namespace ps {
int run_sort_rec(const SortArgs& a) { return Pipeline<Rec>::run(a); }
size_t ws_bytes_rec(int64_t n, int64_t n_B, int64_t n_P) { return Pipeline<Rec>::ws_bytes(n, n_B, n_P); }
// First recorded index violation of this family's kernels (checked builds);
// clears the record.  Returns 1 if one was recorded, 0 if none.
int viol_read_rec(unsigned long long* out)
{
#ifdef PS_CHECKED
    cudaError_t e = cudaMemcpyFromSymbol(out, ps_viol, 4 * sizeof(unsigned long long));
    if (e != cudaSuccess) return fail_cuda(e);
    const unsigned long long zero[4] = {0, 0, 0, 0};
    e = cudaMemcpyToSymbol(ps_viol, zero, sizeof(zero));
    if (e != cudaSuccess) return fail_cuda(e);
    return out[0] ? 1 : 0;
#else
    for (int i = 0; i < 4; i++) out[i] = 0;
    return 0;
#endif
}
}  // namespace ps

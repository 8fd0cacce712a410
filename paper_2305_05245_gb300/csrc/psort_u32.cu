// psort_u32.cu -- kernels and pipeline instantiated for the uint32_t key family.
#include "psort_pipeline.cuh"

namespace ps {
int run_sort_u32(const SortArgs& a) { return Pipeline<uint32_t>::run(a); }
size_t ws_bytes_u32(int64_t n, int64_t n_B, int64_t n_P) { return Pipeline<uint32_t>::ws_bytes(n, n_B, n_P); }
int run_sort_u32_on(const SortArgs& a, char* ws, size_t cap) { return Pipeline<uint32_t>::run_on(a, ws, cap); }
int run_front_u32(const SortArgs* t, const SortArgs* sm, unsigned long long* next)
{
    return Pipeline<uint32_t>::run_front(t, sm, next);
}
size_t ws_bytes_args_u32(const SortArgs& a) { return Pipeline<uint32_t>::ws_bytes_for(a); }
// First recorded index violation of this family's kernels (checked builds);
// clears the record.  Returns 1 if one was recorded, 0 if none.
int viol_read_u32(unsigned long long* out)
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

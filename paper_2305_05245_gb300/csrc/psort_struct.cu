// psort_struct.cu -- sorting fixed-size records by an embedded uint64 key
// (Table 1's Pair and Particle inputs).  The four steps run on (key,
// position) pairs; the records themselves move once, by a gather.
#include "psort_internal.h"

namespace ps {

// Copy every record into the workspace and pull out its key and position.
// One thread per 8-byte word of the array; the word at key_offset of record
// i also becomes keys[i] (with pos[i] = i).
__global__ void k_struct_split(const uint64_t* rec, uint64_t* copy, int64_t words_total, int words,
                               int key_word, uint64_t* keys, uint32_t* pos)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < words_total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t v = rec[t];
        copy[t] = v;
        const int64_t i = t / words;
        if (t - i * words == key_word) {
            keys[i] = v;
            pos[i] = (uint32_t)i;
        }
    }
}

// records[i] = copy[pos[i]], W-sized words (8 or 16 bytes), one thread per
// word of the output (coalesced stores; each record is read contiguously).
template <typename W>
__global__ void k_struct_gather(const W* copy, W* rec, const uint32_t* pos, int64_t words_total, int words)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < words_total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / words;
        const int w = (int)(t - i * words);
        rec[t] = copy[(int64_t)pos[i] * words + w];
    }
}

static unsigned grid_for(int64_t work)
{
    const int64_t g = (work + 255) / 256;
    return (unsigned)std::min<int64_t>(g, 152 * 16);
}

int struct_sort(void* records, int64_t n, int64_t rb, int64_t ko, int mode, const ps_params* params,
                cudaStream_t s)
{
    const size_t copy_bytes = (size_t)n * (size_t)rb;
    const size_t pair_off = (copy_bytes + 255) & ~(size_t)255;
    const size_t pos_off = pair_off + (((size_t)n * 8 + 255) & ~(size_t)255);
    const size_t total = pos_off + (size_t)n * 4;
    char* ws = nullptr;
    int rc = ws_alloc((void**)&ws, total, s);
    if (rc != PS_OK) return rc;
    uint64_t* keys = (uint64_t*)(ws + pair_off);
    uint32_t* pos = (uint32_t*)(ws + pos_off);
    const int words = (int)(rb / 8);
    const int64_t wt = n * words;
    {
        ProfScope ps_("struct_split", s);
        k_struct_split<<<grid_for(wt), 256, 0, s>>>((const uint64_t*)records, (uint64_t*)ws, wt, words,
                                                   (int)(ko / 8), keys, pos);
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        rc = sort_records(keys, pos, n, mode, params, s);
        if (rc == PS_OK) {
            ProfScope ps_("struct_gather", s);
            if (rb % 16 == 0 && (uintptr_t)records % 16 == 0) {
                const int64_t w16 = n * (rb / 16);
                k_struct_gather<uint4><<<grid_for(w16), 256, 0, s>>>((const uint4*)ws, (uint4*)records, pos, w16,
                                                                    (int)(rb / 16));
            } else {
                k_struct_gather<uint64_t><<<grid_for(wt), 256, 0, s>>>((const uint64_t*)ws, (uint64_t*)records,
                                                                      pos, wt, words);
            }
            e = cudaGetLastError();
        }
    }
    ws_free(ws, s);
    if (rc != PS_OK) return rc;
    if (e != cudaSuccess) return fail_cuda(e);
    return PS_OK;
}

}  // namespace ps

// psort_pipeline.cuh -- host orchestration of one sort for one key family:
// workspace plan, kernel launches of the four steps, trace output.
#pragma once

#include <algorithm>
#include <cmath>
#include <mutex>
#include <type_traits>
#include <vector>

#include "psort_internal.h"
#include "psort_kernels.cuh"

namespace ps {

// Threads per CTA and keys per thread of the tile sort (TNT, TE), warp-shuffle
// merge levels of the tile sort (TW), of the chunk merge (MNT, ME; MNT*ME is
// the chunk capacity) and of the sample pool (PNT, PE; PNT*PE samples).
// Sample pools measured on GB300 (2^30 keys): 64-bit keys 512 x 8 (planning
// 5.2 -> 4.7 ms against 1024 x 8, although it takes a third refinement level
// in places), 32-bit keys 1024 x 8, records 512 x 8.  Records merge chunks of
// 512 x 16 (8192 records, 2 CTAs per SM): half the chunks of 256 x 16, so
// planning drops from 3.3 to 2.0 ms at 2^28 for 0.6 ms more in the merges.
// Shuffle levels measured on GB300 (2^30 keys): 64-bit keys 2 (a shuffle
// level's compare-exchanges cost more ALU work than a shared-memory level
// beyond that), 32-bit keys 5 (all levels inside a warp); records (2^28) 1.
#ifndef PS_TILE_WLEV32
#define PS_TILE_WLEV32 5
#endif
#ifndef PS_TILE_WLEV64
#define PS_TILE_WLEV64 2
#endif
#ifndef PS_TILE_WLEVREC
#define PS_TILE_WLEVREC 1
#endif
// Target chunk size of a merge, in percent of the room a chunk has after the
// average padding (splitters land within a few percent of their targets;
// oversized chunks take the exact sub-chunk path).
#ifndef PS_MERGE_FILL
#define PS_MERGE_FILL 90
#endif
// Sample-pool samples per child, as a multiple of the fan-in (at least 96),
// and the most children one refinement level makes.
#ifndef PS_POOL_SPC
#define PS_POOL_SPC 2
#endif
#ifndef PS_POOL_JMAX
#define PS_POOL_JMAX 64
#endif
template <typename K> struct Cfg;
template <> struct Cfg<uint32_t> {
    static constexpr int TNT = 256, TE = 32, TW = PS_TILE_WLEV32, MNT = 512, ME = 32, PNT = 1024, PE = 8;
};
template <> struct Cfg<uint64_t> {
    static constexpr int TNT = 256, TE = 32, TW = PS_TILE_WLEV64, MNT = 256, ME = 32, PNT = 512, PE = 8;
};
template <> struct Cfg<Rec> {
    static constexpr int TNT = 256, TE = 16, TW = PS_TILE_WLEVREC, MNT = 512, ME = 16, PNT = 512, PE = 8;
};

constexpr int64_t FMAX = 256;  // largest fan-in of one in-block merge pass
constexpr int MAXLEV = 6;     // refinement levels of one merge job

template <typename K> struct GStore {
    static constexpr size_t bytes = sizeof(K);
};
template <> struct GStore<Rec> {
    static constexpr size_t bytes = 12;  // uint64 key + uint32 payload, structure of arrays
};

static inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Shape of one merge job: fan-in K, refinement levels, the group capacity
// of every level and each level's target child size.
struct MergeShape {
    int K, nlev;
    int64_t G[MAXLEV + 1];
    int64_t cnom[MAXLEV];
    int64_t jcap;
    size_t bytes;
    // byte offsets inside the job's workspace
    size_t o_lo[MAXLEV + 1], o_hi[MAXLEV + 1], o_base[MAXLEV + 1], o_size[MAXLEV + 1], o_ng[MAXLEV + 1];
    size_t o_choff[MAXLEV], o_chgrp[MAXLEV], o_spl[MAXLEV], o_big;
};

// Everything the launches need to know about one sort's shape.
template <typename K, typename CF = Cfg<K>> struct Plan {
    static constexpr int T = CF::TNT * CF::TE;    // tile
    static constexpr int CAP = CF::MNT * CF::ME;  // merge chunk capacity
    static constexpr int POOL = CF::PNT * CF::PE;
    int64_t N;      // extent of the key arrays
    int64_t n_inst; // instances (1 for a single sort)
    int64_t Nmax;   // longest instance
    int64_t Nsum;   // keys over all instances
    int64_t n_B, n_P, L, R0;
    int mode;
    bool direct;    // n_B = n_P = 1: the block sort is the whole sort
    int npass;
    int64_t F[16];
    MergeShape inblock[16], fin;
    // workspace byte offsets
    size_t o_data, o_split, o_off, o_piv, o_c, o_samp, o_merge, total;

    // Chunks of a fan-in K merge are merged with their pieces padded to
    // multiples of ME (aligned merge) while K*(ME-1), the worst-case padding,
    // stays within a quarter of the capacity.
    static bool aligned(int64_t K_) { return K_ * (CF::ME - 1) * 4 <= CAP; }
    // chunks aim at 85% of the capacity left after the average padding
    // (splitters land within about 10% of their targets); oversized ones take
    // the slow exact path
    static int64_t cnom(int64_t K_)
    {
        const int64_t room = aligned(K_) ? CAP - K_ * (CF::ME - 1) / 2 : CAP;
        return room * PS_MERGE_FILL / 100;
    }
    static int64_t jcap(int64_t K_) { return std::max<int64_t>(1, (POOL / 2 - K_) / 2); }
    // children per refinement level: the pool takes about max(SPC*K, 96)
    // samples per child, so J is capped near POOL/max(SPC*K, 96)
    static int64_t jlevel(int64_t K_)
    {
        int64_t ji = POOL / std::max<int64_t>(PS_POOL_SPC * K_, 96);
        ji = std::min<int64_t>(PS_POOL_JMAX, std::max<int64_t>(2, ji));
        return std::min(ji, jcap(K_));
    }

    MergeShape shape(int K_, int64_t G0, int64_t Mmax) const
    {
        MergeShape m{};
        m.K = K_;
        m.jcap = jcap(K_);
        const int64_t jl = jlevel(K_);
        int64_t need = (Mmax + cnom(K_) - 1) / cnom(K_);
        m.nlev = 0;
        if (jl >= 2)
            for (int64_t x = need; x > 1 && m.nlev < MAXLEV; x = (x + jl - 1) / jl) m.nlev++;
        m.G[0] = G0;
        for (int l = 0; l < m.nlev; l++) {
            int64_t c = cnom(K_);
            for (int q = 0; q < m.nlev - 1 - l; q++) c *= jl;
            m.cnom[l] = c;
            m.G[l + 1] = Nsum / c + m.G[l] + 1;
        }
        size_t o = 0;
        for (int l = 0; l <= m.nlev; l++) {
            m.o_lo[l] = o;
            o += align256((size_t)m.G[l] * K_ * 8);
            m.o_hi[l] = o;
            o += align256((size_t)m.G[l] * K_ * 8);
            m.o_base[l] = o;
            o += align256((size_t)m.G[l] * 8);
            m.o_size[l] = o;
            o += align256((size_t)m.G[l] * 8);
            m.o_ng[l] = o;
            o += 256;
        }
        for (int l = 0; l < m.nlev; l++) {
            m.o_choff[l] = o;
            o += align256((size_t)(m.G[l] + 1) * 8);
            m.o_chgrp[l] = o;
            o += align256((size_t)m.G[l + 1] * 4);
            m.o_spl[l] = o;
            o += align256((size_t)m.G[l + 1] * sizeof(Splitter<K>));
        }
        m.o_big = o;  // counter, then the list of oversized groups
        o += align256((size_t)(m.G[m.nlev] + 1) * 8);
        m.bytes = o;
        return m;
    }

    void make(int64_t extent, int64_t ninst, int64_t nmax, int64_t nsum, int64_t nb, int64_t np, int md)
    {
        N = extent;
        n_inst = ninst;
        Nmax = nmax;
        Nsum = nsum;
        n_B = nb;
        n_P = np;
        mode = md;
        direct = n_B == 1 && n_P == 1;
        L = (Nmax + n_B - 1) / n_B;
        R0 = std::max<int64_t>(1, (L + T - 1) / T);
        npass = 0;
        for (int64_t x = R0; x > 1; x = (x + FMAX - 1) / FMAX) npass++;
        size_t mbytes = 0;
        int64_t R = R0, W = T;
        for (int p = 0; p < npass; p++) {
            // A pass of fan-in F merges its chunks in ceil(log2 F) shared-memory
            // levels, so fan-ins are powers of two that share the ceil(log2 R)
            // levels still needed evenly, smaller first: 2048 runs take 32 x 64
            // (11 levels) rather than 46 x 45 (12 levels).  (Smaller first plans
            // 0.15 ms faster than larger first at 2^30 keys; the merges cost the
            // same.)  The levels left never exceed 8 per pass left, so the last
            // fan-in stays within FMAX = 2^8.
            const int rem = npass - p;
            int lvl = 0;
            while ((int64_t(1) << lvl) < R) lvl++;
            const int lp = lvl / rem;
            F[p] = std::min<int64_t>(std::min<int64_t>(int64_t(1) << lp, FMAX), R);
            const int64_t Rp = (L + W - 1) / W;
            const int64_t gpb = (Rp + F[p] - 1) / F[p];
            inblock[p] = shape((int)F[p], n_inst * n_B * gpb, std::min<int64_t>(F[p] * W, L));
            mbytes = std::max(mbytes, inblock[p].bytes);
            R = (R + F[p] - 1) / F[p];
            W *= F[p];
        }
        const int64_t mmax = mode == PS_PIVOT_EXACT ? (Nmax + n_P - 1) / n_P + 1 : Nmax;
        if (!direct) {
            fin = shape((int)n_B, n_inst * n_P, mmax);
            mbytes = std::max(mbytes, fin.bytes);
        }
        size_t o = 0;
        o_data = o;
        o += align256((size_t)N * GStore<K>::bytes + 256);
        o_split = o;
        o += align256((size_t)n_inst * n_B * (n_P + 1) * 8);
        o_off = o;
        o += align256((size_t)n_inst * (n_P + 1) * 8);
        o_piv = o;
        o += align256((size_t)n_inst * n_P * sizeof(K));
        o_c = o;
        o += align256((size_t)n_inst * n_P * 8);
        o_samp = o;
        o += align256((size_t)n_inst * n_B * std::max<int64_t>(n_P - 1, 1) * GStore<K>::bytes + 256);
        o_merge = o;
        o += mbytes;
        total = o;
    }
};

template <typename K> static GBuf<K> gbuf_at(char* base, int64_t n);
template <> inline GBuf<uint32_t> gbuf_at<uint32_t>(char* base, int64_t n) { return GBuf<uint32_t>{(uint32_t*)base, n}; }
template <> inline GBuf<uint64_t> gbuf_at<uint64_t>(char* base, int64_t n) { return GBuf<uint64_t>{(uint64_t*)base, n}; }
template <> inline GBuf<Rec> gbuf_at<Rec>(char* base, int64_t n)
{
    return GBuf<Rec>{(uint64_t*)base, (uint32_t*)(base + align256((size_t)n * 8)), n};
}

template <typename K> static GBuf<K> gbuf_user(const SortArgs& a);
// the caller's arrays span the single sort, or every segment of a batch
static inline int64_t user_extent(const SortArgs& a) { return a.inst_base ? a.extent : a.n; }
template <> inline GBuf<uint32_t> gbuf_user<uint32_t>(const SortArgs& a) { return GBuf<uint32_t>{(uint32_t*)a.keys, user_extent(a)}; }
template <> inline GBuf<uint64_t> gbuf_user<uint64_t>(const SortArgs& a) { return GBuf<uint64_t>{(uint64_t*)a.keys, user_extent(a)}; }
template <> inline GBuf<Rec> gbuf_user<Rec>(const SortArgs& a) { return GBuf<Rec>{(uint64_t*)a.keys, a.payload, user_extent(a)}; }

// A keys-only buffer at p (the separate first-pass source / last-pass
// destination of SortArgs); records never take this path.
template <typename K> static GBuf<K> gbuf_ext(const void* p, const GBuf<K>& fallback);
template <> inline GBuf<uint32_t> gbuf_ext<uint32_t>(const void* p, const GBuf<uint32_t>& f)
{
    return p ? GBuf<uint32_t>{(uint32_t*)p, f.n} : f;
}
template <> inline GBuf<uint64_t> gbuf_ext<uint64_t>(const void* p, const GBuf<uint64_t>& f)
{
    return p ? GBuf<uint64_t>{(uint64_t*)p, f.n} : f;
}
template <> inline GBuf<Rec> gbuf_ext<Rec>(const void*, const GBuf<Rec>& f) { return f; }

// Base address of a keys-only buffer (records have no single base).
template <typename K> static const void* last_ptr(const GBuf<K>& b) { return b.p; }
template <> inline const void* last_ptr<Rec>(const GBuf<Rec>& b) { return b.k; }

template <typename K> static bool same_buf(const GBuf<K>& x, const GBuf<K>& y);
template <> inline bool same_buf<uint32_t>(const GBuf<uint32_t>& x, const GBuf<uint32_t>& y) { return x.p == y.p; }
template <> inline bool same_buf<uint64_t>(const GBuf<uint64_t>& x, const GBuf<uint64_t>& y) { return x.p == y.p; }
template <> inline bool same_buf<Rec>(const GBuf<Rec>& x, const GBuf<Rec>& y) { return x.k == y.k; }

// Profiler label of planning kernel `what` (0 chunk plan, 1 sample pool, 2
// co-ranks, 3 child windows) at refinement level l of an in-block or final
// merge job.
static inline const char* level_label(bool fin, int what, int l)
{
    static const char* const names[2][4][3] = {
        {{"plan_inblock_l1", "plan_inblock_l2", "plan_inblock_l3"},
         {"pool_inblock_l1", "pool_inblock_l2", "pool_inblock_l3"},
         {"corank_inblock_l1", "corank_inblock_l2", "corank_inblock_l3"},
         {"children_inblock_l1", "children_inblock_l2", "children_inblock_l3"}},
        {{"plan_final_l1", "plan_final_l2", "plan_final_l3"},
         {"pool_final_l1", "pool_final_l2", "pool_final_l3"},
         {"corank_final_l1", "corank_final_l2", "corank_final_l3"},
         {"children_final_l1", "children_final_l2", "children_final_l3"}}};
    return names[fin ? 1 : 0][what][l < 2 ? l : 2];
}

// Raise a kernel's dynamic shared-memory limit once per (device, kernel) to
// the largest size asked so far, so that launches queued later (for example
// while a stream is being captured into a CUDA graph) make no attribute call.
struct SmemAttrCache {
    std::mutex mu;
    struct Entry {
        const void* f;
        int dev;
        size_t bytes;
    };
    std::vector<Entry> set;
};
inline SmemAttrCache& smem_attr_cache()
{
    static SmemAttrCache c;
    return c;
}
template <typename KF> static cudaError_t smem_attr(KF* f, size_t bytes)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    SmemAttrCache& c = smem_attr_cache();
    std::lock_guard<std::mutex> lk(c.mu);
    for (auto& x : c.set)
        if (x.f == (const void*)f && x.dev == dev) {
            if (x.bytes >= bytes) return cudaSuccess;
            e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
            if (e == cudaSuccess) x.bytes = bytes;
            return e;
        }
    e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) c.set.push_back({(const void*)f, dev, bytes});
    return e;
}

static inline int xf_of(int dtype)
{
    switch (dtype) {
    case PS_I32: case PS_I64: return 1;
    case PS_F32: case PS_F64: return 2;
    default: return 0;
    }
}

// The caller's pivot buffers of a trace, viewed as a key buffer.
template <typename K> static GBuf<K> trace_gbuf(const ps_trace* t);
template <> inline GBuf<uint32_t> trace_gbuf<uint32_t>(const ps_trace* t) { return GBuf<uint32_t>{(uint32_t*)t->pivots, INT64_MAX}; }
template <> inline GBuf<uint64_t> trace_gbuf<uint64_t>(const ps_trace* t) { return GBuf<uint64_t>{(uint64_t*)t->pivots, INT64_MAX}; }
template <> inline GBuf<Rec> trace_gbuf<Rec>(const ps_trace* t)
{
    return GBuf<Rec>{(uint64_t*)t->pivots, t->pivot_payload, INT64_MAX};
}

template <typename K, typename CF = Cfg<K>> struct Pipeline {
    using C = CF;
    using PlanK = Plan<K, CF>;
    static constexpr int TNT = C::TNT, TE = C::TE, MNT = C::MNT, ME = C::ME, PNT = C::PNT, PE = C::PE;
    static constexpr int T = TNT * TE, CAP = MNT * ME, POOL = PNT * PE;

    static size_t pool_smem(int Kr)
    {
        return STagged<K>::bytes(POOL) + 4 * (size_t)POOL + 4 * (size_t)(POOL / 2 + 1) + 4 * (size_t)(Kr + 1) + 64;
    }
    static constexpr int BE = ME / 2;  // keys per thread of the oversized-group path
    static size_t merge_smem(int Kr)
    {
        return TileBuf<K, ME>::type::bytes(CAP) + 16 * (size_t)Kr + 4 * (size_t)(Kr + 1) + 64;
    }
    static size_t big_smem(int Kr)
    {
        return TileBuf<K, BE>::type::bytes(MNT * BE) + 32 * (size_t)Kr + 4 * (size_t)(Kr + 1) + 64;
    }
    static size_t tile_smem() { return TileBuf<K, TE>::type::bytes(T) + 64; }

    // The instances' own buffers (plain keys only).
    static K* const* iptrs(const SortArgs& a)
    {
        if constexpr (sizeof(K) == 4 || sizeof(K) == 8) return (K* const*)a.inst_ptrs;
        return nullptr;
    }

    static Inst inst_of(const PlanK& pl, const SortArgs& a)
    {
        Inst in;
        in.base = a.inst_base;
        in.n = a.inst_n;
        in.count = pl.n_inst;
        in.n0 = pl.Nmax;
        return in;
    }

    template <int XF>
    static cudaError_t tile_sort(GBuf<K> src, GBuf<K> dst, const PlanK& pl, const SortArgs& a_, cudaStream_t s)
    {
        // the tile sort is the whole sort when there is one block, one
        // partition and no in-block pass
        const bool fin = pl.direct && pl.npass == 0 && !a_.keep_order_keys;
        auto f = fin ? k_tile_sort<TNT, TE, K, XF, true, C::TW> : k_tile_sort<TNT, TE, K, XF, false, C::TW>;
        cudaError_t e = smem_attr(f, tile_smem());
        if (e != cudaSuccess) return e;
        const int64_t grid = pl.n_inst * pl.n_B * pl.R0;
        ProfScope ps_("tile_sort", s);
        f<<<(unsigned)grid, TNT, tile_smem(), s>>>(src, dst, inst_of(pl, a_), pl.n_B, pl.R0, iptrs(a_));
        return cudaGetLastError();
    }

    // Multiway merge of every group of `job` from src into dst: level-0 windows,
    // sh.nlev refinement levels (sample pool, co-ranks, child windows), then
    // one CTA per final group.
    // variant: ps_merge_variant of the last level's chunk merge.
    template <int XF>
    // G0: groups of the job (default: the shape's capacity, every group).
    // own: write the output to the instances' own buffers (SortArgs::inst_ptrs).
    static cudaError_t merge(const MergeJob& job, const MergeShape& sh, GBuf<K> src, GBuf<K> dst,
                             const PlanK& pl, char* ws, cudaStream_t s, int variant = PS_MERGE_TREE,
                             int64_t G0 = -1, K* const* own = nullptr)
    {
        if (G0 < 0) G0 = sh.G[0];
        const bool fin = job.kind == 1;
        char* m = ws + pl.o_merge;
        const int Kr = sh.K;
        Level Lv[MAXLEV + 1];
        for (int l = 0; l <= sh.nlev; l++) {
            Lv[l].K = Kr;
            Lv[l].cap = sh.G[l];
            Lv[l].lo = (int64_t*)(m + sh.o_lo[l]);
            Lv[l].hi = (int64_t*)(m + sh.o_hi[l]);
            Lv[l].base = (int64_t*)(m + sh.o_base[l]);
            Lv[l].size = (int64_t*)(m + sh.o_size[l]);
            Lv[l].ng = (int64_t*)(m + sh.o_ng[l]);
        }
        cudaError_t e;
        {
            ProfScope ps_(fin ? "windows_final" : "windows_inblock", s);
            const int64_t nt = G0 * Kr;
            k_root_windows<<<(unsigned)((nt + 255) / 256), 256, 0, s>>>(job, G0, Lv[0]);
        }
        auto fp = k_pool<PNT, PE, K, PS_POOL_SPC>;
        if ((e = smem_attr(fp, pool_smem(Kr))) != cudaSuccess) return e;
        for (int l = 0; l < sh.nlev; l++) {
            int64_t* choff = (int64_t*)(m + sh.o_choff[l]);
            int* chgrp = (int*)(m + sh.o_chgrp[l]);
            Splitter<K>* spl = (Splitter<K>*)(m + sh.o_spl[l]);
            {
                ProfScope ps_(level_label(fin, 0, l), s);
                k_chunk_plan<1024><<<1, 1024, 0, s>>>(Lv[l], sh.cnom[l], sh.jcap, choff);
            }
            {
                ProfScope ps_(level_label(fin, 1, l), s);
                fp<<<(unsigned)sh.G[l], PNT, pool_smem(Kr), s>>>(Lv[l], src, choff, chgrp, spl, sh.G[l + 1],
                                                                 Lv[l + 1]);
            }
            {
                ProfScope ps_(level_label(fin, 2, l), s);
                const int64_t nt = sh.G[l + 1] * Kr;
                k_corank<K><<<(unsigned)((nt + 255) / 256), 256, 0, s>>>(Lv[l], src, spl, choff, chgrp, Lv[l + 1]);
            }
            {
                ProfScope ps_(level_label(fin, 3, l), s);
                k_child_stats<256><<<(unsigned)((sh.G[l + 1] + 7) / 8), 256, 0, s>>>(Lv[l], choff, chgrp, Lv[l + 1]);
            }
        }
        int64_t* big = (int64_t*)(m + sh.o_big);
        unsigned long long* nbig = (unsigned long long*)big;
        if ((e = cudaMemsetAsync(nbig, 0, 8, s)) != cudaSuccess) return e;
        const Level& Lf = Lv[sh.nlev];
        const int64_t gf = sh.G[sh.nlev];
        if (variant == PS_MERGE_SELECT) {
            if (own) return cudaErrorInvalidValue;  // the selection tree writes dst only
            // one thread per group, each with its own selection tree
            int KP = 1;
            while (KP < Kr) KP <<= 1;
            const size_t per = (size_t)KP * (sizeof(K) + 2 * sizeof(int64_t) + sizeof(int));
            const int tpb = (int)std::max<size_t>(1, std::min<size_t>(32, (size_t)(160 << 10) / per));
            auto fs = k_merge_select<K, XF>;
            if ((e = smem_attr(fs, (size_t)tpb * per)) != cudaSuccess) return e;
            ProfScope ps_(fin ? "merge_final" : "merge_inblock", s);
            fs<<<(unsigned)((gf + tpb - 1) / tpb), 32, (size_t)tpb * per, s>>>(Lf, src, dst, pl.N, KP, tpb);
            return cudaGetLastError();
        }
        auto fm = variant == PS_MERGE_SORT ? k_merge<MNT, ME, K, XF, false, false, true>
                  : PlanK::aligned(Kr)   ? k_merge<MNT, ME, K, XF, false, true>
                                           : k_merge<MNT, ME, K, XF, false, false>;
        if ((e = smem_attr(fm, merge_smem(Kr))) != cudaSuccess) return e;
        {
            ProfScope ps_(fin ? "merge_final" : "merge_inblock", s);
            fm<<<(unsigned)gf, MNT, merge_smem(Kr), s>>>(Lf, src, dst, pl.N, big + 1, nbig, own, job.in);
        }
        auto fb = k_merge<MNT, BE, K, XF, true, false>;
        if ((e = smem_attr(fb, big_smem(Kr))) != cudaSuccess) return e;
        {
            ProfScope ps_(fin ? "merge_big_final" : "merge_big_inblock", s);
            fb<<<(unsigned)std::min<int64_t>(gf, 2 * 152), MNT, big_smem(Kr), s>>>(Lf, src, dst, pl.N, big + 1,
                                                                                    nbig, own, job.in);
        }
        return cudaGetLastError();
    }

    template <int XF> static cudaError_t run_xf(const SortArgs& a, const PlanK& pl, char* ws)
    {
        cudaStream_t s = a.stream;
        GBuf<K> user = gbuf_user<K>(a);
        GBuf<K> wsb = gbuf_at<K>(ws + pl.o_data, pl.N);
        const GBuf<K> first = gbuf_ext<K>(a.src_keys, user);  // read by the first pass
        const GBuf<K> last = gbuf_ext<K>(a.dst_keys, user);   // written by the last pass
        const Inst in = inst_of(pl, a);
        cudaError_t e;
        // Step 1: sort each block (tiles, then in-block merge passes).  The
        // passes alternate between the caller's buffer and the workspace copy;
        // the block sort ends in the workspace, or in the caller's buffer when
        // it is the whole sort (one block, one partition).  Presorted: the
        // caller's buffer already holds the sorted blocks (order keys).
        const bool end_in_user = pl.direct;
        GBuf<K> cur = ((pl.npass % 2 == 0) != end_in_user) ? wsb : user;
        if (end_in_user && pl.npass == 0) cur = last;
        if (a.presorted) cur = user;
        else if ((e = tile_sort<XF>(first, cur, pl, a, s)) != cudaSuccess) return e;
        int64_t W = T;
        for (int p = 0; p < pl.npass && !a.presorted; p++) {
            MergeJob job{};  // in-block pass p
            job.kind = 0;
            job.K = (int)pl.F[p];
            job.in = in;
            job.n_B = pl.n_B;
            job.N = pl.N;
            job.W = W;
            const int64_t Rp = (pl.L + W - 1) / W;
            job.gpb = (Rp + pl.F[p] - 1) / pl.F[p];
            GBuf<K> nxt = same_buf(cur, wsb) ? user : wsb;
            if (p + 1 == pl.npass && end_in_user) nxt = last;
            if (p + 1 == pl.npass && end_in_user && !a.keep_order_keys) {
                if ((e = merge<XF>(job, pl.inblock[p], cur, nxt, pl, ws, s, PS_MERGE_TREE, -1, iptrs(a))) !=
                    cudaSuccess)
                    return e;
            } else if ((e = merge<0>(job, pl.inblock[p], cur, nxt, pl, ws, s)) != cudaSuccess) {
                return e;
            }
            cur = nxt;
            W *= pl.F[p];
        }
        if (pl.direct && !(a.trace && pl.n_inst == 1)) return cudaGetLastError();
        // Steps 2 and 3: pivots, split table, offsets.
        int64_t* splits = (int64_t*)(ws + pl.o_split);
        int64_t* offs = (int64_t*)(ws + pl.o_off);
        K* piv = (K*)(ws + pl.o_piv);
        int64_t* cvec = (int64_t*)(ws + pl.o_c);
        const int64_t nrows = pl.n_inst * pl.n_B;
        {
            ProfScope ps_("split_borders", s);
            k_split_borders<<<(unsigned)((nrows + 255) / 256), 256, 0, s>>>(in, pl.n_B, pl.n_P, splits);
        }
        if (pl.n_P > 1) {
            const int64_t npiv = pl.n_inst * (pl.n_P - 1);
            if (a.mode == PS_PIVOT_EXACT) {
                auto f = k_pses<512, K>;
                size_t sm = 16 * (size_t)pl.n_B + 64;
                if ((e = smem_attr(f, sm)) != cudaSuccess) return e;
                ProfScope ps_("pses", s);
                f<<<(unsigned)npiv, 512, sm, s>>>(cur, in, pl.n_B, pl.n_P, piv, cvec, splits);
            } else {
                GBuf<K> samp = gbuf_at<K>(ws + pl.o_samp, nrows * (pl.n_P - 1));
                const int64_t ns = nrows * (pl.n_P - 1);
                {
                    ProfScope ps_("psrs_samples", s);
                    k_psrs_samples<K><<<(unsigned)((ns + 255) / 256), 256, 0, s>>>(cur, samp, in, pl.n_B, pl.n_P);
                }
                auto f = k_psrs_select<512, K>;
                size_t sm = 16 * (size_t)pl.n_B + 64;
                if ((e = smem_attr(f, sm)) != cudaSuccess) return e;
                {
                    ProfScope ps_("psrs_select", s);
                    f<<<(unsigned)npiv, 512, sm, s>>>(samp, in, pl.n_B, pl.n_P, piv);
                }
                ProfScope ps_("psrs_splits", s);
                k_psrs_splits<K><<<(unsigned)((ns + 255) / 256), 256, 0, s>>>(cur, piv, in, pl.n_B, pl.n_P, splits);
            }
        }
        {
            ProfScope ps_("offsets", s);
            const int64_t no = pl.n_inst * (pl.n_P + 1);
            k_offsets<<<(unsigned)((no + 255) / 256), 256, 0, s>>>(splits, in, pl.n_B, pl.n_P, offs);
        }
        // Step 4: merge the k-th partitions of all blocks into the caller's
        // buffer (nothing to merge when the block sort was the whole sort).
        MergeJob job{};
        job.kind = 1;
        job.K = (int)pl.n_B;
        job.in = in;
        job.n_B = pl.n_B;
        job.N = pl.N;
        job.splits = splits;
        job.offsets = offs;
        job.n_P = pl.n_P;
        if (!pl.direct && !std::is_same<K, Rec>::value && a.host_out && a.copy_stream && a.out_ranges > 1 &&
            pl.n_inst == 1 && a.mode == PS_PIVOT_EXACT) {
            // partition ranges, each copied out while the next is merged
            const int64_t nr = std::min<int64_t>(a.out_ranges, pl.n_P);
            const size_t kb = GStore<K>::bytes;
            auto start = [&](int64_t k) { return (int64_t)(((unsigned __int128)k * (uint64_t)pl.N) / (uint64_t)pl.n_P); };
            for (int64_t r = 0; r < nr && e == cudaSuccess; r++) {
                const int64_t k0 = r * pl.n_P / nr, k1 = (r + 1) * pl.n_P / nr;
                job.k0 = k0;
                if ((e = merge<XF>(job, pl.fin, cur, last, pl, ws, s, a.merge_variant, k1 - k0)) != cudaSuccess) break;
                cudaEvent_t ev;
                if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) break;
                e = cudaEventRecord(ev, s);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(a.copy_stream, ev, 0);
                const int64_t o0 = start(k0), o1 = start(k1);
                if (e == cudaSuccess && o1 > o0)
                    e = cudaMemcpyAsync((char*)a.host_out + o0 * kb, (const char*)last_ptr(last) + o0 * kb,
                                        (size_t)(o1 - o0) * kb, cudaMemcpyDeviceToHost, a.copy_stream);
                cudaEventDestroy(ev);
            }
            if (e != cudaSuccess) return e;
            // the caller's stream completes after the last copy
            cudaEvent_t done;
            if ((e = cudaEventCreateWithFlags(&done, cudaEventDisableTiming)) != cudaSuccess) return e;
            e = cudaEventRecord(done, a.copy_stream);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s, done, 0);
            cudaEventDestroy(done);
            if (e != cudaSuccess) return e;
        } else if (!pl.direct && (e = merge<XF>(job, pl.fin, cur, last, pl, ws, s, a.merge_variant, -1, iptrs(a))) !=
                                     cudaSuccess) {
            return e;
        }
        // Trace (single sorts only).
        if (a.trace && pl.n_inst == 1) {
            const ps_trace* t = a.trace;
            if (t->pivots && pl.n_P > 1) {
                GBuf<K> tp = trace_buf(t);
                ProfScope ps_("trace_pivots", s);
                k_trace_pivots<K, XF><<<(unsigned)((pl.n_P - 1 + 255) / 256), 256, 0, s>>>(piv, pl.n_P - 1, tp);
            }
            if (t->c && pl.n_P > 1) {
                if (a.mode == PS_PIVOT_EXACT)
                    e = cudaMemcpyAsync(t->c, cvec, (size_t)(pl.n_P - 1) * 8, cudaMemcpyDeviceToDevice, s);
                else
                    e = cudaMemsetAsync(t->c, 0, (size_t)(pl.n_P - 1) * 8, s);
                if (e != cudaSuccess) return e;
            }
            if (t->splits) {
                e = cudaMemcpyAsync(t->splits, splits, (size_t)pl.n_B * (pl.n_P + 1) * 8, cudaMemcpyDeviceToDevice, s);
                if (e != cudaSuccess) return e;
            }
            if (t->offsets) {
                e = cudaMemcpyAsync(t->offsets, offs, (size_t)(pl.n_P + 1) * 8, cudaMemcpyDeviceToDevice, s);
                if (e != cudaSuccess) return e;
            }
        }
        return cudaGetLastError();
    }

    static GBuf<K> trace_buf(const ps_trace* t) { return trace_gbuf<K>(t); }

    static void make_plan(PlanK& pl, const SortArgs& a)
    {
        if (a.inst_base)
            pl.make(a.extent, a.n_inst, a.n_max, a.n_sum, a.n_B, a.n_P, a.mode);
        else
            pl.make(a.n, 1, a.n, a.n, a.n_B, a.n_P, a.mode);
    }

    // The short instances of a batch in one persistent launch
    // (k_batch_front): t (optional) holds instances of at most one tile,
    // sm (optional) instances of at most 1024 keys; *next is zeroed here on
    // the stream before the launch.  Both argument sets share the keys
    // buffer, the dtype and, when set, the own-buffer pointers.
    static int run_front(const SortArgs* t, const SortArgs* sm, unsigned long long* next)
    {
        if (!t && !sm) return PS_OK;
        if (!next) return PS_ERR_INVALID_ARG;
        const SortArgs& a = t ? *t : *sm;
        cudaError_t e;
        switch (xf_of(a.dtype)) {
        case 1: e = front_xf<1>(t, sm, next); break;
        case 2: e = front_xf<2>(t, sm, next); break;
        default: e = front_xf<0>(t, sm, next); break;
        }
        return e == cudaSuccess ? PS_OK : fail_cuda(e);
    }
    template <int XF> static cudaError_t front_xf(const SortArgs* t, const SortArgs* sm, unsigned long long* next)
    {
        constexpr int NT = C::TNT, E = C::TE;
        const SortArgs& a = t ? *t : *sm;
        if ((t && t->n_max > NT * E) || (sm && sm->n_max > (int64_t)SMALL_SEG)) return cudaErrorInvalidValue;
        auto f = k_batch_front<NT, E, K, XF, C::TW>;
        const size_t smb = TileBuf<K, E>::type::bytes(NT * E) + 64;
        cudaError_t e = smem_attr(f, smb);
        if (e != cudaSuccess) return e;
        auto inst_of = [](const SortArgs* x) {
            Inst in;
            in.base = x ? x->inst_base : nullptr;
            in.n = x ? x->inst_n : nullptr;
            in.count = x ? x->n_inst : 0;
            in.n0 = 0;
            return in;
        };
        const Inst ti = inst_of(t), si = inst_of(sm);
        const int64_t items = ti.count + (si.count + NT / 32 - 1) / (NT / 32);
        int dev = 0, sms = 0, per_sm = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, NT, smb);
        if (e != cudaSuccess) return e;
        const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(items, (int64_t)sms * std::max(per_sm, 1)));
        e = cudaMemsetAsync(next, 0, sizeof(*next), a.stream);
        if (e != cudaSuccess) return e;
        GBuf<K> user = gbuf_user<K>(a);
        ProfScope ps_("batch_front", a.stream);
        f<<<(unsigned)grid, NT, smb, a.stream>>>(user, ti, t ? iptrs(*t) : nullptr, si, sm ? iptrs(*sm) : nullptr,
                                                 next);
        return cudaGetLastError();
    }

    static int run(const SortArgs& a)
    {
        PlanK pl;
        make_plan(pl, a);
        char* ws = nullptr;
        int rc = ws_alloc((void**)&ws, pl.total, a.stream);
        if (rc != PS_OK) return rc;
        cudaError_t e;
        switch (xf_of(a.dtype)) {
        case 1: e = run_xf<1>(a, pl, ws); break;
        case 2: e = run_xf<2>(a, pl, ws); break;
        default: e = run_xf<0>(a, pl, ws); break;
        }
        ws_free(ws, a.stream);
        if (e != cudaSuccess) return fail_cuda(e);
        return PS_OK;
    }

    // The same pipeline on a workspace the caller provides (cap bytes at ws);
    // allocates nothing.  PS_ERR_INVALID_ARG if the plan does not fit.
    static int run_on(const SortArgs& a, char* ws, size_t cap)
    {
        PlanK pl;
        make_plan(pl, a);
        if (pl.total > cap) return PS_ERR_INVALID_ARG;
        cudaError_t e;
        switch (xf_of(a.dtype)) {
        case 1: e = run_xf<1>(a, pl, ws); break;
        case 2: e = run_xf<2>(a, pl, ws); break;
        default: e = run_xf<0>(a, pl, ws); break;
        }
        if (e != cudaSuccess) return fail_cuda(e);
        return PS_OK;
    }

    // Workspace of one (possibly multi-instance) sort as described by a.
    static size_t ws_bytes_for(const SortArgs& a)
    {
        PlanK pl;
        make_plan(pl, a);
        return pl.total;
    }

    static size_t ws_bytes(int64_t n, int64_t nb, int64_t np)
    {
        PlanK pl;
        pl.make(n, 1, n, n, nb, np, PS_PIVOT_REGULAR);
        return pl.total;
    }
};

}  // namespace ps

// psort_pipeline.cuh -- host orchestration of one sort for one key family:
// workspace plan, kernel launches of the four steps, trace output.
#pragma once

#include <algorithm>

#include "psort_internal.h"
#include "psort_kernels.cuh"

namespace ps {

// Threads per CTA (NT) and keys per thread (E) of the tile sort and merge
// kernels; PNT*PE is the sample-pool size.
template <typename K> struct Cfg;
template <> struct Cfg<uint32_t> {
    static constexpr int NT = 512, E = 16, PNT = 512, PE = 16;
};
template <> struct Cfg<uint64_t> {
    static constexpr int NT = 512, E = 16, PNT = 512, PE = 16;
};
template <> struct Cfg<Rec> {
    static constexpr int NT = 512, E = 8, PNT = 512, PE = 8;
};

constexpr int64_t FMAX = 512;  // largest fan-in of one in-block merge pass

template <typename K> struct GStore {
    static constexpr size_t bytes = sizeof(K);
};
template <> struct GStore<Rec> {
    static constexpr size_t bytes = 12;  // uint64 key + uint32 payload, structure of arrays
};

static inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Everything the launches need to know about one sort's shape.
template <typename K> struct Plan {
    static constexpr int T = Cfg<K>::NT * Cfg<K>::E;  // tile = merge chunk capacity
    static constexpr int POOL = Cfg<K>::PNT * Cfg<K>::PE;
    int64_t N, n_B, n_P, L, R0;
    int npass;
    int64_t F[16];
    int64_t G_max, CH_max, CR_max;
    // workspace byte offsets
    size_t o_data, o_split, o_off, o_piv, o_c, o_samp, o_choff, o_chgrp, o_spl, o_cr, total;

    static int64_t cnom() { return T / 2; }
    static int64_t jcap(int64_t K_) { return std::max<int64_t>(1, (POOL / 2 - K_) / 2); }
    int64_t ch_ub(int64_t G) const { return N / cnom() + G + 1; }

    void make(int64_t n, int64_t nb, int64_t np)
    {
        N = n;
        n_B = nb;
        n_P = np;
        L = (N + n_B - 1) / n_B;
        R0 = (L + T - 1) / T;
        npass = 0;
        for (int64_t x = R0; x > 1; x = (x + FMAX - 1) / FMAX) npass++;
        int64_t R = R0;
        G_max = n_P;
        CH_max = ch_ub(n_P);
        CR_max = CH_max * n_B;
        int64_t W = T;
        for (int p = 0; p < npass; p++) {
            int rem = npass - p;
            int64_t f = 2;  // smallest fan-in with f^rem >= R
            while (true) {
                long double q = 1;
                for (int i = 0; i < rem; i++) q *= (long double)f;
                if (q >= (long double)R || f >= FMAX) break;
                f++;
            }
            F[p] = std::min<int64_t>(f, R);
            int64_t Rp = (L + W - 1) / W;
            int64_t gpb = (Rp + F[p] - 1) / F[p];
            int64_t G = n_B * gpb;
            G_max = std::max(G_max, G);
            CH_max = std::max(CH_max, ch_ub(G));
            CR_max = std::max(CR_max, ch_ub(G) * F[p]);
            R = (R + F[p] - 1) / F[p];
            W *= F[p];
        }
        size_t o = 0;
        o_data = o;
        o += align256((size_t)N * GStore<K>::bytes + 256);
        o_split = o;
        o += align256((size_t)n_B * (n_P + 1) * 8);
        o_off = o;
        o += align256((size_t)(n_P + 1) * 8);
        o_piv = o;
        o += align256((size_t)n_P * sizeof(K));
        o_c = o;
        o += align256((size_t)n_P * 8);
        o_samp = o;
        o += align256((size_t)n_B * std::max<int64_t>(n_P - 1, 1) * GStore<K>::bytes + 256);
        o_choff = o;
        o += align256((size_t)(G_max + 1) * 8);
        o_chgrp = o;
        o += align256((size_t)CH_max * 4);
        o_spl = o;
        o += align256((size_t)CH_max * sizeof(Splitter<K>));
        o_cr = o;
        o += align256((size_t)CR_max * 8);
        total = o;
    }
};

template <typename K> static GBuf<K> gbuf_at(char* base, int64_t n);
template <> inline GBuf<uint32_t> gbuf_at<uint32_t>(char* base, int64_t) { return GBuf<uint32_t>{(uint32_t*)base}; }
template <> inline GBuf<uint64_t> gbuf_at<uint64_t>(char* base, int64_t) { return GBuf<uint64_t>{(uint64_t*)base}; }
template <> inline GBuf<Rec> gbuf_at<Rec>(char* base, int64_t n)
{
    return GBuf<Rec>{(uint64_t*)base, (uint32_t*)(base + align256((size_t)n * 8))};
}

template <typename K> static GBuf<K> gbuf_user(const SortArgs& a);
template <> inline GBuf<uint32_t> gbuf_user<uint32_t>(const SortArgs& a) { return GBuf<uint32_t>{(uint32_t*)a.keys}; }
template <> inline GBuf<uint64_t> gbuf_user<uint64_t>(const SortArgs& a) { return GBuf<uint64_t>{(uint64_t*)a.keys}; }
template <> inline GBuf<Rec> gbuf_user<Rec>(const SortArgs& a) { return GBuf<Rec>{(uint64_t*)a.keys, a.payload}; }

template <typename K> static bool same_buf(const GBuf<K>& x, const GBuf<K>& y);
template <> inline bool same_buf<uint32_t>(const GBuf<uint32_t>& x, const GBuf<uint32_t>& y) { return x.p == y.p; }
template <> inline bool same_buf<uint64_t>(const GBuf<uint64_t>& x, const GBuf<uint64_t>& y) { return x.p == y.p; }
template <> inline bool same_buf<Rec>(const GBuf<Rec>& x, const GBuf<Rec>& y) { return x.k == y.k; }

template <typename KF> static cudaError_t smem_attr(KF* f, size_t bytes)
{
    return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

static inline int xf_of(int dtype)
{
    switch (dtype) {
    case PS_I32: case PS_I64: return 1;
    case PS_F32: case PS_F64: return 2;
    default: return 0;
    }
}

template <typename K> struct Pipeline {
    using C = Cfg<K>;
    static constexpr int NT = C::NT, E = C::E, PNT = C::PNT, PE = C::PE;
    static constexpr int T = NT * E, POOL = PNT * PE;

    static size_t pool_smem(int Kr) { return STagged<K>::bytes(POOL) + 8 * (size_t)Kr + 4 * (size_t)(Kr + 1) + 64; }
    static size_t merge_smem(int Kr) { return SBuf<K>::bytes(T) + 24 * (size_t)Kr + 4 * (size_t)(Kr + 1) + 64; }
    static size_t tile_smem() { return SBuf<K>::bytes(T) + 4 * (size_t)(NT + 1) + 64; }

    template <int XF>
    static cudaError_t tile_sort(GBuf<K> src, GBuf<K> dst, const Plan<K>& pl, cudaStream_t s)
    {
        auto f = k_tile_sort<NT, E, K, XF>;
        cudaError_t e = smem_attr(f, tile_smem());
        if (e != cudaSuccess) return e;
        const int64_t grid = pl.n_B * pl.R0;
        ProfScope ps_("tile_sort", s);
        f<<<(unsigned)grid, NT, tile_smem(), s>>>(src, dst, pl.N, pl.L, pl.R0);
        return cudaGetLastError();
    }

    // Multiway merge of every group of `job` from src into dst.
    template <int XF>
    static cudaError_t merge(const MergeJob& job, int64_t G, GBuf<K> src, GBuf<K> dst, const Plan<K>& pl,
                             char* ws, cudaStream_t s)
    {
        const bool fin = job.kind == 1;
        int64_t* choff = (int64_t*)(ws + pl.o_choff);
        int* chgrp = (int*)(ws + pl.o_chgrp);
        Splitter<K>* spl = (Splitter<K>*)(ws + pl.o_spl);
        int64_t* cr = (int64_t*)(ws + pl.o_cr);
        const int64_t* nch = choff + G;
        const int64_t chub = pl.ch_ub(G);
        {
            ProfScope ps_(fin ? "chunk_plan_final" : "chunk_plan_inblock", s);
            k_chunk_plan<1024><<<1, 1024, 0, s>>>(job, G, Plan<K>::cnom(), Plan<K>::jcap(job.K), choff);
        }
        auto fp = k_pool<PNT, PE, K>;
        cudaError_t e = smem_attr(fp, pool_smem(job.K));
        if (e != cudaSuccess) return e;
        {
            ProfScope ps_(fin ? "pool_final" : "pool_inblock", s);
            fp<<<(unsigned)G, PNT, pool_smem(job.K), s>>>(job, src, choff, chgrp, spl);
        }
        const int64_t nthr = chub * job.K;
        {
            ProfScope ps_(fin ? "corank_final" : "corank_inblock", s);
            k_corank<K><<<(unsigned)((nthr + 255) / 256), 256, 0, s>>>(job, src, spl, choff, chgrp, nch, cr);
        }
        auto fm = k_merge<NT, E, K, XF>;
        e = smem_attr(fm, merge_smem(job.K));
        if (e != cudaSuccess) return e;
        {
            ProfScope ps_(fin ? "merge_final" : "merge_inblock", s);
            fm<<<(unsigned)chub, NT, merge_smem(job.K), s>>>(job, src, dst, cr, choff, chgrp, nch);
        }
        return cudaGetLastError();
    }

    template <int XF> static cudaError_t run_xf(const SortArgs& a, const Plan<K>& pl, char* ws)
    {
        cudaStream_t s = a.stream;
        GBuf<K> user = gbuf_user<K>(a);
        GBuf<K> wsb = gbuf_at<K>(ws + pl.o_data, pl.N);
        cudaError_t e;
        // Step 1: sort each block (tiles, then in-block merge passes).
        GBuf<K> cur = (pl.npass % 2 == 0) ? wsb : user;
        if ((e = tile_sort<XF>(user, cur, pl, s)) != cudaSuccess) return e;
        int64_t W = T;
        for (int p = 0; p < pl.npass; p++) {
            MergeJob job{};
            job.kind = 0;
            job.K = (int)pl.F[p];
            job.N = pl.N;
            job.L = pl.L;
            job.W = W;
            int64_t Rp = (pl.L + W - 1) / W;
            job.gpb = (Rp + pl.F[p] - 1) / pl.F[p];
            GBuf<K> nxt = same_buf(cur, wsb) ? user : wsb;
            if ((e = merge<0>(job, pl.n_B * job.gpb, cur, nxt, pl, ws, s)) != cudaSuccess) return e;
            cur = nxt;
            W *= pl.F[p];
        }
        // Steps 2 and 3: pivots, split table, offsets.
        int64_t* splits = (int64_t*)(ws + pl.o_split);
        int64_t* offs = (int64_t*)(ws + pl.o_off);
        K* piv = (K*)(ws + pl.o_piv);
        int64_t* cvec = (int64_t*)(ws + pl.o_c);
        {
            ProfScope ps_("split_borders", s);
            k_split_borders<<<(unsigned)((pl.n_B + 255) / 256), 256, 0, s>>>(pl.N, pl.L, pl.n_B, pl.n_P, splits);
        }
        if (pl.n_P > 1) {
            if (a.mode == PS_PIVOT_EXACT) {
                auto f = k_pses<512, K>;
                size_t sm = 16 * (size_t)pl.n_B + 64;
                if ((e = smem_attr(f, sm)) != cudaSuccess) return e;
                ProfScope ps_("pses", s);
                f<<<(unsigned)(pl.n_P - 1), 512, sm, s>>>(cur, pl.N, pl.L, pl.n_B, pl.n_P, piv, cvec, splits);
            } else {
                const int64_t nb1 = (pl.N + pl.L - 1) / pl.L;
                GBuf<K> samp = gbuf_at<K>(ws + pl.o_samp, pl.n_B * (pl.n_P - 1));
                const int64_t ns = nb1 * (pl.n_P - 1);
                {
                    ProfScope ps_("psrs_samples", s);
                    k_psrs_samples<K><<<(unsigned)((ns + 255) / 256), 256, 0, s>>>(cur, samp, pl.N, pl.L, nb1, pl.n_P);
                }
                auto f = k_psrs_select<512, K>;
                size_t sm = 16 * (size_t)nb1 + 64;
                if ((e = smem_attr(f, sm)) != cudaSuccess) return e;
                {
                    ProfScope ps_("psrs_select", s);
                    f<<<(unsigned)(pl.n_P - 1), 512, sm, s>>>(samp, nb1, pl.n_P, piv);
                }
                const int64_t nt = pl.n_B * (pl.n_P - 1);
                ProfScope ps_("psrs_splits", s);
                k_psrs_splits<K><<<(unsigned)((nt + 255) / 256), 256, 0, s>>>(cur, piv, pl.N, pl.L, pl.n_B,
                                                                             pl.n_P, splits);
            }
        }
        {
            ProfScope ps_("offsets", s);
            k_offsets<<<(unsigned)((pl.n_P + 1 + 255) / 256), 256, 0, s>>>(splits, pl.n_B, pl.n_P, offs);
        }
        // Step 4: merge the k-th partitions of all blocks into the caller's buffer.
        MergeJob job{};
        job.kind = 1;
        job.K = (int)pl.n_B;
        job.N = pl.N;
        job.L = pl.L;
        job.splits = splits;
        job.offsets = offs;
        job.n_P = pl.n_P;
        if ((e = merge<XF>(job, pl.n_P, cur, user, pl, ws, s)) != cudaSuccess) return e;
        // Trace.
        if (a.trace) {
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

    static GBuf<K> trace_buf(const ps_trace* t);

    static int run(const SortArgs& a)
    {
        Plan<K> pl;
        pl.make(a.n, a.n_B, a.n_P);
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

    static size_t ws_bytes(int64_t n, int64_t nb, int64_t np)
    {
        Plan<K> pl;
        pl.make(n, nb, np);
        return pl.total;
    }
};

template <> inline GBuf<uint32_t> Pipeline<uint32_t>::trace_buf(const ps_trace* t) { return GBuf<uint32_t>{(uint32_t*)t->pivots}; }
template <> inline GBuf<uint64_t> Pipeline<uint64_t>::trace_buf(const ps_trace* t) { return GBuf<uint64_t>{(uint64_t*)t->pivots}; }
template <> inline GBuf<Rec> Pipeline<Rec>::trace_buf(const ps_trace* t)
{
    return GBuf<Rec>{(uint64_t*)t->pivots, t->pivot_payload};
}

}  // namespace ps

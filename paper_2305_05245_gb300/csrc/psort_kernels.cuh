// psort_kernels.cuh -- device code of the GB300 parallel samplesort.
//
// Four steps of Tokuue & Ishiyama (arXiv 2305.05245), Sec. 2, mapped to
// kernels:
//   step 1 (sort each block)   k_tile_sort: tiles of NT*E keys sorted in shared
//                              memory (register sorting network + merge-path
//                              levels); blocks longer than a tile are finished
//                              by in-block multiway merge passes (merge job 0).
//   step 2 (pivots)            k_psrs_samples + k_psrs_select (regular
//                              sampling, Sec. 2.3) or k_pses (exact splitting,
//                              Eq. 1 and Eq. 2, value bisection with per-block
//                              binary-search counts as Sec. 2.3 describes).
//   step 3 (partitioning)      k_psrs_splits / k_pses (split table), then
//                              k_offsets (O_k = sum_b s[b][k], Sec. 2).
//   step 4 (multiway merge)    merge job 1: each partition's pieces are cut
//                              into chunks at splitters taken from a sorted
//                              sample pool (k_pool, k_corank) and every chunk
//                              is merged in shared memory (k_merge).
// Keys travel as order keys kappa (unsigned integers whose order is the sort
// order); the transform is fused into the first load and the last store.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

// Registers a record (uint64 key + uint32 payload) counts for when a data
// kernel's CTAs per SM are chosen (data_ctas below).
#ifndef PS_REC_REGW
#define PS_REC_REGW 3
#endif

namespace ps {

// ----------------------------------------------------------- checked builds
// With -DPS_CHECKED every global and shared access of the sort validates its
// index; the first violation (site, index, bound, CTA) is recorded in ps_viol
// and the access is skipped instead of performed.  Without the flag the
// checks compile to nothing.
#ifdef PS_CHECKED
static __device__ unsigned long long ps_viol[4];
static __device__ __noinline__ void ps_violation(int site, long long idx, long long bound)
{
    if (atomicCAS(&ps_viol[0], 0ull, (unsigned long long)site) == 0ull) {
        ps_viol[1] = (unsigned long long)idx;
        ps_viol[2] = (unsigned long long)bound;
        ps_viol[3] = blockIdx.x;
    }
}
#define PS_IN(i, n, site) (((long long)(i) >= 0 && (long long)(i) < (long long)(n)) ? true : (ps::ps_violation((site), (long long)(i), (long long)(n)), false))
#else
#define PS_IN(i, n, site) true
#endif

// ---------------------------------------------------------------- key types

// A record: 64-bit key and 32-bit payload, ordered by (key, payload).
struct Rec {
    uint64_t k;
    uint32_t p;
};

__device__ __forceinline__ bool key_lt(uint32_t a, uint32_t b) { return a < b; }
__device__ __forceinline__ bool key_lt(uint64_t a, uint64_t b) { return a < b; }
__device__ __forceinline__ bool key_lt(const Rec& a, const Rec& b)
{
    return a.k < b.k || (a.k == b.k && a.p < b.p);
}

// Traits: the value domain of each key type as an unsigned integer U, used
// by the value bisection of exact splitting.
template <typename K> struct KT;
template <> struct KT<uint32_t> {
    using U = uint32_t;
    __device__ static U to_u(uint32_t k) { return k; }
    __device__ static uint32_t from_u(U u) { return u; }
    __device__ static U umax() { return 0xFFFFFFFFu; }
    __device__ static uint32_t maxkey() { return 0xFFFFFFFFu; }
};
template <> struct KT<uint64_t> {
    using U = uint64_t;
    __device__ static U to_u(uint64_t k) { return k; }
    __device__ static uint64_t from_u(U u) { return u; }
    __device__ static U umax() { return ~0ull; }
    __device__ static uint64_t maxkey() { return ~0ull; }
};
template <> struct KT<Rec> {
    using U = unsigned __int128;
    __device__ static U to_u(const Rec& r) { return ((U)r.k << 32) | (U)r.p; }
    __device__ static Rec from_u(U u) { return Rec{(uint64_t)(u >> 32), (uint32_t)u}; }
    __device__ static U umax() { return (((U)1) << 96) - 1; }
    __device__ static Rec maxkey() { return Rec{~0ull, 0xFFFFFFFFu}; }
};

// ------------------------------------------------------- order-key transform
// XF = 0: unsigned (identity), 1: two's complement (flip the sign bit),
// 2: IEEE float (totalOrder: negative values inverted, others get the sign bit).
template <int XF> __device__ __forceinline__ uint32_t kappa(uint32_t x)
{
    if (XF == 1) return x ^ 0x80000000u;
    if (XF == 2) return (x & 0x80000000u) ? ~x : (x | 0x80000000u);
    return x;
}
template <int XF> __device__ __forceinline__ uint32_t kappa_inv(uint32_t k)
{
    if (XF == 1) return k ^ 0x80000000u;
    if (XF == 2) return (k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k;
    return k;
}
template <int XF> __device__ __forceinline__ uint64_t kappa(uint64_t x)
{
    if (XF == 1) return x ^ 0x8000000000000000ull;
    if (XF == 2) return (x & 0x8000000000000000ull) ? ~x : (x | 0x8000000000000000ull);
    return x;
}
template <int XF> __device__ __forceinline__ uint64_t kappa_inv(uint64_t k)
{
    if (XF == 1) return k ^ 0x8000000000000000ull;
    if (XF == 2) return (k & 0x8000000000000000ull) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;
    return k;
}

template <int XF> __device__ __forceinline__ uint32_t xform(uint32_t x) { return kappa<XF>(x); }
template <int XF> __device__ __forceinline__ uint64_t xform(uint64_t x) { return kappa<XF>(x); }

// ------------------------------------------------------------ global buffers
template <typename K> struct GBuf;
template <> struct GBuf<uint32_t> {
    uint32_t* p;
    int64_t n;  // element count (checked builds only)
    __device__ uint32_t ld(int64_t i) const { return PS_IN(i, n, 1) ? p[i] : 0u; }
    __device__ void st(int64_t i, uint32_t v) const { if (PS_IN(i, n, 2)) p[i] = v; }
    template <int XF> __device__ uint32_t ldx(int64_t i) const { return kappa<XF>(ld(i)); }
    template <int XF> __device__ void stx(int64_t i, uint32_t v) const { st(i, kappa_inv<XF>(v)); }
};
template <> struct GBuf<uint64_t> {
    uint64_t* p;
    int64_t n;
    __device__ uint64_t ld(int64_t i) const { return PS_IN(i, n, 1) ? p[i] : 0ull; }
    __device__ void st(int64_t i, uint64_t v) const { if (PS_IN(i, n, 2)) p[i] = v; }
    template <int XF> __device__ uint64_t ldx(int64_t i) const { return kappa<XF>(ld(i)); }
    template <int XF> __device__ void stx(int64_t i, uint64_t v) const { st(i, kappa_inv<XF>(v)); }
};
template <> struct GBuf<Rec> {
    uint64_t* k;
    uint32_t* p;
    int64_t n;
    __device__ Rec ld(int64_t i) const { return PS_IN(i, n, 1) ? Rec{k[i], p[i]} : Rec{0ull, 0u}; }
    __device__ void st(int64_t i, const Rec& v) const
    {
        if (PS_IN(i, n, 2)) {
            k[i] = v.k;
            p[i] = v.p;
        }
    }
    template <int XF> __device__ Rec ldx(int64_t i) const { return ld(i); }
    template <int XF> __device__ void stx(int64_t i, const Rec& v) const { st(i, v); }
};

template <int XF> __device__ __forceinline__ Rec xform(const Rec& x) { return x; }

// ---------------------------------------------- shared-memory buffers (padded)
// One pad slot after every W elements, so that thread t reading or writing
// its E consecutive elements (blocked layout) hits distinct banks: W = 32 for
// 4-byte keys; for 8-byte keys W = 16 when E <= 16 and W = 32 when E = 32
// (a thread's 32 keys then span two 128-byte rows; with W = 16 threads t and
// t + 8 of a half-warp would share a bank).
template <typename K> struct PadOf;
template <> struct PadOf<uint32_t> { static constexpr int v = 32; };
template <> struct PadOf<uint64_t> { static constexpr int v = 16; };
template <> struct PadOf<Rec> { static constexpr int v = 16; };
template <typename K, int E> struct TilePad {
    static constexpr int v = (sizeof(K) == 8 && E >= 32) ? 32 : PadOf<K>::v;
};

template <typename K, int W = PadOf<K>::v> struct SBuf;
constexpr int log2c(int w) { return w <= 1 ? 0 : 1 + log2c(w / 2); }
template <int W> struct SBuf<uint32_t, W> {
    static_assert((W & (W - 1)) == 0, "the pad period is a power of two");
    uint32_t* a;
    int cap;  // physical slots (checked builds only)
    __device__ __forceinline__ static int at(int i) { return i + (i >> log2c(W)); }
    __device__ __forceinline__ uint32_t ld(int i) const { return PS_IN(at(i), cap, 4) ? a[at(i)] : 0u; }
    __device__ __forceinline__ void st(int i, uint32_t v) const { if (PS_IN(at(i), cap, 5)) a[at(i)] = v; }
    static __host__ __device__ size_t bytes(int n) { return (((size_t)n + n / W + 1) * 4 + 15) & ~(size_t)15; }
    static __device__ SBuf carve(char*& sp, int n)
    {
        SBuf b{(uint32_t*)sp, n + n / W + 1};
        sp += bytes(n);
        return b;
    }
};
template <int W> struct SBuf<uint64_t, W> {
    static_assert((W & (W - 1)) == 0, "the pad period is a power of two");
    uint64_t* a;
    int cap;
    __device__ __forceinline__ static int at(int i) { return i + (i >> log2c(W)); }
    __device__ __forceinline__ uint64_t ld(int i) const { return PS_IN(at(i), cap, 4) ? a[at(i)] : 0ull; }
    __device__ __forceinline__ void st(int i, uint64_t v) const { if (PS_IN(at(i), cap, 5)) a[at(i)] = v; }
    static __host__ __device__ size_t bytes(int n) { return (((size_t)n + n / W + 1) * 8 + 15) & ~(size_t)15; }
    static __device__ SBuf carve(char*& sp, int n)
    {
        SBuf b{(uint64_t*)sp, n + n / W + 1};
        sp += bytes(n);
        return b;
    }
};
template <int W> struct SBuf<Rec, W> {
    SBuf<uint64_t, W> k;
    SBuf<uint32_t> p;
    __device__ __forceinline__ Rec ld(int i) const { return Rec{k.ld(i), p.ld(i)}; }
    __device__ __forceinline__ void st(int i, const Rec& v) const { k.st(i, v.k); p.st(i, v.p); }
    static __host__ __device__ size_t bytes(int n) { return SBuf<uint64_t, W>::bytes(n) + SBuf<uint32_t>::bytes(n); }
    static __device__ SBuf carve(char*& sp, int n)
    {
        SBuf b;
        b.k = SBuf<uint64_t, W>::carve(sp, n);
        b.p = SBuf<uint32_t>::carve(sp, n);
        return b;
    }
};

// Shared-memory buffer of a kernel that gives each thread E keys.
template <typename K, int E> struct TileBuf {
    using type = SBuf<K, TilePad<K, E>::v>;
};

// ------------------------------------------- asynchronous global->shared copies
// cp.async (Ampere-and-later LDGSTS): each thread queues element copies
// without staging them in registers, so a CTA keeps many loads in flight.
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\ncp.async.wait_all;\n" ::: "memory");
}
template <int W>
__device__ __forceinline__ void cp_elem(const SBuf<uint32_t, W>& s, int i, const GBuf<uint32_t>& g, int64_t j)
{
    if (PS_IN(s.at(i), s.cap, 6) && PS_IN(j, g.n, 3)) cp_async4(s.a + s.at(i), g.p + j);
}
template <int W>
__device__ __forceinline__ void cp_elem(const SBuf<uint64_t, W>& s, int i, const GBuf<uint64_t>& g, int64_t j)
{
    if (PS_IN(s.at(i), s.cap, 6) && PS_IN(j, g.n, 3)) cp_async8(s.a + s.at(i), g.p + j);
}
template <int W>
__device__ __forceinline__ void cp_elem(const SBuf<Rec, W>& s, int i, const GBuf<Rec>& g, int64_t j)
{
    if (PS_IN(s.k.at(i), s.k.cap, 6) && PS_IN(j, g.n, 3)) {
        cp_async8(s.k.a + s.k.at(i), g.k + j);
        cp_async4(s.p.a + s.p.at(i), g.p + j);
    }
}

// Storage views used by the merge routine: plain keys, or keys carrying a
// 64-bit tag (run index and position of a pool sample).  Comparison is on
// the key only; the merge is stable, so ties keep piece order.
template <typename K, int W = PadOf<K>::v> struct SKeys {
    using V = K;
    SBuf<K, W> b;
    __device__ __forceinline__ V ld(int i) const { return b.ld(i); }
    __device__ __forceinline__ void st(int i, const V& v) const { b.st(i, v); }
    __device__ __forceinline__ static bool lt(const V& x, const V& y) { return key_lt(x, y); }
};
template <typename B> struct ViewOf;
template <typename K, int W> struct ViewOf<SBuf<K, W>> {
    using type = SKeys<K, W>;
};

// A thread's E blocked keys from and to shared memory (positions p .. p+E-1).
template <int E, typename B, typename V>
__device__ __forceinline__ void load_block(const B& b, int p, V (&r)[E])
{
#pragma unroll
    for (int j = 0; j < E; j++) r[j] = b.ld(p + j);
}
template <int E, typename S>
__device__ __forceinline__ void store_block(const S& s, int p, const typename S::V (&out)[E])
{
#pragma unroll
    for (int i = 0; i < E; i++) s.st(p + i, out[i]);
}

template <typename K> struct Tagged {
    K key;
    uint64_t tag;
};
template <typename K> struct STagged {
    using V = Tagged<K>;
    SBuf<K> kb;
    SBuf<uint64_t> tb;
    __device__ __forceinline__ V ld(int i) const { return V{kb.ld(i), tb.ld(i)}; }
    __device__ __forceinline__ void st(int i, const V& v) const { kb.st(i, v.key); tb.st(i, v.tag); }
    __device__ __forceinline__ static bool lt(const V& x, const V& y) { return key_lt(x.key, y.key); }
    static __host__ __device__ size_t bytes(int n) { return SBuf<K>::bytes(n) + SBuf<uint64_t>::bytes(n); }
};

// ------------------------------------------------------- block-wide helpers
template <int NT> __device__ int64_t block_sum(int64_t v)
{
    __shared__ int64_t red[NT / 32];
    __shared__ int64_t total;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        int64_t w = threadIdx.x < NT / 32 ? red[threadIdx.x] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xFFFFFFFFu, w, o);
        if (threadIdx.x == 0) total = w;
    }
    __syncthreads();
    int64_t t = total;
    __syncthreads();
    return t;
}

// Exclusive scan of one int64 per thread in thread order; returns this
// thread's exclusive prefix and writes the block total to *tot.
template <int NT> __device__ int64_t block_exscan(int64_t v, int64_t* tot)
{
    __shared__ int64_t wsum[NT / 32];
    __shared__ int64_t total;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int64_t w = lane < NT / 32 ? wsum[lane] : 0;
        int64_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xFFFFFFFFu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < NT / 32) wsum[lane] = wi - w;
        if (lane == 31) total = wi;
    }
    __syncthreads();
    int64_t r = wsum[warp] + x - v;
    *tot = total;
    __syncthreads();
    return r;
}

// ------------------------------------------------- register sorting network
// Batcher's odd-even merge sort (Knuth, TAOCP vol. 3, 5.3.4) on E register
// values, E a power of two; every index is a compile-time constant.
template <typename K> __device__ __forceinline__ void cas(K& a, K& b)
{
    bool s = key_lt(b, a);
    K lo = s ? b : a;
    K hi = s ? a : b;
    a = lo;
    b = hi;
}
// Odd-even merge of the N elements starting at LO taken with stride R: merge
// the even and the odd subsequences recursively, then compare neighbours.
template <int LO, int N, int R> struct OddEvenMerge {
    template <typename K, int E> __device__ __forceinline__ static void run(K (&a)[E])
    {
        constexpr int M = R * 2;
        if constexpr (M < N) {
            OddEvenMerge<LO, N, M>::run(a);
            OddEvenMerge<LO + R, N, M>::run(a);
#pragma unroll
            for (int i = LO + R; i + R < LO + N; i += M) cas(a[i], a[i + R]);
        } else {
            cas(a[LO], a[LO + R]);
        }
    }
};
template <int LO, int N> struct OddEvenSort {
    template <typename K, int E> __device__ __forceinline__ static void run(K (&a)[E])
    {
        if constexpr (N > 1) {
            OddEvenSort<LO, N / 2>::run(a);
            OddEvenSort<LO + N / 2, N / 2>::run(a);
            OddEvenMerge<LO, N, 1>::run(a);
        }
    }
};
template <int E, typename K> __device__ __forceinline__ void reg_sort(K (&r)[E])
{
    static_assert((E & (E - 1)) == 0, "E must be a power of two");
    OddEvenSort<0, E>::run(r);
}

// ------------------------------------------------ warp-shuffle merge levels
// Exchange of a key with the lane whose index differs by the bits of m.
__device__ __forceinline__ uint32_t shfl_key(uint32_t v, int m) { return __shfl_xor_sync(0xFFFFFFFFu, v, m); }
__device__ __forceinline__ uint64_t shfl_key(uint64_t v, int m)
{
    const uint32_t lo = __shfl_xor_sync(0xFFFFFFFFu, (uint32_t)v, m);
    const uint32_t hi = __shfl_xor_sync(0xFFFFFFFFu, (uint32_t)(v >> 32), m);
    return ((uint64_t)hi << 32) | lo;
}
__device__ __forceinline__ Rec shfl_key(const Rec& v, int m) { return Rec{shfl_key(v.k, m), shfl_key(v.p, m)}; }
// The lower lane of a compare pair keeps the smaller key, the upper lane the
// larger one (equal keys are identical bit patterns, so either may stay).
template <typename K> __device__ __forceinline__ K keep(const K& mine, const K& other, bool upper)
{
    return (key_lt(other, mine) != upper) ? other : mine;
}
// Each lane holds a sorted run of E keys (blocked: lane l holds positions
// l*E .. l*E+E-1 of its warp's 32*E keys).  LEV bitonic merge levels double
// the sorted runs LEV times without shared memory (Batcher's bitonic merge,
// Knuth TAOCP vol. 3, 5.3.4, ex. 10): at level s, units of U = 2^(s+1)
// lanes hold two sorted runs; the first stage compares position i of the
// unit with position 2m-1-i (m = half the unit: lanes l and l^(U-1), registers
// j and E-1-j) and leaves two bitonic halves, every key of the lower one no
// larger than any of the upper one; half-cleaners at lane distances U/4 .. 1
// (shuffles) and register distances E/2 .. 1 (in-thread) then sort each
// half.  Every index is a compile-time constant or a lane bit.
template <int E, int LEV, typename K>
__device__ __forceinline__ void warp_merge_levels(K (&r)[E])
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int s = 0; s < LEV; s++) {
        const int U = 2 << s;
        const bool hi_run = (lane & (U >> 1)) != 0;
#pragma unroll
        for (int j = 0; j < E / 2; j++) {
            const K pa = shfl_key(r[E - 1 - j], U - 1);  // partner's E-1-j faces my j
            const K pb = shfl_key(r[j], U - 1);          // partner's j faces my E-1-j
            r[j] = keep(r[j], pa, hi_run);
            r[E - 1 - j] = keep(r[E - 1 - j], pb, hi_run);
        }
#pragma unroll
        for (int d = U >> 2; d >= 1; d >>= 1) {
            const bool up = (lane & d) != 0;
#pragma unroll
            for (int j = 0; j < E; j++) r[j] = keep(r[j], shfl_key(r[j], d), up);
        }
#pragma unroll
        for (int d = E / 2; d >= 1; d >>= 1)
#pragma unroll
            for (int j = 0; j < E; j++)
                if ((j & d) == 0) cas(r[j], r[j + d]);
    }
}

// -------------------------------------------- shared-memory multiway merge
// Serial merge of E outputs from the heads A[ai..aend) and B[bi..bend) of one
// merge unit (stable: A wins ties).  Reads one element past an exhausted
// side, which the buffers' spare slot makes safe.  STOP guards the last
// partial thread (cnt < E) of a chunk.
template <int E, bool STOP, typename S>
__device__ __forceinline__ void serial_merge(const S& s, int ai, int aend, int bi, int bend, int cnt,
                                             typename S::V (&out)[E])
{
    using V = typename S::V;
    V a = s.ld(ai), b = s.ld(bi);
#pragma unroll
    for (int i = 0; i < E; i++) {
        if (!STOP || i < cnt) {
            const bool p = (bi >= bend) || ((ai < aend) && !S::lt(b, a));
            out[i] = p ? a : b;
            // advance the side that was taken (predicated loads, no selects)
            if (p) a = s.ld(++ai);
            else b = s.ld(++bi);
        }
    }
}

// Merge-path split of diagonal d of the unit A = [us, um), B = [um, ue):
// the number of A elements among the unit's first d outputs.
template <typename S>
__device__ __forceinline__ int merge_path(const S& s, int us, int um, int ue, int d)
{
    int a0 = d - (ue - um) > 0 ? d - (ue - um) : 0;
    int a1 = d < um - us ? d : um - us;
    while (a0 < a1) {
        const int mid = (a0 + a1) >> 1;
        if (!S::lt(s.ld(um + d - 1 - mid), s.ld(us + mid))) a0 = mid + 1;
        else a1 = mid;
    }
    return a0;
}

// Tile levels: NT*E elements in pieces of E that double each level (units of
// U = 2, 4, ... pieces' worth, all powers of two); every thread owns exactly E
// outputs that never straddle a unit.
// The power-of-two levels keep every unit in bitonic order: its first half
// A = [us, um) ascending, its second half B = [um, ue) descending (B's
// smallest key at ue-1).  A head that runs past its half then reads the other
// half's largest keys, in descending order, which are never smaller than
// anything still to be taken from the other side (Knuth TAOCP vol. 3, 5.2.4,
// merging with sentinels; Batcher's bitonic sequences): the serial merge and
// the merge-path search need no end-of-run tests.  When a phantom key equals
// the other side's head, every key left on that side equals it too, so the
// values written are the right ones.  A run whose keys are identical bit
// patterns when equal (plain keys) is all this needs.  Used for 32-bit keys
// (bitonic_levels below).

// Measured on GB300 (2^30 keys, tile sort): 32-bit keys 6.09 -> 5.80 ms with
// the bitonic layout, 64-bit keys 11.94 -> 12.42 ms; so only 32-bit keys use it
// (BIT below), 64-bit keys keep the end-of-run tests and ascending halves.
template <typename V> constexpr bool bitonic_levels() { return sizeof(V) == 4; }

// Stores a thread's E ascending keys, which start at position pos0 of a run
// of R keys: ascending when the run is the first half of its unit of 2R,
// descending inside the run when it is the second half (BIT only).  last: the
// run is the whole sorted tile (always ascending).
template <int E, typename S, bool BIT = bitonic_levels<typename S::V>()>
__device__ __forceinline__ void store_bitonic(const S& s, int pos0, int R, bool last, const typename S::V (&out)[E])
{
    const int rs = pos0 & ~(R - 1);
    if (BIT && !last && (rs & R)) {
        const int top = 2 * rs + R - 1 - pos0;  // mirrored position of pos0
#pragma unroll
        for (int i = 0; i < E; i++) s.st(top - i, out[i]);
    } else {
        store_block<E>(s, pos0, out);
    }
}

// Merge-path split of diagonal d of a bitonic unit (B stored descending).
template <typename S>
__device__ __forceinline__ int merge_path_bitonic(const S& s, int us, int um, int ue, int d)
{
    int a0 = d - (ue - um) > 0 ? d - (ue - um) : 0;
    int a1 = d < um - us ? d : um - us;
    while (a0 < a1) {
        const int mid = (a0 + a1) >> 1;
        // B's element of rank d-1-mid sits at ue-1-(d-1-mid)
        if (!S::lt(s.ld(ue - d + mid), s.ld(us + mid))) a0 = mid + 1;
        else a1 = mid;
    }
    return a0;
}

// Tile levels: NT*E elements in sorted runs of U0/2 (stored by store_bitonic)
// that double each level (units of U = U0, 2*U0, ... keys, all powers of
// two); every thread owns exactly E outputs that never straddle a unit.
template <int NT, int E, typename S>
__device__ void merge_levels_pow2(const S& s, int U0 = 2 * E)
{
    using V = typename S::V;
    const int pos0 = threadIdx.x * E;
#pragma unroll 1
    for (int U = U0; U <= NT * E; U <<= 1) {
        const int us = pos0 & ~(U - 1), um = us + U / 2, ue = us + U;
        const int d = pos0 - us;
        V out[E];
        if constexpr (bitonic_levels<V>()) {
            const int x = merge_path_bitonic(s, us, um, ue, d);
            int ai = us + x, bj = ue - 1 - (d - x);  // heads: A ascending, B descending
            V a = s.ld(ai), b = s.ld(bj);
#pragma unroll
            for (int i = 0; i < E; i++) {
                const bool p = !S::lt(b, a);  // A wins ties
                out[i] = p ? a : b;
                if (p) a = s.ld(++ai);
                else b = s.ld(--bj);
            }
        } else {
            const int x = merge_path(s, us, um, ue, d);
            serial_merge<E, false>(s, us + x, um, um + (d - x), ue, E, out);
        }
        __syncthreads();
        store_bitonic<E>(s, pos0, U, U == NT * E, out);
        __syncthreads();
    }
}

// General levels: the n elements of `s` form P sorted pieces with boundaries
// off[0..P] (off[0] = 0, off[P] = n, in shared memory); adjacent units are
// merged level by level until one sorted run remains, in place.  At level l a
// unit is 2^(l+1) consecutive pieces, so the unit holding a position is the
// position's piece index shifted right by l+1 (found once per thread).  A
// thread's E outputs may cross into later units; each crossing restarts the
// merge at the next unit's head.  Ties keep the lower piece first.
// Requires n <= NT*E.
template <int NT, int E, typename S>
__device__ void merge_pieces(const S& s, const int* off, int P, int n)
{
    using V = typename S::V;
    const int pos0 = threadIdx.x * E;
    const int cnt = n - pos0 < E ? n - pos0 : E;
    int p0 = 0;  // last piece starting at or before pos0
    if (cnt > 0) {
        int hi = P - 1;
        while (p0 < hi) {
            const int mid = (p0 + hi + 1) >> 1;
            if (off[mid] <= pos0) p0 = mid;
            else hi = mid - 1;
        }
    }
    for (int sh = 1; (1 << (sh - 1)) < P; sh++) {
        const int w = 1 << (sh - 1);
        V out[E];
        if (cnt > 0) {
            int u = p0 >> sh;
            int us = off[min(u * 2 * w, P)], um = off[min(u * 2 * w + w, P)], ue = off[min(u * 2 * w + 2 * w, P)];
            const int x = merge_path(s, us, um, ue, pos0 - us);
            int ai = us + x, bi = um + (pos0 - us - x);
            int left = ue - pos0;  // outputs left in this unit
            V a = s.ld(ai), b = s.ld(bi);
#pragma unroll
            for (int i = 0; i < E; i++) {
                if (i < cnt) {
                    if (left == 0) {
                        // this unit is exhausted: continue with the next non-empty unit
                        do {
                            u++;
                            us = ue;
                            um = off[min(u * 2 * w + w, P)];
                            ue = off[min(u * 2 * w + 2 * w, P)];
                        } while (us == ue && ue < n);
                        ai = us;
                        bi = um;
                        left = ue - us;
                        a = s.ld(ai);
                        b = s.ld(bi);
                    }
                    const bool p = (bi >= ue) || ((ai < um) && !S::lt(b, a));
                    out[i] = p ? a : b;
                    const int nx = p ? ai + 1 : bi + 1;
                    const V c = s.ld(nx);
                    if (p) {
                        a = c;
                        ai = nx;
                    } else {
                        b = c;
                        bi = nx;
                    }
                    left--;
                }
            }
        }
        __syncthreads();
        if (cnt > 0) {
#pragma unroll
            for (int i = 0; i < E; i++)
                if (i < cnt) s.st(pos0 + i, out[i]);
        }
        __syncthreads();
    }
}

// Aligned levels: like merge_pieces, but every piece boundary off[0..P] is a
// multiple of E (the pieces were padded with copies of the largest key), so
// every merge unit starts and ends on a thread boundary and each thread runs
// the plain two-way merge of its unit.  The padding sorts last; since a pad
// equals the largest key bit for bit, the first n - (padding) outputs are the
// real keys in order.
template <int NT, int E, typename S>
__device__ void merge_pieces_aligned(const S& s, const int* off, int P, int n)
{
    using V = typename S::V;
    const int pos0 = threadIdx.x * E;
    const bool act = pos0 < n;
    int p0 = 0;  // last piece starting at or before pos0
    if (act) {
        int hi = P - 1;
        while (p0 < hi) {
            const int mid = (p0 + hi + 1) >> 1;
            if (off[mid] <= pos0) p0 = mid;
            else hi = mid - 1;
        }
    }
    for (int sh = 1; (1 << (sh - 1)) < P; sh++) {
        const int w = 1 << (sh - 1);
        V out[E];
        if (act) {
            const int u = p0 >> sh;
            const int us = off[min(u * 2 * w, P)], um = off[min(u * 2 * w + w, P)];
            const int ue = off[min(u * 2 * w + 2 * w, P)];
            const int x = merge_path(s, us, um, ue, pos0 - us);
            serial_merge<E, false>(s, us + x, um, um + (pos0 - us - x), ue, E, out);
        }
        __syncthreads();
        if (act) store_block<E>(s, pos0, out);
        __syncthreads();
    }
}

// Number of elements of the sorted range src[lo, hi) that are < v (lower
// bound, STRICT = true) or <= v (upper bound, STRICT = false).
template <bool STRICT, typename K>
__device__ __forceinline__ int64_t bound(const GBuf<K>& src, int64_t lo, int64_t hi, const K& v)
{
    int64_t a = lo, b = hi;
    while (a < b) {
        int64_t m = a + ((b - a) >> 1);
        K x = src.ld(m);
        bool go_right = STRICT ? key_lt(x, v) : !key_lt(v, x);
        if (go_right) a = m + 1;
        else b = m;
    }
    return a - lo;
}

// ------------------------------------------------------------- instances
// A batch of independent sorts that share n_B and n_P (the batched entry
// point bins segments by size; a single sort is one instance).  Instance i
// occupies [off(i), off(i) + len(i)) of the key arrays; its blocks have
// length ceil(len(i) / n_B).
struct Inst {
    const int64_t* base;  // per-instance start (nullptr: one instance at 0)
    const int64_t* n;     // per-instance length
    int64_t count;
    int64_t n0;           // length of the single instance when base is null
    __device__ __forceinline__ int64_t off(int64_t i) const { return base ? base[i] : 0; }
    __device__ __forceinline__ int64_t len(int64_t i) const { return base ? n[i] : n0; }
    // The instance holding absolute position x (instances at increasing offsets).
    __device__ __forceinline__ int64_t find(int64_t x) const
    {
        if (!base) return 0;
        int64_t a = 0, b = count - 1;
        while (a < b) {
            const int64_t m = (a + b + 1) >> 1;
            if (base[m] <= x) a = m;
            else b = m - 1;
        }
        return a;
    }
};

// Bounds [bs, be) of block b (relative to its instance) for instance length N.
__device__ __forceinline__ void block_bounds(int64_t N, int64_t n_B, int64_t b, int64_t& bs, int64_t& be)
{
    const int64_t L = (N + n_B - 1) / n_B;
    bs = b * L < N ? b * L : N;
    be = bs + L < N ? bs + L : N;
}

// CTAs per SM a data-pass kernel of NT threads with E keys per thread is
// compiled for: as many as the register file holds at about 16 + w*E
// registers a thread (w = 32-bit words a key takes in registers), and no
// more than 1024 threads per SM in all.
template <typename K, int NT, int E> constexpr int data_ctas()
{
    constexpr int w = sizeof(K) == 4 ? 1 : sizeof(K) == 8 ? 2 : PS_REC_REGW;
    constexpr int c = 65536 / (NT * (16 + w * E));
    constexpr int cap = 1024 / NT < 1 ? 1 : 1024 / NT;
    return c < 1 ? 1 : (c > cap ? cap : c);
}

// ------------------------------------------------------------ step 1: tiles
// Loads of one tile straight into registers, for plain keys: warp w takes
// tile positions [w*32*E, (w+1)*32*E) and lane l the 16-byte vectors at
// positions w*32*E + v*32*VEC + l*VEC (VEC keys each), so that every warp-wide
// load covers 32*16 contiguous bytes.  Which keys a lane holds does not
// matter (they are sorted next), so no shared-memory staging is needed.
// A full tile whose start is 16-byte aligned takes vector loads; a short or
// unaligned one takes guarded scalar loads at the same positions.  Missing
// keys of a short tile become the largest key.
template <int NT, int E, typename K, int XF>
__device__ __forceinline__ void tile_load_regs(const GBuf<K>& src, int64_t o, int n, K (&r)[E])
{
    constexpr int VEC = 16 / (int)sizeof(K);
    static_assert(E % VEC == 0, "keys per thread must be a multiple of the vector width");
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int base = w * 32 * E + lane * VEC;
    const K* g = src.p + o;
    if (n == NT * E && ((uintptr_t)g & 15) == 0) {
#pragma unroll
        for (int v = 0; v < E / VEC; v++) {
            const int i = base + v * 32 * VEC;
            if constexpr (sizeof(K) == 8) {
                ulonglong2 x = make_ulonglong2(0, 0);
                if (PS_IN(o + i + 1, src.n, 3)) x = __ldcs((const ulonglong2*)(g + i));
                r[v * 2] = xform<XF>((K)x.x);
                r[v * 2 + 1] = xform<XF>((K)x.y);
            } else {
                uint4 x = make_uint4(0, 0, 0, 0);
                if (PS_IN(o + i + 3, src.n, 3)) x = __ldcs((const uint4*)(g + i));
                r[v * 4] = xform<XF>((K)x.x);
                r[v * 4 + 1] = xform<XF>((K)x.y);
                r[v * 4 + 2] = xform<XF>((K)x.z);
                r[v * 4 + 3] = xform<XF>((K)x.w);
            }
        }
    } else {
#pragma unroll
        for (int v = 0; v < E / VEC; v++)
#pragma unroll
            for (int q = 0; q < VEC; q++) {
                const int i = base + v * 32 * VEC + q;
                r[v * VEC + q] = i < n ? xform<XF>(src.ld(o + i)) : KT<K>::maxkey();
            }
    }
}
// Records: the same positions, two records per step (a 16-byte vector of
// keys and an 8-byte vector of payloads from the two arrays).
template <int NT, int E, typename K, int XF>
__device__ __forceinline__ void tile_load_regs(const GBuf<Rec>& src, int64_t o, int n, Rec (&r)[E])
{
    static_assert(E % 2 == 0, "records per thread must be even");
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int base = w * 32 * E + lane * 2;
    const uint64_t* gk = src.k + o;
    const uint32_t* gp = src.p + o;
    if (n == NT * E && ((uintptr_t)gk & 15) == 0 && ((uintptr_t)gp & 7) == 0) {
#pragma unroll
        for (int v = 0; v < E / 2; v++) {
            const int i = base + v * 64;
            ulonglong2 x = make_ulonglong2(0, 0);
            uint2 y = make_uint2(0, 0);
            if (PS_IN(o + i + 1, src.n, 3)) {
                x = __ldcs((const ulonglong2*)(gk + i));
                y = __ldcs((const uint2*)(gp + i));
            }
            r[v * 2] = Rec{x.x, y.x};
            r[v * 2 + 1] = Rec{x.y, y.y};
        }
    } else {
#pragma unroll
        for (int v = 0; v < E / 2; v++)
#pragma unroll
            for (int q = 0; q < 2; q++) {
                const int i = base + v * 64 + q;
                r[v * 2 + q] = i < n ? src.ld(o + i) : KT<Rec>::maxkey();
            }
    }
}

// One tile of n <= NT*E keys, read from src at so and written to dst at dso
// (FINAL: with the inverse transform): loads straight into registers
// (tile_load_regs), a register sorting network per thread, WLEV warp-shuffle
// merge levels, then shared-memory merge-path levels for the rest.  Missing
// keys of a short tile count as the largest key, which sorts last and is
// never written.  The final loop still reads sb: a caller that reuses sb
// synchronises the CTA first.
template <int NT, int E, typename K, int XF, bool FINAL, int WLEV, typename SB>
__device__ __forceinline__ void tile_sort_body(const SB& sb, const GBuf<K>& src, int64_t so, const GBuf<K>& dst,
                                               int64_t dso, int n)
{
    constexpr int T = NT * E;
    using SV = typename ViewOf<SB>::type;
    K r[E];
    tile_load_regs<NT, E, K, XF>(src, so, n, r);
    reg_sort<E>(r);
    if constexpr (WLEV > 0) warp_merge_levels<E, WLEV>(r);
    store_bitonic<E>(SV{sb}, threadIdx.x * E, E << WLEV, (E << WLEV) >= T, r);
    __syncthreads();
    merge_levels_pow2<NT, E>(SV{sb}, E << (WLEV + 1));
    for (int i = threadIdx.x; i < n; i += NT) {
        if (FINAL) dst.template stx<XF>(dso + i, sb.ld(i));
        else dst.st(dso + i, sb.ld(i));
    }
}

// One CTA sorts one tile of NT*E keys of one block of one instance (tiles
// never straddle a block boundary; every block gets R0 tile slots, the
// number the longest block needs).  Loads apply the order-key transform XF.
// FINAL: the tile is the whole sorted result, so the store applies the
// inverse transform.
// iptr (plain keys, batches): instance i's keys live in their own buffer
// iptr[i] (in the compact layout they would start at in.off(i)); the tile is
// read from there and, when FINAL, written back there.
template <int NT, int E, typename K, int XF, bool FINAL, int WLEV = 0>
__global__ void __launch_bounds__(NT, (data_ctas<K, NT, E>()))
    k_tile_sort(GBuf<K> src, GBuf<K> dst, Inst in, int64_t n_B, int64_t R0, K* const* iptr)
{
    constexpr int T = NT * E;
    constexpr bool PLAIN = sizeof(K) == 4 || sizeof(K) == 8;
    using SB = typename TileBuf<K, E>::type;
    extern __shared__ __align__(16) char smem[];
    char* sp = smem;
    SB sb = SB::carve(sp, T);
    const int64_t per_inst = n_B * R0;
    const int64_t inst = blockIdx.x / per_inst;
    const int64_t rest = blockIdx.x - inst * per_inst;
    const int64_t b = rest / R0, t = rest - b * R0;
    if (inst >= in.count) return;
    int64_t bs, be;
    block_bounds(in.len(inst), n_B, b, bs, be);
    const int64_t ts = bs + t * T;
    if (ts >= be) return;
    const int64_t o = in.off(inst) + ts;
    const int n = (int)(be - ts < T ? be - ts : T);
    if constexpr (PLAIN) {
        if (iptr) {
            const GBuf<K> own{iptr[inst] + ts, (int64_t)n};
            if (FINAL) tile_sort_body<NT, E, K, XF, FINAL, WLEV>(sb, own, 0, own, 0, n);
            else tile_sort_body<NT, E, K, XF, FINAL, WLEV>(sb, own, 0, dst, o, n);
            return;
        }
    }
    tile_sort_body<NT, E, K, XF, FINAL, WLEV>(sb, src, o, dst, o, n);
}

// ------------------------------------------- batches: persistent front kernel
// Sorts every short instance of a batch in one launch of a grid sized to the
// GPU (persistent CTAs).  Work items come from one device counter (*next,
// zero at launch): items [0, tiles.count) are instances of at most NT*E keys,
// each sorted by the whole CTA (tile_sort_body); the items after them are
// groups of NT/32 instances of at most 1024 keys, one per warp, each sorted
// in registers (32 keys per lane, a sorting network, then five warp-shuffle
// merge levels: 32 runs of 32 become one run of 1024) and written out through
// the warp's own part of shared memory.  Larger items come first, so the
// short ones fill in behind them.  tptr/sptr (optional): each instance in
// its own buffer, as in k_tile_sort.
template <int NT, int E, typename K, int XF, int WLEV>
__global__ void __launch_bounds__(NT, (data_ctas<K, NT, E>()))
    k_batch_front(GBuf<K> keys, Inst tiles, K* const* tptr, Inst small, K* const* sptr, unsigned long long* next)
{
    static_assert(E == 32 && NT * E >= (NT / 32) * 1024, "one 1024-key run per warp in the tile buffer");
    constexpr int T = NT * E;
    constexpr int WARPS = NT / 32;
    using SB = typename TileBuf<K, E>::type;
    using SV = typename ViewOf<SB>::type;
    extern __shared__ __align__(16) char smem[];
    __shared__ unsigned long long item_s;
    char* sp = smem;
    SB sb = SB::carve(sp, T);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long n_groups = (small.count + WARPS - 1) / WARPS;
    const unsigned long long total = (unsigned long long)(tiles.count + n_groups);
    for (;;) {
        // thread 0 writes item_s again only after the barrier that ends the
        // item, which every thread reaches after reading it
        if (threadIdx.x == 0) item_s = atomicAdd(next, 1ull);
        __syncthreads();
        const unsigned long long item = item_s;
        if (item >= total) return;
        if (item < (unsigned long long)tiles.count) {
            const int64_t i = (int64_t)item;
            const int n = (int)tiles.len(i);
            if (tptr) {
                const GBuf<K> own{tptr[i], (int64_t)n};
                tile_sort_body<NT, E, K, XF, true, WLEV>(sb, own, 0, own, 0, n);
            } else {
                tile_sort_body<NT, E, K, XF, true, WLEV>(sb, keys, tiles.off(i), keys, tiles.off(i), n);
            }
        } else {
            const int64_t i = (int64_t)(item - (unsigned long long)tiles.count) * WARPS + w;
            if (i < small.count) {
                const int n = (int)small.len(i);
                const GBuf<K> g = sptr ? GBuf<K>{sptr[i], (int64_t)n} : keys;
                const int64_t o = sptr ? 0 : small.off(i);
                K r[E];
#pragma unroll
                for (int j = 0; j < E; j++) {
                    const int x = j * 32 + lane;  // coalesced; which keys a lane holds does not matter
                    r[j] = x < n ? xform<XF>(g.ld(o + x)) : KT<K>::maxkey();
                }
                reg_sort<E>(r);
                warp_merge_levels<E, 5>(r);  // lane l now holds positions l*32 .. l*32+31
                store_block<E>(SV{sb}, w * 1024 + lane * E, r);
                __syncwarp();
                for (int x = lane; x < n; x += 32) g.template stx<XF>(o + x, sb.ld(w * 1024 + x));
            }
        }
        __syncthreads();  // the tile buffer is free again
    }
}

// ----------------------------------------------------------- merge jobs
// A merge job is a set of groups; group g merges K sorted runs of `src`
// into one sorted range of `dst` starting at out_base(g).  Groups are
// numbered instance by instance.
//   kind 0 (in-block pass, step 1): group = (instance, block b, index gi); run
//          r covers [bs + (gi*K + r)*W, +W) clipped to the block; output in place.
//   kind 1 (final merge, step 4): group = (instance, partition k); run r =
//          block r's piece [bs + s[r][k], bs + s[r][k+1]); output at O_k.
struct MergeJob {
    int kind;
    int K;
    Inst in;
    int64_t n_B;
    int64_t N;                       // extent of the key arrays
    int64_t W, gpb;                  // kind 0
    const int64_t* splits;           // kind 1: rows (inst*n_B + b), n_P+1 columns
    const int64_t* offsets;          // kind 1: rows inst, n_P+1 absolute offsets
    int64_t n_P;                     // kind 1
    int64_t k0;                      // kind 1, one instance: group g is partition k0 + g
    __device__ __forceinline__ void run(int64_t g, int r, int64_t& lo, int64_t& hi) const
    {
        if (kind == 0) {
            const int64_t gpi = n_B * gpb, inst = g / gpi, lg = g - inst * gpi;
            const int64_t b = lg / gpb, gi = lg - b * gpb;
            int64_t bs, be;
            block_bounds(in.len(inst), n_B, b, bs, be);
            const int64_t o = in.off(inst), s = bs + (gi * K + r) * W;
            lo = o + (s < be ? s : be);
            hi = o + (s + W < be ? s + W : be);
        } else {
            const int64_t inst = g / n_P, k = g - inst * n_P + k0;
            int64_t bs, be;
            block_bounds(in.len(inst), n_B, r, bs, be);
            const int64_t* row = splits + (inst * n_B + r) * (n_P + 1);
            lo = in.off(inst) + bs + row[k];
            hi = in.off(inst) + bs + row[k + 1];
        }
    }
    __device__ __forceinline__ int64_t out_base(int64_t g) const
    {
        if (kind == 0) {
            const int64_t gpi = n_B * gpb, inst = g / gpi, lg = g - inst * gpi;
            const int64_t b = lg / gpb, gi = lg - b * gpb;
            int64_t bs, be;
            block_bounds(in.len(inst), n_B, b, bs, be);
            const int64_t s = bs + gi * K * W;
            return in.off(inst) + (s < be ? s : be);
        }
        const int64_t inst = g / n_P, k = g - inst * n_P + k0;
        return offsets[inst * (n_P + 1) + k];
    }
    // number of elements of group g
    __device__ __forceinline__ int64_t size(int64_t g) const
    {
        if (kind == 0) {
            const int64_t gpi = n_B * gpb, inst = g / gpi, lg = g - inst * gpi;
            const int64_t b = lg / gpb;
            int64_t bs, be;
            block_bounds(in.len(inst), n_B, b, bs, be);
            const int64_t s = out_base(g), e = s + (int64_t)K * W, end = in.off(inst) + be;
            return (e < end ? e : end) - s;
        }
        const int64_t inst = g / n_P, k = g - inst * n_P + k0;
        return offsets[inst * (n_P + 1) + k + 1] - offsets[inst * (n_P + 1) + k];
    }
};

// Window table of one refinement level: group g merges the K sorted runs
// [lo[g*K + r], hi[g*K + r]) of the source into [base[g], base[g] + size[g])
// of the destination; *ng groups exist (a device-side count).
struct Level {
    int K;
    int64_t cap;  // group capacity of the tables (checked builds validate against it)
    int64_t* lo;
    int64_t* hi;
    int64_t* base;
    int64_t* size;
    int64_t* ng;
};

// Level 0 of a merge job: its groups' runs, output bases and sizes.
template <int DUMMY = 0>
__global__ void k_root_windows(MergeJob job, int64_t G, Level L)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= G * job.K) return;
    const int64_t g = idx / job.K;
    const int r = (int)(idx - g * job.K);
    int64_t lo, hi;
    job.run(g, r, lo, hi);
    if (hi < lo) hi = lo;
    if (!PS_IN(g, L.cap, 20)) return;
    L.lo[idx] = lo;
    L.hi[idx] = hi;
    if (r == 0) {
        L.base[g] = job.out_base(g);
        L.size[g] = job.size(g);
    }
    if (idx == 0) *L.ng = G;
}

// Children per group: ceil(M / cnom), at most jcap (so that the sample pool
// always holds more samples than splitters), at least 1.
__device__ __forceinline__ int64_t chunks_for(int64_t M, int64_t cnom, int64_t jcap)
{
    int64_t j = (M + cnom - 1) / cnom;
    if (j > jcap) j = jcap;
    return j < 1 ? 1 : j;
}

// Child counts of every group of a level -> exclusive scan choff[0..G].
// One CTA; G may be large (loops with a carry).
template <int NT>
__global__ void __launch_bounds__(NT) k_chunk_plan(Level L, int64_t cnom, int64_t jcap, int64_t* choff)
{
    const int64_t G = *L.ng < L.cap ? *L.ng : L.cap;
    (void)PS_IN(*L.ng, L.cap + 1, 21);
    int64_t carry = 0;
    for (int64_t base = 0; base < G; base += NT) {
        const int64_t g = base + threadIdx.x;
        const int64_t j = g < G ? chunks_for(L.size[g], cnom, jcap) : 0;
        int64_t tot;
        const int64_t ex = block_exscan<NT>(j, &tot);
        if (g < G) choff[g] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) choff[G] = carry;
}

// floor(a * b / c) for non-negative operands; 64-bit arithmetic when the
// product fits (the common case), 128-bit otherwise.
__device__ __forceinline__ int64_t muldiv(int64_t a, int64_t b, int64_t c)
{
    if (a < (1ll << 31) && b < (1ll << 31)) return (a * b) / c;
    return (int64_t)(((unsigned __int128)a * (uint64_t)b) / (uint64_t)c);
}

template <typename K> struct Splitter {
    K key;
    uint32_t run;
    uint32_t pos;  // position of the splitter inside its run (from the window start)
};

// Per group: cut every run into blocks of S elements (the last block of a run
// may be shorter) and take each block's last element as a sample standing for
// the block's keys; S is chosen so that the pool holds about J*max(SPC*K, 96)
// samples (at most POOL).
// The pool is sorted in shared memory (a multiway merge of the per-run sample
// lists, stable, so ties order by run then position).  Splitter j (1..J-1) is
// the first sample whose cumulative weight reaches j*M/J; child j-1 ends with
// it (inclusive) and child j starts after it.
// The sorted pool also bounds every co-rank: if c samples of run r precede
// splitter j in the pool, the splitter's co-rank in run r lies in
// [c*S, min(c*S + S - 1, len_r)] (all samples: exactly len_r).  These windows
// go to the child level's lo/hi tables, where k_corank narrows them to the
// exact co-rank with a search over at most S elements.
template <int NT, int E, typename K, int SPC>
__global__ void __launch_bounds__(NT) k_pool(Level L, GBuf<K> src, const int64_t* choff, int* chgrp,
                                             Splitter<K>* spl, int64_t ccap, Level C)
{
    constexpr int POOL = NT * E;
    extern __shared__ __align__(16) char smem[];
    const int64_t g = blockIdx.x;
    const int64_t ng = *L.ng < L.cap ? *L.ng : L.cap;
    if (g >= ng) return;
    const int64_t c0 = choff[g];
    const int64_t J = choff[g + 1] - c0;
    if (!PS_IN(c0 + J - 1, ccap, 22) || c0 < 0 || J < 1 || c0 + J > ccap) return;
    // every slot first holds a splitter above all keys, so that a slot the
    // assignment below could miss yields an empty child (and an oversized
    // sibling, merged exactly) rather than stale bytes
    const int Kr = L.K;
    const int64_t* lo = L.lo + g * Kr;
    const int64_t* hi = L.hi + g * Kr;
    for (int64_t j = threadIdx.x; j < J; j += NT) {
        chgrp[c0 + j] = (int)g;
        spl[c0 + j] = Splitter<K>{KT<K>::maxkey(), 0xFFFFFFFFu, 0xFFFFFFFFu};
    }
    // default co-rank windows: the whole run
    for (int64_t t = threadIdx.x; t < (J - 1) * Kr; t += NT) {
        const int64_t c = c0 + 1 + t / Kr;
        const int r = (int)(t % Kr);
        if (!PS_IN(c, C.cap, 35)) continue;
        C.lo[c * Kr + r] = lo[r];
        C.hi[c * Kr + r] = hi[r] > lo[r] ? hi[r] : lo[r];
    }
    if (J <= 1) return;
    __syncthreads();
    char* sp = smem;
    STagged<K> pool{SBuf<K>::carve(sp, POOL), SBuf<uint64_t>::carve(sp, POOL)};
    int* mpos = (int*)sp;                 // pool position of every run's i-th sample
    int* jpos = mpos + POOL;              // pool position of splitter j (-1: none)
    int* off = jpos + (POOL / 2 + 1);
    const int64_t M = L.size[g];
    // about max(SPC*K, 96) samples per child: enough to place every splitter
    // within a few percent of its target rank (each run's co-rank is known
    // to within its S-key block), and no more than the pool holds
    int64_t ptarget = J * (SPC * (int64_t)Kr > 96 ? SPC * (int64_t)Kr : 96);
    if (ptarget > POOL) ptarget = POOL;
    const int64_t room = ptarget - Kr > 1 ? ptarget - Kr : 1;
    const int64_t S = M <= room ? 1 : (M + room - 1) / room;
    const int per = (Kr + NT - 1) / NT;
    const int r0 = threadIdx.x * per;
    int64_t mine = 0;
    for (int r = r0; r < r0 + per && r < Kr; r++) mine += (hi[r] - lo[r] + S - 1) / S;
    int64_t P64;
    int64_t ex = block_exscan<NT>(mine, &P64);
    for (int r = r0; r < r0 + per && r < Kr; r++) {
        off[r] = (int)ex;
        ex += (hi[r] - lo[r] + S - 1) / S;
    }
    if (threadIdx.x == 0) off[Kr] = (int)P64;
    for (int64_t j = threadIdx.x; j < J && j <= POOL / 2; j += NT) jpos[j] = -1;
    __syncthreads();
    const int P = (int)P64;  // <= M/S + K <= POOL
    if (!PS_IN(P, POOL + 1, 23) || P > POOL) return;
    for (int i = threadIdx.x; i < P; i += NT) {
        int x = 0, y = Kr - 1;  // run holding pool slot i: last r with off[r] <= i
        while (x < y) {
            const int m = (x + y + 1) >> 1;
            if (off[m] <= i) x = m;
            else y = m - 1;
        }
        int64_t q = (int64_t)(i - off[x]) * S + (S - 1);
        const int64_t last = hi[x] - lo[x] - 1;
        if (q > last) q = last;
        if (!PS_IN(q, last + 1, 24)) continue;
        cp_elem(pool.kb, i, src, lo[x] + q);
        pool.tb.st(i, ((uint64_t)x << 32) | (uint64_t)(i - off[x]));  // run, ordinal in the run
    }
    cp_async_wait_all();
    __syncthreads();
    merge_pieces<NT, E>(pool, off, Kr, P);
    // weights: sample o of run x (ordinal o, at position min(o*S + S-1, len-1))
    // stands for S keys, or for the len - o*S keys of its run's last block
    const int q0 = threadIdx.x * E;
    int64_t wsum = 0;
#pragma unroll
    for (int i = 0; i < E; i++) {
        if (q0 + i < P) {
            const uint64_t tag = pool.tb.ld(q0 + i);
            const int x = (int)(tag >> 32);
            if (!PS_IN(x, Kr, 25)) continue;
            const int64_t o = (int64_t)(uint32_t)tag, len = hi[x] - lo[x];
            wsum += o == off[x + 1] - off[x] - 1 ? len - o * S : S;
            const int64_t slot = off[x] + o;
            if (PS_IN(slot, off[x + 1], 36) && slot < off[x + 1]) mpos[slot] = q0 + i;
        }
    }
    int64_t tot;
    int64_t cb = block_exscan<NT>(wsum, &tot);
    // A splitter's co-rank exceeds its cumulative weight by the partial block
    // of every other run, (S-1)/2 keys on average: aim the weights that much lower.
    const int64_t adj = (int64_t)(Kr - 1) * (S - 1) / 2;
    // Splitter j goes to the sample whose cumulative weight range (cb, ci]
    // holds its target t_j = max(1, floor(j*M/J) - adj).  The targets grow with
    // j, so each thread walks them along its samples: the first j with
    // t_j > cb comes from one division (for cb >= 1 only unclamped targets
    // qualify, and those satisfy j >= (cb + adj + 1) * J / M), later ones from
    // floor((j+1)*M/J) = floor(j*M/J) + floor(M/J) + carry of the remainders.
    int64_t j = 1;
    if (cb > 0) {
        j = muldiv(cb + adj + 1, J, M) - 1;
        if (j < 1) j = 1;
    }
    const int64_t Mq = M / J, Mr = M - Mq * J;
    int64_t qj = muldiv(j, M, J), rj = j * M - qj * J;
#pragma unroll
    for (int i = 0; i < E; i++) {
        if (q0 + i < P) {
            const Tagged<K> e = pool.ld(q0 + i);
            const int x = (int)(e.tag >> 32);
            if (!PS_IN(x, Kr, 26)) continue;
            const int64_t o = (int64_t)(uint32_t)e.tag, len = hi[x] - lo[x];
            const bool lastblk = o == off[x + 1] - off[x] - 1;
            const int64_t ci = cb + (lastblk ? len - o * S : S);
            for (; j < J; j++) {
                int64_t t = qj - adj;
                if (t < 1) t = 1;
                if (t > ci) break;
                if (t > cb) {
                    const int64_t q = lastblk ? len - 1 : o * S + (S - 1);
                    spl[c0 + j] = Splitter<K>{e.key, (uint32_t)x, (uint32_t)q};
                    if (j <= POOL / 2) jpos[j] = q0 + i;
                }
                qj += Mq;
                rj += Mr;
                if (rj >= J) {
                    rj -= J;
                    qj++;
                }
            }
            cb = ci;
        }
    }
    __syncthreads();
    // co-rank windows of splitters 1..J-1 in every run: c = run r's samples
    // ahead of the splitter in the pool (binary search of their positions)
    for (int64_t t = threadIdx.x; t < (J - 1) * Kr; t += NT) {
        const int64_t j = 1 + t / Kr;
        const int r = (int)(t % Kr);
        const int m = j <= POOL / 2 ? jpos[j] : -1;
        if (m < 0) continue;  // unassigned: the whole run (maximal key)
        int a = off[r], b = off[r + 1];
        const int base = a;
        while (a < b) {
            const int mid = (a + b) >> 1;
            if (mpos[mid] < m) a = mid + 1;
            else b = mid;
        }
        const int64_t c = a - base, len = hi[r] - lo[r];
        const int64_t wlo = c * S < len ? c * S : len;
        const int64_t whi = c * S + S - 1 < len ? c * S + S - 1 : len;
        const int64_t cc = c0 + j;
        if (!PS_IN(cc, C.cap, 37)) continue;
        C.lo[cc * Kr + r] = lo[r] + wlo;
        C.hi[cc * Kr + r] = lo[r] + whi;
    }
}

// Co-ranks: for child c (not the first of its group) and run r, where child
// c starts in run r: runs before the splitter's run contribute their
// elements <= key, runs after it their elements < key, the splitter's own run
// everything up to and including the splitter.  Writes the child level's lo.
// One thread per (child, run) pair: its binary search touches a few 32-byte
// sectors of the window, and the kernel runs near DRAM bandwidth (a warp per
// pair reading whole windows was measured 4x slower).
template <typename K>
__global__ void k_corank(Level L, GBuf<K> src, const Splitter<K>* spl, const int64_t* choff, const int* chgrp,
                         Level C)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int Kr = L.K;
    const int64_t c = idx / Kr;
    const int r = (int)(idx - c * Kr);
    const int64_t ng = *L.ng < L.cap ? *L.ng : L.cap;
    if (c >= choff[ng]) return;
    if (!PS_IN(c, C.cap, 27) || c >= C.cap) return;
    const int64_t g = chgrp[c];
    if (!PS_IN(g, ng, 28) || g < 0 || g >= ng) return;
    const int64_t lo = L.lo[g * Kr + r], hi = L.hi[g * Kr + r];
    int64_t v;
    if (c == choff[g]) {
        v = lo;
    } else {
        const Splitter<K> e = spl[c];
        // the sample pool's window for this co-rank (within the run)
        int64_t a = C.lo[c * Kr + r], b = C.hi[c * Kr + r];
        a = a < lo ? lo : (a > hi ? hi : a);
        b = b < a ? a : (b > hi ? hi : b);
        if ((uint32_t)r < e.run) v = a + bound<false>(src, a, b, e.key);
        else if ((uint32_t)r > e.run) v = a + bound<true>(src, a, b, e.key);
        else v = lo + (int64_t)e.pos + 1;
        v = v < lo ? lo : (v > hi ? hi : v);
    }
    C.lo[c * Kr + r] = v;
}

// Child level completion: hi from the next sibling's lo (or the parent's hi
// for the last child), output base and size.  One warp per child (NT/32
// children per CTA), warp-shuffle sums.
template <int NT>
__global__ void __launch_bounds__(NT) k_child_stats(Level L, const int64_t* choff, const int* chgrp, Level C)
{
    const int lane = threadIdx.x & 31;
    const int64_t c = (int64_t)blockIdx.x * (NT / 32) + (threadIdx.x >> 5);
    const int64_t ng = *L.ng < L.cap ? *L.ng : L.cap;
    int64_t nch = choff[ng];
    (void)PS_IN(nch, C.cap + 1, 29);
    if (nch > C.cap) nch = C.cap;
    if (c >= nch) return;  // whole warps leave together
    const int Kr = L.K;
    const int64_t g = chgrp[c];
    if (!PS_IN(g, ng, 30) || g < 0 || g >= ng) return;
    const bool last = c + 1 >= choff[g + 1];
    int64_t before = 0, sz = 0;
    for (int r = lane; r < Kr; r += 32) {
        const int64_t lo = C.lo[c * Kr + r];
        int64_t hi = last ? L.hi[g * Kr + r] : C.lo[(c + 1) * Kr + r];
        (void)PS_IN(hi - lo, INT64_MAX, 34);  // siblings' windows must not run backwards
        if (hi < lo) hi = lo;
        C.hi[c * Kr + r] = hi;
        before += lo - L.lo[g * Kr + r];
        sz += hi - lo;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        before += __shfl_xor_sync(0xFFFFFFFFu, before, o);
        sz += __shfl_xor_sync(0xFFFFFFFFu, sz, o);
    }
    if (lane == 0) {
        C.base[c] = L.base[g] + before;
        C.size[c] = sz;
        if (c == 0) *C.ng = nch;
    }
}

// Smallest key v such that the windows [a[r], b[r]) of sorted runs hold at
// least t elements <= v (t >= 1): bisection over the key's value domain,
// each step counting with one binary search per run (Sec. 2.3).  Each run's
// search window shrinks with the value interval: elements left of it are
// known to be <= every remaining candidate, elements right of it are known
// to be larger.  Runs are handled by threads in contiguous ranges of at most
// MAXPER (enough for the largest n_B, 4096 runs, at NT threads); all threads
// get the result.
constexpr int MAX_RUNS = 4096;
// The search may start from a bracket [lo0, hi0] known to hold the answer;
// every window then starts at the elements >= lo0 and ends after those <= hi0.
template <int NT, typename K, int MAXPER = (MAX_RUNS + NT - 1) / NT>
__device__ K select_value(const GBuf<K>& src, const int64_t* a, const int64_t* b, int nruns, int64_t t,
                          typename KT<K>::U lo0 = 0, typename KT<K>::U hi0 = KT<K>::umax())
{
    using U = typename KT<K>::U;
    U lo = lo0, hi = hi0;
    (void)PS_IN(nruns, NT * MAXPER + 1, 38);  // more runs than the register windows hold
    const int per = (nruns + NT - 1) / NT;
    const int r0 = threadIdx.x * per;
    int64_t wa[MAXPER], wb[MAXPER];
    int64_t below = 0;  // this thread's elements left of its windows
#pragma unroll
    for (int q = 0; q < MAXPER; q++) {
        const int r = r0 + q;
        const bool ok = q < per && r < nruns;
        wa[q] = ok ? a[r] : 0;
        wb[q] = ok ? b[r] : 0;
        if (ok && lo0 > 0) {  // elements < lo0 are below every candidate
            const int64_t c = bound<true>(src, wa[q], wb[q], KT<K>::from_u(lo0));
            wa[q] += c;
            below += c;
        }
        if (ok && hi0 < KT<K>::umax()) wb[q] = wa[q] + bound<false>(src, wa[q], wb[q], KT<K>::from_u(hi0));
    }
    while (lo < hi) {
        const U mid = lo + ((hi - lo) >> 1);
        const K vm = KT<K>::from_u(mid);
        int64_t c[MAXPER];
        int64_t cnt = below;
#pragma unroll
        for (int q = 0; q < MAXPER; q++) {
            c[q] = bound<false>(src, wa[q], wb[q], vm);
            cnt += c[q];
        }
        cnt = block_sum<NT>(cnt);
        if (cnt >= t) {
            hi = mid;
#pragma unroll
            for (int q = 0; q < MAXPER; q++) wb[q] = wa[q] + c[q];
        } else {
            lo = mid + 1;
#pragma unroll
            for (int q = 0; q < MAXPER; q++) {
                wa[q] += c[q];
                below += c[q];
            }
        }
    }
    return KT<K>::from_u(lo);
}

// Exact co-ranks x[r] in windows [a[r], b[r]) such that the t smallest
// elements (order: key, run, position) are exactly the prefixes [a[r], x[r]).
// Copies of the boundary value are taken from runs in run order.
template <int NT, typename K>
__device__ void exact_corank(const GBuf<K>& src, const int64_t* a, const int64_t* b, int nruns, int64_t t,
                             int64_t* x)
{
    const int per = (nruns + NT - 1) / NT;
    const int r0 = threadIdx.x * per;
    if (t <= 0) {
        for (int r = r0; r < r0 + per && r < nruns; r++) x[r] = a[r];
        __syncthreads();
        return;
    }
    K v = select_value<NT, K>(src, a, b, nruns, t);
    int64_t lbs = 0, eqs = 0;
    for (int r = r0; r < r0 + per && r < nruns; r++) {
        int64_t lb = bound<true>(src, a[r], b[r], v);
        int64_t ub = bound<false>(src, a[r], b[r], v);
        lbs += lb;
        eqs += ub - lb;
    }
    const int64_t below = block_sum<NT>(lbs);
    int64_t tot;
    int64_t pre = block_exscan<NT>(eqs, &tot);
    const int64_t need = t - below;
    for (int r = r0; r < r0 + per && r < nruns; r++) {
        int64_t lb = bound<true>(src, a[r], b[r], v);
        int64_t eq = bound<false>(src, a[r], b[r], v) - lb;
        int64_t rem = need - pre;
        if (rem < 0) rem = 0;
        int64_t take = eq < rem ? eq : rem;
        pre += eq;
        x[r] = a[r] + lb + take;
    }
    __syncthreads();
}

// Merge one group of the last level per CTA (its windows, base and size come
// from the level's table).  BIG = false: groups of at most NT*E elements are
// merged in shared memory; larger ones (possible when a sample pool misjudged
// a split) are appended to `big` and left to the BIG = true launch, which cuts
// each into exact sub-chunks (exact_corank) and merges those one after another.
// Output keys pass through the inverse transform XF.
// ALIGNED (non-BIG only): pieces are padded to multiples of E in shared
// memory and merged by merge_pieces_aligned; a group whose padded size
// exceeds the capacity goes to the BIG launch like an oversized one.
// SORTCHUNK (non-BIG only): the pieces are copied side by side and the chunk
// is sorted as a whole, ignoring that the pieces are sorted (the "copy and
// sort" way of multiway merging, Sec. 2.2).
// iptr (plain keys, batches): the output goes to the instances' own buffers
// instead of dst; a group never straddles two instances, so each chunk finds
// its instance once (in) and writes iptr[i] + (position - in.off(i)).
template <int NT, int E, typename K, int XF, bool BIG, bool ALIGNED, bool SORTCHUNK = false>
__global__ void __launch_bounds__(NT, (BIG ? 1 : data_ctas<K, NT, E>())) k_merge(Level C, GBuf<K> src, GBuf<K> dst, int64_t nout, int64_t* big,
                                              unsigned long long* nbig, K* const* iptr, Inst in)
{
    static_assert(!(BIG && ALIGNED), "the oversized-group path merges unpadded pieces");
    static_assert(!(SORTCHUNK && (BIG || ALIGNED)), "copy-and-sort chunks are unpadded and fit the capacity");
    constexpr int CAP = NT * E;
    using SB = typename TileBuf<K, E>::type;
    using SV = typename ViewOf<SB>::type;
    extern __shared__ __align__(16) char smem[];
    const int Kr = C.K;
    char* sp = smem;
    SB sb = SB::carve(sp, CAP);
    int64_t* a = (int64_t*)sp;                       // window starts
    int64_t* b = BIG ? a + Kr : nullptr;             // window ends (BIG only)
    int64_t* x = BIG ? a + 2 * Kr : nullptr;         // sub-chunk ends (BIG only)
    int* len = (int*)(a + (BIG ? 3 : 1) * Kr);       // piece lengths of the current (sub-)chunk
    int* off = len + Kr;                             // piece offsets in shared memory
    const int per = (Kr + NT - 1) / NT;
    const int r0 = threadIdx.x * per;
    int64_t nwork = BIG ? (int64_t)*nbig : *C.ng;
    if (nwork > C.cap) nwork = C.cap;
    const int64_t stride = BIG ? gridDim.x : (nwork > 0 ? nwork : 1);
    for (int64_t w = blockIdx.x; w < nwork; w += stride) {
        const int64_t c = BIG ? big[w] : w;
        if (!PS_IN(c, C.cap, 31) || c < 0 || c >= C.cap) continue;
        int64_t out = C.base[c];
        int64_t M = C.size[c];
        if (out < 0 || M < 0 || out + M > nout) continue;  // never write outside the output
        if (!BIG && M > CAP) {
            if (threadIdx.x == 0) {
                const unsigned long long slot = atomicAdd(nbig, 1ull);
                if (PS_IN(slot, C.cap, 32) && slot < (unsigned long long)C.cap) big[slot] = c;
            }
            continue;
        }
        for (int r = threadIdx.x; r < Kr; r += NT) {
            a[r] = C.lo[c * Kr + r];
            if constexpr (BIG) b[r] = C.hi[c * Kr + r];
            else len[r] = (int)(C.hi[c * Kr + r] - C.lo[c * Kr + r]);
        }
        __syncthreads();
        while (M > 0) {
            const int64_t take = M <= CAP ? M : CAP;
            if constexpr (BIG) {
                if (M > CAP) exact_corank<NT, K>(src, a, b, Kr, take, x);
                else {
                    for (int r = threadIdx.x; r < Kr; r += NT) x[r] = b[r];
                    __syncthreads();
                }
                for (int r = threadIdx.x; r < Kr; r += NT) len[r] = (int)(x[r] - a[r]);
                __syncthreads();
            }
            auto slot = [](int l) { return ALIGNED ? (l + E - 1) & ~(E - 1) : l; };
            int64_t mine = 0;
            for (int r = r0; r < r0 + per && r < Kr; r++) mine += slot(len[r]);
            int64_t tot;
            int64_t ex = block_exscan<NT>(mine, &tot);
            if (ALIGNED && tot > CAP) {  // padded pieces do not fit (uniform over the CTA)
                if (threadIdx.x == 0) {
                    const unsigned long long q = atomicAdd(nbig, 1ull);
                    if (PS_IN(q, C.cap, 32) && q < (unsigned long long)C.cap) big[q] = c;
                }
                break;
            }
            for (int r = r0; r < r0 + per && r < Kr; r++) {
                off[r] = (int)ex;
                ex += slot(len[r]);
            }
            if (threadIdx.x == 0) off[Kr] = (int)(ALIGNED ? tot : take);
            __syncthreads();
            // one warp per run: coalesced copies of the pieces into shared memory
            const int lane = threadIdx.x & 31;
            for (int r = threadIdx.x >> 5; r < Kr; r += NT / 32) {
                const int64_t s0 = a[r];
                const int n_r = len[r], o = off[r];
                for (int i = lane; i < n_r; i += 32) cp_elem(sb, o + i, src, s0 + i);
                if (ALIGNED && lane < slot(n_r) - n_r) sb.st(o + n_r + lane, KT<K>::maxkey());
            }
            cp_async_wait_all();
            __syncthreads();
            if constexpr (SORTCHUNK) {
                K r[E];
                load_block<E>(sb, threadIdx.x * E, r);
#pragma unroll
                for (int j = 0; j < E; j++)
                    if (threadIdx.x * E + j >= (int)take) r[j] = KT<K>::maxkey();
                reg_sort<E>(r);
                store_bitonic<E>(SV{sb}, threadIdx.x * E, E, E >= CAP, r);
                __syncthreads();
                merge_levels_pow2<NT, E>(SV{sb});
            } else if (ALIGNED) {
                merge_pieces_aligned<NT, E>(SV{sb}, off, Kr, (int)tot);
            } else {
                merge_pieces<NT, E>(SV{sb}, off, Kr, (int)take);
            }
            bool own_done = false;
            if constexpr (sizeof(K) == 4 || sizeof(K) == 8) {
                if (iptr) {
                    const int64_t ii = in.find(out);
                    const GBuf<K> own{iptr[ii] + (out - in.off(ii)), take};
                    for (int i = threadIdx.x; i < (int)take; i += NT) own.template stx<XF>(i, sb.ld(i));
                    own_done = true;
                }
            }
            if (!own_done)
                for (int i = threadIdx.x; i < (int)take; i += NT) dst.template stx<XF>(out + i, sb.ld(i));
            out += take;
            M -= take;
            if constexpr (BIG) {
                for (int r = threadIdx.x; r < Kr; r += NT) a[r] = x[r];
                __syncthreads();
            }
        }
    }
}

// Selection-tree merge (Sec. 2.2): one thread merges one whole group of the
// last level.  Its run heads live in shared memory; a loser tree over KP
// leaves (KP a power of two >= K; leaves K..KP-1 are empty runs) holds at
// every inner node the loser of the match played there and at node 0 the
// overall winner.  Each output takes the winner's head, advances that run
// (reading device memory) and replays the matches on its leaf-to-root path.
// Order: non-empty before empty, then key, then run index (ties to the lower
// block, as the merge of Sec. 2.2 needs no particular tie rule but the
// output must be unique).  TPB threads per CTA, each with its own tree.
template <typename K, int XF>
__global__ void k_merge_select(Level C, GBuf<K> src, GBuf<K> dst, int64_t nout, int KP, int TPB)
{
    extern __shared__ __align__(16) char smem[];
    const int Kr = C.K;
    int64_t ng = *C.ng;
    if (ng > C.cap) ng = C.cap;
    const int64_t c = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (threadIdx.x >= TPB || c >= ng) return;
    char* mine = smem + (size_t)threadIdx.x * KP * (sizeof(K) + 2 * sizeof(int64_t) + sizeof(int));
    K* head = (K*)mine;
    int64_t* pos = (int64_t*)(head + KP);
    int64_t* end = pos + KP;
    int* tree = (int*)(end + KP);
    const int64_t out0 = C.base[c], M = C.size[c];
    if (out0 < 0 || M < 0 || out0 + M > nout) return;
    for (int r = 0; r < KP; r++) {
        int64_t lo = 0, hi = 0;
        if (r < Kr) {
            lo = C.lo[c * Kr + r];
            hi = C.hi[c * Kr + r];
        }
        pos[r] = lo;
        end[r] = hi > lo ? hi : lo;
        head[r] = lo < hi ? src.ld(lo) : KT<K>::maxkey();
        tree[r] = -1;
    }
    // r beats q: r is non-empty and q empty, or both non-empty and
    // (head, run) of r is smaller
    auto beats = [&](int r, int q) {
        const bool er = pos[r] >= end[r], eq = pos[q] >= end[q];
        if (er != eq) return eq;
        if (er) return r < q;
        if (key_lt(head[r], head[q])) return true;
        if (key_lt(head[q], head[r])) return false;
        return r < q;
    };
    // build: leaves enter one by one; the first arrival at an inner node
    // waits there, the second plays it, the loser stays
    for (int r = 0; r < KP; r++) {
        int cand = r;
        int node = (r + KP) >> 1;
        bool placed = false;
        while (node >= 1) {
            if (tree[node] < 0) {
                tree[node] = cand;
                placed = true;
                break;
            }
            if (beats(tree[node], cand)) {
                const int t = tree[node];
                tree[node] = cand;
                cand = t;
            }
            node >>= 1;
        }
        if (!placed) tree[0] = cand;
    }
    for (int64_t i = 0; i < M; i++) {
        const int w = tree[0];
        dst.template stx<XF>(out0 + i, head[w]);
        pos[w]++;
        if (pos[w] < end[w]) head[w] = src.ld(pos[w]);
        int cand = w;
        for (int node = (w + KP) >> 1; node >= 1; node >>= 1) {
            if (beats(tree[node], cand)) {
                const int t = tree[node];
                tree[node] = cand;
                cand = t;
            }
        }
        tree[0] = cand;
    }
}

// ------------------------------------------------------------ step 2 and 3
// Regular sampling (Sec. 2.3): sample j (1..n_P-1) of non-empty sorted block
// b of length m is block[floor(j*m/n_P)].  Trailing blocks are the only
// empty ones, so the non-empty blocks of an instance are b < ceil(N/L).
// Samples of (instance, block) occupy row inst*n_B + b of n_P-1 slots.
template <typename K>
__global__ void k_psrs_samples(GBuf<K> blk, GBuf<K> samples, Inst in, int64_t n_B, int64_t n_P)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t per = n_P - 1;
    if (idx >= in.count * n_B * per) return;
    const int64_t row = idx / per, j = idx - row * per + 1;
    const int64_t inst = row / n_B, b = row - inst * n_B;
    int64_t bs, be;
    block_bounds(in.len(inst), n_B, b, bs, be);
    const int64_t m = be - bs;
    if (m <= 0) return;
    const int64_t pos = (int64_t)(((unsigned __int128)j * (uint64_t)m) / (uint64_t)n_P);
    if (!PS_IN(pos, m, 33)) return;
    samples.st(idx, blk.ld(in.off(inst) + bs + pos));
}

// PSRS pivot k of an instance = element of rank (k-1)*nb1 + floor((nb1-1)/2)
// of its sorted pool of samples; the pool is nb1 sorted lists, so the rank is
// found by the same value bisection as exact splitting, without sorting the
// pool.  One CTA per (instance, pivot).
template <int NT, typename K>
__global__ void __launch_bounds__(NT) k_psrs_select(GBuf<K> samples, Inst in, int64_t n_B, int64_t n_P, K* piv)
{
    extern __shared__ __align__(16) char smem[];
    int64_t* a = (int64_t*)smem;
    int64_t* b = a + n_B;
    const int64_t inst = blockIdx.x / (n_P - 1), k = blockIdx.x - inst * (n_P - 1) + 1;
    const int64_t N = in.len(inst);
    if (N <= 0) {
        if (threadIdx.x == 0) piv[blockIdx.x] = KT<K>::from_u(0);
        return;
    }
    const int64_t L = (N + n_B - 1) / n_B;
    const int64_t nb1 = (N + L - 1) / L;
    const int64_t per = n_P - 1;
    for (int64_t r = threadIdx.x; r < nb1; r += NT) {
        a[r] = (inst * n_B + r) * per;
        b[r] = a[r] + per;
    }
    __syncthreads();
    const int64_t q = (k - 1) * nb1 + (nb1 - 1) / 2;
    const K v = select_value<NT, K>(samples, a, b, (int)nb1, q + 1);
    if (threadIdx.x == 0) piv[blockIdx.x] = v;
}

// PSRS splits: s[b][k] = number of elements <= P_k in sorted block b.
template <typename K>
__global__ void k_psrs_splits(GBuf<K> blk, const K* piv, Inst in, int64_t n_B, int64_t n_P, int64_t* splits)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= in.count * n_B * (n_P - 1)) return;
    const int64_t row = idx / (n_P - 1), k = idx - row * (n_P - 1) + 1;
    const int64_t inst = row / n_B, b = row - inst * n_B;
    int64_t bs, be;
    block_bounds(in.len(inst), n_B, b, bs, be);
    const int64_t o = in.off(inst);
    splits[row * (n_P + 1) + k] = bound<false>(blk, o + bs, o + be, piv[inst * (n_P - 1) + k - 1]);
}

// PSES (Sec. 2.3): r_k = floor(k*N/n_P); P_k = smallest v with #{x <= v} >=
// max(r_k, 1) (Eq. 1); c_k = r_k - #{x < P_k} (Eq. 2); split of block b =
// #{x < P_k in b} plus the copies of P_k it contributes, taken greedily in
// block order until c_k copies are placed.  One CTA per (instance, pivot).
template <int NT, typename K>
__global__ void __launch_bounds__(NT) k_pses(GBuf<K> blk, Inst in, int64_t n_B, int64_t n_P, K* piv,
                                             int64_t* cvec, int64_t* splits)
{
    extern __shared__ __align__(16) char smem[];
    int64_t* a = (int64_t*)smem;
    int64_t* b = a + n_B;
    const int64_t inst = blockIdx.x / (n_P - 1), k = blockIdx.x - inst * (n_P - 1) + 1;
    const int64_t N = in.len(inst), o = in.off(inst);
    for (int64_t r = threadIdx.x; r < n_B; r += NT) {
        int64_t bs, be;
        block_bounds(N, n_B, r, bs, be);
        a[r] = o + bs;
        b[r] = o + be;
    }
    __syncthreads();
    if (N <= 0) {
        for (int64_t r = threadIdx.x; r < n_B; r += NT) splits[(inst * n_B + r) * (n_P + 1) + k] = 0;
        if (threadIdx.x == 0) {
            piv[blockIdx.x] = KT<K>::from_u(0);
            cvec[blockIdx.x] = 0;
        }
        return;
    }
    const int64_t rk = (int64_t)(((unsigned __int128)k * (uint64_t)N) / (uint64_t)n_P);
    const int64_t t = rk > 0 ? rk : 1;
    // Bracket for the value search: with p_b = min(floor(t*m_b/N), m_b-1) and
    // q_b = ceil(t*m_b/N) - 1 in every non-empty block b, at least t elements
    // are <= max_b block_b[p_b] and fewer than t are below min_b block_b[q_b]
    // (the p_b + 1 and the q_b add up to >= t and < t), so P_k lies between.
    using U = typename KT<K>::U;
    U lo0 = 0, hi0 = KT<K>::umax();
    if constexpr (sizeof(U) <= 8) {
        __shared__ unsigned long long s_lo, s_hi;
        if (threadIdx.x == 0) {
            s_lo = ~0ull;
            s_hi = 0ull;
        }
        __syncthreads();
        for (int64_t r = threadIdx.x; r < n_B; r += NT) {
            const int64_t m = b[r] - a[r];
            if (m <= 0) continue;
            const unsigned __int128 tm = (unsigned __int128)t * (uint64_t)m;
            int64_t p = (int64_t)(tm / (uint64_t)N);
            if (p > m - 1) p = m - 1;
            const int64_t q = (int64_t)((tm + (uint64_t)N - 1) / (uint64_t)N) - 1;
            atomicMax(&s_hi, (unsigned long long)KT<K>::to_u(blk.ld(a[r] + p)));
            atomicMin(&s_lo, (unsigned long long)KT<K>::to_u(blk.ld(a[r] + q)));
        }
        __syncthreads();
        if (s_lo <= s_hi) {
            lo0 = (U)s_lo;
            hi0 = (U)s_hi;
        }
    }
    const K v = select_value<NT, K>(blk, a, b, (int)n_B, t, lo0, hi0);
    const int per = (int)((n_B + NT - 1) / NT);
    const int r0 = threadIdx.x * per;
    int64_t lbs = 0, eqs = 0;
    for (int r = r0; r < r0 + per && r < n_B; r++) {
        int64_t lb = bound<true>(blk, a[r], b[r], v);
        lbs += lb;
        eqs += bound<false>(blk, a[r], b[r], v) - lb;
    }
    const int64_t below = block_sum<NT>(lbs);
    int64_t tot;
    int64_t pre = block_exscan<NT>(eqs, &tot);
    const int64_t ck = rk - below;
    for (int r = r0; r < r0 + per && r < n_B; r++) {
        int64_t lb = bound<true>(blk, a[r], b[r], v);
        int64_t eq = bound<false>(blk, a[r], b[r], v) - lb;
        int64_t rem = ck - pre;
        if (rem < 0) rem = 0;
        int64_t take = eq < rem ? eq : rem;
        pre += eq;
        splits[(inst * n_B + r) * (n_P + 1) + k] = lb + take;
    }
    if (threadIdx.x == 0) {
        piv[blockIdx.x] = v;
        cvec[blockIdx.x] = ck;
    }
}

// Split-table borders: s[b][0] = 0 and s[b][n_P] = block length.
template <int DUMMY = 0>
__global__ void k_split_borders(Inst in, int64_t n_B, int64_t n_P, int64_t* splits)
{
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= in.count * n_B) return;
    const int64_t inst = row / n_B, b = row - inst * n_B;
    int64_t bs, be;
    block_bounds(in.len(inst), n_B, b, bs, be);
    splits[row * (n_P + 1)] = 0;
    splits[row * (n_P + 1) + n_P] = be - bs;
}

// O_k = off(instance) + sum over its blocks of s[b][k]: the elements of
// partitions 0..k-1, i.e. the exclusive scan of the partition totals (Sec. 2),
// for k = 0..n_P, as absolute positions.
template <int DUMMY = 0>
__global__ void k_offsets(const int64_t* splits, Inst in, int64_t n_B, int64_t n_P, int64_t* offsets)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= in.count * (n_P + 1)) return;
    const int64_t inst = idx / (n_P + 1), k = idx - inst * (n_P + 1);
    int64_t s = in.off(inst);
    for (int64_t b = 0; b < n_B; b++) s += splits[(inst * n_B + b) * (n_P + 1) + k];
    offsets[idx] = s;
}

// Trace output: pivots back in the caller's representation.
template <typename K, int XF>
__global__ void k_trace_pivots(const K* piv, int64_t n, GBuf<K> out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out.template stx<XF>(i, piv[i]);
}

}  // namespace ps

/*
 * psort_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded CPU restatement of the four-step parallel
 * samplesort of Tokuue & Ishiyama, "Performance Evaluation of Parallel
 * Sortings on the Supercomputer Fugaku" (arXiv 2305.05245), Section 2:
 *   step 1  sort each block            (Sec. 2, enumerate item 1; Sec. 2.1)
 *   step 2  select n_P-1 pivots        (Sec. 2.3: PSRS regular sampling,
 *                                       PSES exact splitting, Eq. 1, Eq. 2)
 *   step 3  partition every block      (Sec. 2, item 3; Sec. 2.3)
 *   step 4  multiway merge of the k-th partitions at sequential offsets
 *                                      (Sec. 2, item 4; Sec. 2.2 selection tree)
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg may
 * load this file.  It shares no code, header, table or helper with the CUDA
 * library; the product path never calls it.
 *
 * Readings of points the paper leaves open:
 *   R1 block length L = ceil(N/n_B); trailing blocks may be short or empty.
 *   R2 PSRS: sample j (j = 1..n_P-1) of a non-empty sorted block of length m
 *      is block[floor(j*m/n_P)]; empty blocks give no samples; pivot
 *      P_k = S[(k-1)*n_B' + floor((n_B'-1)/2)] of the sorted pool S, where n_B'
 *      is the number of non-empty blocks.
 *   R3 PSES: r_k = floor(k*N/n_P); P_k is the smallest value v with
 *      #{x <= v} >= max(r_k, 1); c_k = r_k - #{x < P_k} (Eq. 1, Eq. 2).
 *   R4 PSES split: the c_k copies of P_k that belong below the k-th split are
 *      taken greedily from blocks in block order.
 *   R5 order: keys compare by their order key kappa (sign flip for signed
 *      integers, IEEE totalOrder bits for floats, so -0.0 < +0.0); records
 *      compare by (kappa(key), payload).
 *   R6 merge ties go to the lower block index.
 *
 * Parity status: every function below is pinned by tests/test_oracle.py
 * (worked examples of Fig. 1 and Fig. 2, brute force on tiny inputs, the
 * closed form of PSES pivots, partition-membership invariants, the PSRS
 * partition-size bound of Shi and Schaeffer).  One choice stays a reading:
 * the paper gives no formula for the PSRS sample and pivot indices (R2), so
 * beyond Fig. 1, Fig. 2(a) and the bound, the exact PSRS pivot values are
 * parity unpinned.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { ORA_I32 = 0, ORA_I64 = 1, ORA_F32 = 2, ORA_F64 = 3, ORA_U32 = 4, ORA_U64 = 5, ORA_PAIR = 6 };
enum { ORA_REGULAR = 0, ORA_EXACT = 1 };

/* One element: its order key, its payload (0 for keys-only input) and its
 * original bit pattern (returned unchanged in the output). */
typedef struct {
    uint64_t k;
    uint32_t p;
    uint64_t v;
} elem;

/* ---- order key (R5) --------------------------------------------------- */

/* Order key of one stored key.  Integers: flip the sign bit so that two's
 * complement order becomes unsigned order.  Floats: IEEE 754 totalOrder on
 * non-NaN values -- a negative number's bits are inverted (larger magnitude
 * sorts lower), a non-negative number gets its sign bit set. */
static uint64_t order_key(int dtype, uint64_t bits)
{
    switch (dtype) {
    case ORA_I32: return (uint64_t)((uint32_t)bits ^ 0x80000000u);
    case ORA_U32: return (uint64_t)(uint32_t)bits;
    case ORA_F32: {
        uint32_t u = (uint32_t)bits;
        if (u & 0x80000000u) return (uint64_t)(uint32_t)~u;
        return (uint64_t)(u | 0x80000000u);
    }
    case ORA_I64: return bits ^ 0x8000000000000000ull;
    case ORA_F64:
        if (bits & 0x8000000000000000ull) return ~bits;
        return bits | 0x8000000000000000ull;
    default: return bits; /* ORA_U64, ORA_PAIR keys are unsigned 64-bit */
    }
}

/* Strict "a before b" in the total order of R5. */
static int less(const elem* a, const elem* b)
{
    if (a->k != b->k) return a->k < b->k;
    return a->p < b->p;
}

/* Value comparison against a (k, p) value. */
static int elem_lt_val(const elem* a, uint64_t k, uint32_t p)
{
    return a->k < k || (a->k == k && a->p < p);
}
static int elem_le_val(const elem* a, uint64_t k, uint32_t p)
{
    return a->k < k || (a->k == k && a->p <= p);
}

/* ---- step 1: sort each block (Sec. 2, item 1) ------------------------- */

/* Textbook bottom-up merge sort (stable) of a[0..n). */
static void merge_sort(elem* a, int64_t n, elem* tmp)
{
    for (int64_t w = 1; w < n; w *= 2) {
        for (int64_t lo = 0; lo < n; lo += 2 * w) {
            int64_t mid = lo + w < n ? lo + w : n;
            int64_t hi = lo + 2 * w < n ? lo + 2 * w : n;
            int64_t i = lo, j = mid, o = lo;
            while (i < mid && j < hi) {
                if (less(&a[j], &a[i])) tmp[o++] = a[j++];
                else tmp[o++] = a[i++];
            }
            while (i < mid) tmp[o++] = a[i++];
            while (j < hi) tmp[o++] = a[j++];
        }
        memcpy(a, tmp, (size_t)n * sizeof(elem));
    }
}

/* Number of elements of the sorted block a[0..m) that are < value (lower
 * bound) or <= value (upper bound), by binary search (Sec. 2.3). */
static int64_t count_lt(const elem* a, int64_t m, uint64_t k, uint32_t p)
{
    int64_t lo = 0, hi = m;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (elem_lt_val(&a[mid], k, p)) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}
static int64_t count_le(const elem* a, int64_t m, uint64_t k, uint32_t p)
{
    int64_t lo = 0, hi = m;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (elem_le_val(&a[mid], k, p)) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

/* ---- step 4: selection tree (Sec. 2.2, Knuth vol. 3 tree of winners) --- */

typedef struct {
    const elem* base; /* first element of the piece */
    int64_t pos, end; /* current head and end of the piece */
} leaf;

/* Winner of two leaves: the one whose head is smaller; an exhausted leaf
 * always loses; on equal heads the lower leaf (block) index wins (R6). */
static int winner(const leaf* lv, int a, int b)
{
    int ea = lv[a].pos >= lv[a].end, eb = lv[b].pos >= lv[b].end;
    if (ea) return b;
    if (eb) return a;
    if (less(&lv[b].base[lv[b].pos], &lv[a].base[lv[a].pos])) return b;
    return a;
}

/* Merge n_leaves sorted pieces into out[0..total) with a tree of winners:
 * tree[1] is the overall winner, node i has children 2i and 2i+1, leaves sit
 * at tree[size + j].  Each extraction replays the path from the leaf that
 * advanced to the root: O(log n_B) per element (Sec. 2.2). */
static void tree_merge(leaf* lv, int n_leaves, elem* out, int64_t total)
{
    int size = 1;
    while (size < n_leaves) size *= 2;
    /* pad with permanently exhausted leaves */
    leaf* all = (leaf*)calloc((size_t)size, sizeof(leaf));
    int* tree = (int*)malloc(sizeof(int) * 2 * (size_t)size);
    for (int j = 0; j < n_leaves; j++) all[j] = lv[j];
    for (int j = 0; j < size; j++) tree[size + j] = j;
    for (int i = size - 1; i >= 1; i--) tree[i] = winner(all, tree[2 * i], tree[2 * i + 1]);
    for (int64_t o = 0; o < total; o++) {
        int w = tree[1];
        out[o] = all[w].base[all[w].pos];
        all[w].pos++;
        for (int i = (size + w) / 2; i >= 1; i /= 2) tree[i] = winner(all, tree[2 * i], tree[2 * i + 1]);
    }
    free(all);
    free(tree);
}

/* ---- the four steps ---------------------------------------------------- */

static uint64_t load_bits(int dtype, const void* keys, int64_t i)
{
    switch (dtype) {
    case ORA_I32: case ORA_U32: case ORA_F32: return ((const uint32_t*)keys)[i];
    default: return ((const uint64_t*)keys)[i];
    }
}
static void store_bits(int dtype, void* keys, int64_t i, uint64_t v)
{
    switch (dtype) {
    case ORA_I32: case ORA_U32: case ORA_F32: ((uint32_t*)keys)[i] = (uint32_t)v; break;
    default: ((uint64_t*)keys)[i] = v; break;
    }
}

/* Inverse of order_key for the value found by the PSES search. */
static uint64_t key_bits(int dtype, uint64_t k)
{
    switch (dtype) {
    case ORA_I32: return (uint64_t)((uint32_t)k ^ 0x80000000u);
    case ORA_U32: return k;
    case ORA_F32: {
        uint32_t u = (uint32_t)k;
        if (u & 0x80000000u) return (uint64_t)(u & 0x7fffffffu);
        return (uint64_t)(uint32_t)~u;
    }
    case ORA_I64: return k ^ 0x8000000000000000ull;
    case ORA_F64:
        if (k & 0x8000000000000000ull) return k & 0x7fffffffffffffffull;
        return ~k;
    default: return k;
    }
}

/*
 * ora_sort: sort n keys (and payloads for ORA_PAIR) with the four-step
 * samplesort and report its intermediates.
 *   keys, payload          input (payload only for ORA_PAIR; may be NULL otherwise)
 *   n_B, n_P               numbers of blocks and partitions (>= 1)
 *   out_keys, out_payload  sorted output
 *   piv_bits, piv_payload  n_P-1 pivots P_1..P_{n_P-1} (original key bits)
 *   c                      n_P-1 tie counts c_k (exact splitting only)
 *   splits                 n_B x (n_P+1) split table, row b = block b
 *   offsets                n_P+1 partition offsets O_0..O_{n_P}
 * Any of piv_bits .. offsets may be NULL.  Returns 0, or -1 on bad arguments
 * or allocation failure.
 */
int ora_sort(int dtype, int mode, int64_t n, const void* keys, const uint32_t* payload,
             int64_t n_B, int64_t n_P, void* out_keys, uint32_t* out_payload,
             uint64_t* piv_bits, uint32_t* piv_payload, int64_t* c, int64_t* splits,
             int64_t* offsets)
{
    if (n < 0 || n_B < 1 || n_P < 1 || dtype < 0 || dtype > ORA_PAIR) return -1;
    if (mode != ORA_REGULAR && mode != ORA_EXACT) return -1;
    int64_t N = n;
    elem* a = (elem*)malloc(sizeof(elem) * (size_t)(N > 0 ? N : 1));
    elem* tmp = (elem*)malloc(sizeof(elem) * (size_t)(N > 0 ? N : 1));
    int64_t* s = (int64_t*)calloc((size_t)(n_B * (n_P + 1)), sizeof(int64_t));
    uint64_t* pk = (uint64_t*)calloc((size_t)n_P, sizeof(uint64_t));
    uint32_t* pp = (uint32_t*)calloc((size_t)n_P, sizeof(uint32_t));
    int64_t* cc = (int64_t*)calloc((size_t)n_P, sizeof(int64_t));
    int64_t* O = (int64_t*)calloc((size_t)(n_P + 1), sizeof(int64_t));
    if (!a || !tmp || !s || !pk || !pp || !cc || !O) {
        free(a); free(tmp); free(s); free(pk); free(pp); free(cc); free(O);
        return -1;
    }
    for (int64_t i = 0; i < N; i++) {
        uint64_t bits = load_bits(dtype == ORA_PAIR ? ORA_U64 : dtype, keys, i);
        a[i].k = order_key(dtype, bits);
        a[i].p = (dtype == ORA_PAIR && payload) ? payload[i] : 0u;
        a[i].v = bits;
    }

    /* Block division (R1, Sec. 2: contiguous blocks of ceil(N/n_B) elements). */
    int64_t L = (N + n_B - 1) / n_B;
#define BLO(b) ((b) * L < N ? (b) * L : N)
#define BHI(b) (((b) + 1) * L < N ? ((b) + 1) * L : N)

    /* Step 1: sort each block sequentially. */
    for (int64_t b = 0; b < n_B; b++) merge_sort(a + BLO(b), BHI(b) - BLO(b), tmp + BLO(b));

    /* Step 2: pivots P_1..P_{n_P-1} (stored at index k-1). */
    if (n_P > 1 && N > 0) {
        if (mode == ORA_REGULAR) {
            /* PSRS (Sec. 2.3): n_P-1 regular samples from each sorted block,
             * sort the n_B'(n_P-1) samples, take pivots at regular intervals (R2). */
            int64_t nb1 = 0;
            for (int64_t b = 0; b < n_B; b++) nb1 += BHI(b) > BLO(b);
            int64_t ns = nb1 * (n_P - 1), q = 0;
            elem* S = (elem*)malloc(sizeof(elem) * (size_t)ns);
            elem* St = (elem*)malloc(sizeof(elem) * (size_t)ns);
            for (int64_t b = 0; b < n_B; b++) {
                int64_t m = BHI(b) - BLO(b);
                if (m == 0) continue;
                for (int64_t j = 1; j < n_P; j++) {
                    int64_t idx = (int64_t)(((unsigned __int128)j * (uint64_t)m) / (uint64_t)n_P);
                    S[q++] = a[BLO(b) + idx];
                }
            }
            merge_sort(S, ns, St);
            for (int64_t k = 1; k < n_P; k++) {
                const elem* e = &S[(k - 1) * nb1 + (nb1 - 1) / 2];
                pk[k - 1] = e->k;
                pp[k - 1] = e->p;
            }
            free(S);
            free(St);
        } else {
            /* PSES (Sec. 2.3, Eq. 1, Eq. 2): bisection over the value domain;
             * at each candidate count the elements <= v in every block by
             * binary search and test Eq. 1 (R3). */
            for (int64_t k = 1; k < n_P; k++) {
                int64_t r = (int64_t)(((unsigned __int128)k * (uint64_t)N) / (uint64_t)n_P);
                int64_t want = r > 0 ? r : 1;
                /* value space: (k << 32 | p) as a 96-bit number in [0, 2^96) */
                unsigned __int128 lo = 0, hi = ((unsigned __int128)1 << 96) - 1;
                while (lo < hi) {
                    unsigned __int128 mid = lo + (hi - lo) / 2;
                    uint64_t vk = (uint64_t)(mid >> 32);
                    uint32_t vp = (uint32_t)mid;
                    int64_t cnt = 0;
                    for (int64_t b = 0; b < n_B; b++)
                        cnt += count_le(a + BLO(b), BHI(b) - BLO(b), vk, vp);
                    if (cnt >= want) hi = mid;
                    else lo = mid + 1;
                }
                pk[k - 1] = (uint64_t)(lo >> 32);
                pp[k - 1] = (uint32_t)lo;
                int64_t below = 0;
                for (int64_t b = 0; b < n_B; b++)
                    below += count_lt(a + BLO(b), BHI(b) - BLO(b), pk[k - 1], pp[k - 1]);
                cc[k - 1] = r - below; /* Eq. 2 */
            }
        }
    }

    /* Step 3: split table (Sec. 2, item 3): s[b][k] = number of elements of
     * sorted block b that fall in partitions 0..k-1. */
    for (int64_t b = 0; b < n_B; b++) {
        int64_t m = BHI(b) - BLO(b);
        s[b * (n_P + 1) + 0] = 0;
        s[b * (n_P + 1) + n_P] = m;
    }
    for (int64_t k = 1; k < n_P; k++) {
        int64_t taken = 0; /* copies of P_k already placed below the split (R4) */
        for (int64_t b = 0; b < n_B; b++) {
            const elem* blk = a + BLO(b);
            int64_t m = BHI(b) - BLO(b), v;
            if (N == 0) v = 0;
            else if (mode == ORA_REGULAR) {
                v = count_le(blk, m, pk[k - 1], pp[k - 1]); /* x <= P_k goes below */
            } else {
                int64_t lb = count_lt(blk, m, pk[k - 1], pp[k - 1]);
                int64_t eq = count_le(blk, m, pk[k - 1], pp[k - 1]) - lb;
                int64_t need = cc[k - 1] - taken;
                if (need < 0) need = 0;
                int64_t take = eq < need ? eq : need;
                taken += take;
                v = lb + take;
            }
            s[b * (n_P + 1) + k] = v;
        }
    }

    /* Offsets: total of each partition, then the sequential (exclusive) scan
     * from the start of the output (Sec. 2). */
    O[0] = 0;
    for (int64_t k = 0; k < n_P; k++) {
        int64_t t = 0;
        for (int64_t b = 0; b < n_B; b++) t += s[b * (n_P + 1) + k + 1] - s[b * (n_P + 1) + k];
        O[k + 1] = O[k] + t;
    }

    /* Step 4: merge the k-th partition of every block into out[O_k ..). */
    leaf* lv = (leaf*)malloc(sizeof(leaf) * (size_t)n_B);
    for (int64_t k = 0; k < n_P; k++) {
        for (int64_t b = 0; b < n_B; b++) {
            lv[b].base = a + BLO(b);
            lv[b].pos = s[b * (n_P + 1) + k];
            lv[b].end = s[b * (n_P + 1) + k + 1];
        }
        tree_merge(lv, (int)n_B, tmp + O[k], O[k + 1] - O[k]);
    }
    free(lv);

    for (int64_t i = 0; i < N; i++) {
        store_bits(dtype == ORA_PAIR ? ORA_U64 : dtype, out_keys, i, tmp[i].v);
        if (dtype == ORA_PAIR && out_payload) out_payload[i] = tmp[i].p;
    }
    for (int64_t k = 0; k + 1 < n_P; k++) {
        if (piv_bits) piv_bits[k] = key_bits(dtype, pk[k]);
        if (piv_payload) piv_payload[k] = pp[k];
        if (c) c[k] = mode == ORA_EXACT ? cc[k] : 0;
    }
    if (splits) memcpy(splits, s, sizeof(int64_t) * (size_t)(n_B * (n_P + 1)));
    if (offsets) memcpy(offsets, O, sizeof(int64_t) * (size_t)(n_P + 1));
#undef BLO
#undef BHI
    free(a); free(tmp); free(s); free(pk); free(pp); free(cc); free(O);
    return 0;
}

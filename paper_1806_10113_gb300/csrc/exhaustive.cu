// exhaustive.cu -- evaluates the makespan of every one of the n! orders of
// each task group and reduces them to best / worst / sum (the brute-force
// search of Sec. 1 of the paper; the best / mean / worst over all orders of
// the NoReorder setup of Sec. 6.2).
//
// Decomposition.  The model's recurrence (tm_device.cuh) only adds and
// takes maxima, so the makespan is max-plus linear in the engine times
// (h, k, d) entering any suffix of the order.  Split an order into a prefix
// pi over n - 4 tasks and a suffix sigma over the remaining 4-task set S:
// entering S, h is the HtD sum of pi's tasks, which depends on S only, so
//     makespan(pi, sigma) = max(d_pi + alpha_S, k_pi + beta_sigma, gamma_sigma)
// with alpha, beta, gamma fixed per (S, sigma) (struct SuffixTab).  A prep
// kernel tabulates them for every 4-subset of every group (24 orders each).
// The enumeration kernel then walks the prefixes of S's complement
// depth-first (one recurrence step per tree node) and, per prefix, spends
// one add and one three-way max per order of S, plus shared tree
// reductions for the minimum and the sum.
//
// Work items.  For a group of n >= 4 tasks, P = n - 4 prefix positions; an
// item fixes S and a head of f = P - pd leading prefix positions, and its
// thread walks the last pd positions (pd = min(P, pdmax)): pd! prefixes x 24
// orders.  Threads take contiguous item ranges holding the same number of
// orders (+- one item).
//
// Reduction.  Every thread keeps its best / worst makespan with the lowest
// lexicographic rank reaching it and the sum.  Inside one item the walk
// visits orders in increasing rank (ascending depth-first choices, then the
// 24 orders of S in lexicographic order), so the walk only records the
// item's min / max and the first prefix reaching each; at the item's end,
// where all lanes of a warp arrive together, that prefix is replayed to get
// the exact rank, if the item can change the running best / worst.  Keys
// (value << 32 | rank) merge through 64-bit atomics (reduced across the warp
// first), so the order in which items are visited does not matter.  A
// finalize kernel writes tm_stats and handles n <= 3.
#include <algorithm>

#include "tm_device.cuh"

namespace tmgpu {
namespace {

constexpr int kEnumBlock = 128;
constexpr unsigned kFull = 0xFFFFFFFFu;

// 4-subsets of {0..11} in colexicographic order: the subsets of {0..n-1}
// are the first C(n, 4) entries, for every n.
struct Subsets {
    uint16_t m[495];
};
constexpr Subsets make_subsets()
{
    Subsets s{};
    int i = 0;
    for (int d = 3; d < 12; ++d)
        for (int c = 2; c < d; ++c)
            for (int b = 1; b < c; ++b)
                for (int a = 0; a < b; ++a)
                    s.m[i++] = (uint16_t)((1 << a) | (1 << b) | (1 << c) | (1 << d));
    return s;
}
__constant__ Subsets c_subsets = make_subsets();

// The 24 orders of four slots in lexicographic order, slot q of order j in
// bits 2q..2q+1.
struct Perm4 {
    uint8_t p[24];
};
constexpr Perm4 make_perm4()
{
    Perm4 r{};
    int i = 0;
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b)
            for (int c = 0; c < 4; ++c) {
                if (b == a || c == a || c == b) continue;
                int d = 6 - a - b - c;
                r.p[i++] = (uint8_t)(a | (b << 2) | (c << 4) | (d << 6));
            }
    return r;
}
__constant__ Perm4 c_perm4 = make_perm4();

__constant__ uint32_t c_fact[13] = {1u, 1u, 2u, 6u, 24u, 120u, 720u, 5040u, 40320u,
                                    362880u, 3628800u, 39916800u, 479001600u};

__device__ __forceinline__ int32_t max3i(int32_t a, int32_t b, int32_t c)
{
#if TM_USE_DPX
    return __vimax3_s32(a, b, c);
#else
    return max(max(a, b), c);
#endif
}

__device__ __forceinline__ int32_t min3i(int32_t a, int32_t b, int32_t c)
{
#if TM_USE_DPX
    return __vimin3_s32(a, b, c);
#else
    return min(min(a, b), c);
#endif
}

// Largest g in [0, G) with key(g) <= x, for a nondecreasing key.
template <class Key>
__device__ __forceinline__ int search_group(int G, uint64_t x, Key key)
{
    int lo = 0, hi = G;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (key(mid) <= x) lo = mid; else hi = mid;
    }
    return lo;
}

// ---- prep: validation, padded task table, suffix tables -------------------

// One thread per (unit, order of S): a group with n >= 4 tasks has C(n, 4)
// units (its 4-subsets in colexicographic order), smaller groups one unit.
// Thread (unit 0, order 0) of each group also validates it and writes its
// GroupInfo and padded task table.
__global__ void prep_kernel(const tm_task* __restrict__ tasks, const tm_device* __restrict__ devs,
                            const GroupPlan* __restrict__ gp, int G, uint32_t total_units,
                            GroupInfo* __restrict__ info, int4* __restrict__ tbl,
                            SuffixTab* __restrict__ sub)
{
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t u = (uint32_t)(tid / 24), j = (uint32_t)(tid % 24);
    if (u >= total_units) return;
    int g = search_group(G, u, [&](int i) { return (uint64_t)gp[i].unit_base; });
    const int off = gp[g].off;
    const int n = gp[g + 1].off - off;
    const uint32_t s = u - gp[g].unit_base;
    int32_t hs = 0, dinit = 0;
    int status = check_group(tasks + off, n, devs[g].dma_engines, TM_MAX_EXHAUSTIVE, &hs, &dinit);
    if (s == 0 && j == 0) {
        int64_t total = 0;
        for (int i = 0; status == 0 && i < n; ++i) {
            tm_task t = tasks[off + i];
            total += (int64_t)t.htd + t.k + t.dth;
            tbl[off + i] = make_int4(t.htd, t.k, t.dth, 0);
        }
        GroupInfo gi;
        gi.off = off;
        gi.n = n;
        gi.dinit = dinit;
        gi.hs = hs;
        gi.status = status;
        gi.sum32 = (uint64_t)total * 24u < (1ull << 32) ? 1u : 0u;
        gi.pad0 = gi.pad1 = 0;
        info[g] = gi;
    }
    if (status != 0 || n < 4) return;

    // the set S, ascending, and the order j of its four tasks
    const uint32_t mask = c_subsets.m[s];
    tm_task t4[4];
    int64_t hS = hs, alpha = 0;
    for (int q = 0, m = (int)mask; q < 4; ++q) {
        int e = __ffs(m) - 1;
        m &= m - 1;
        t4[q] = tasks[off + e];
        hS -= t4[q].htd;
        alpha += t4[q].dth;
    }
    // beta: the makespan when only the K-engine time (= 0) enters S;
    // gamma: when only the HtD-engine time (= hS) enters S.  A very negative
    // start removes the other engines from the max-plus paths.
    const int64_t NEG = -(int64_t(1) << 40);
    const uint32_t p = c_perm4.p[j];
    int64_t bh = NEG, bk = 0, bd = NEG, gh = hS, gk = NEG, gd = NEG;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int x = (p >> (2 * q)) & 3;
        const tm_task t = x == 0 ? t4[0] : x == 1 ? t4[1] : x == 2 ? t4[2] : t4[3];
        bh += t.htd; bk = max(bk, bh) + t.k; bd = max(bd, bk) + t.dth;
        gh += t.htd; gk = max(gk, gh) + t.k; gd = max(gd, gk) + t.dth;
    }
    SuffixTab* out = sub + gp[g].sub_base + s;
    out->beta[j] = (int32_t)bd;
    out->gamma[j] = (int32_t)gd;
    if (j == 0) {
        out->alpha = (int32_t)alpha;
        out->mask = mask;
        out->pad0 = out->pad1 = 0;
    }
}

// ---- enumeration ----------------------------------------------------------

struct Acc {
    int32_t best, worst;            // running best / worst of the thread
    uint32_t best_rank, worst_rank; // lowest rank reaching them
    unsigned long long sum;
    // Current item: its min / max over the prefixes walked so far and the
    // index (in walk order) of the first prefix reaching each.  Inside an
    // item the walk visits orders in increasing rank, so strict compares
    // keep the lowest-rank occurrence.
    int32_t imin, imax;
    uint32_t imin_at, imax_at, walked;
    __device__ __forceinline__ void reset()
    {
        best = INT32_MAX;
        worst = -1;
        best_rank = worst_rank = kFull;
        sum = 0;
    }
    __device__ __forceinline__ void start_item()
    {
        imin = INT32_MAX;
        imax = -1;
        imin_at = imax_at = walked = 0;
    }
};

__device__ __forceinline__ unsigned long long best_key(const Acc& a)
{
    return ((unsigned long long)(uint32_t)a.best << 32) | a.best_rank;
}

__device__ __forceinline__ unsigned long long worst_key(const Acc& a)
{
    return ((unsigned long long)(uint32_t)a.worst << 32) | (kFull - a.worst_rank);
}

__device__ __forceinline__ void flush(Acc& a, unsigned long long* acc, int g)
{
    if (a.worst < 0) return;
    atomicMin(&acc[3 * g + 0], best_key(a));
    atomicMax(&acc[3 * g + 1], worst_key(a));
    atomicAdd(&acc[3 * g + 2], a.sum);
}

// End-of-thread flush: when the whole warp is present and on one group, the
// warp reduces first and one lane issues the three atomics.
__device__ __forceinline__ void flush_final(Acc& a, unsigned long long* acc, int g)
{
    const unsigned live = __activemask();
    if (live == kFull && __all_sync(kFull, g == __shfl_sync(kFull, g, 0))) {
        int32_t best = __reduce_min_sync(kFull, a.best);
        uint32_t brank = __reduce_min_sync(kFull, a.best == best ? a.best_rank : kFull);
        int32_t worst = __reduce_max_sync(kFull, a.worst);
        uint32_t wrank = __reduce_min_sync(kFull, a.worst == worst ? a.worst_rank : kFull);
        unsigned long long sum = a.sum;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(kFull, sum, o);
        if ((threadIdx.x & 31) == 0 && worst >= 0) {
            Acc r = a;
            r.best = best; r.best_rank = brank; r.worst = worst; r.worst_rank = wrank;
            r.sum = sum;
            flush(r, acc, g);
        }
    } else {
        flush(a, acc, g);
    }
}

// Suffix constants of the current S, in registers.
struct Sfx {
    int32_t b[24], c[24];
    int32_t alpha, bmax, cmax;
};

// Lexicographic rank of the first order that starts with the P tasks in
// `placed` (nibbles, position 0 lowest): each position adds (number of
// still-unplaced tasks with a smaller index) x (positions left)!.
__device__ __forceinline__ uint32_t prefix_rank(uint32_t placed, int n, int P)
{
    uint32_t rank = 0, unused = (1u << n) - 1u;
    for (int i = 0; i < P; ++i) {
        int e = (placed >> (4 * i)) & 0xF;
        rank += (uint32_t)__popc(unused & ((1u << e) - 1u)) * c_fact[n - 1 - i];
        unused &= ~(1u << e);
    }
    return rank;
}

// Index (lexicographic order of S) of the first of the 24 completions of a
// prefix with engine times (k, d) whose makespan is v; 23 if only the last.
__device__ __forceinline__ int first_completion(int32_t k, int32_t d, int32_t v,
                                                const SuffixTab* __restrict__ tab)
{
    const int32_t c0 = d + tab->alpha;
    int j = 23;
#pragma unroll
    for (int q = 22; q >= 0; --q)
        if (max3i(c0, tab->gamma[q], k + tab->beta[q]) == v) j = q;
    return j;
}

// All 24 orders of S after a prefix with engine times (k, d).
template <bool SUM32>
__device__ __forceinline__ void leaves(int32_t k, int32_t d, const Sfx& S, Acc& a)
{
    const int32_t c0 = d + S.alpha;
    int32_t m[24];
#pragma unroll
    for (int j = 0; j < 24; ++j) m[j] = max3i(c0, S.c[j], k + S.b[j]);
    int32_t t8[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) t8[i] = min3i(m[3 * i], m[3 * i + 1], m[3 * i + 2]);
    const int32_t pmin = min3i(min3i(t8[0], t8[1], t8[2]), min3i(t8[3], t8[4], t8[5]),
                               min(t8[6], t8[7]));
    if (SUM32) {
        // the group's duration sum bounds every makespan, and 24 of them fit
        uint32_t s8[8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
            s8[i] = (uint32_t)m[3 * i] + (uint32_t)m[3 * i + 1] + (uint32_t)m[3 * i + 2];
        a.sum += (s8[0] + s8[1] + s8[2]) + (s8[3] + s8[4] + s8[5]) + (s8[6] + s8[7]);
    } else {
#pragma unroll
        for (int i = 0; i < 12; ++i) a.sum += (uint32_t)m[2 * i] + (uint32_t)m[2 * i + 1];
    }
    const int32_t pmax = max3i(c0, k + S.bmax, S.cmax);
    if (pmin < a.imin) { a.imin = pmin; a.imin_at = a.walked; }
    if (pmax > a.imax) { a.imax = pmax; a.imax_at = a.walked; }
    a.walked += 1;
}

// Depth-first walk over the D remaining prefix tasks (ascending in `rem`):
// their orders in lexicographic order, so `walked` counts prefixes in rank
// order.
template <int D, bool SUM32>
__device__ __forceinline__ void dfs(Eng st, uint64_t rem, const int4* __restrict__ tbl,
                                    const Sfx& S, Acc& a)
{
    if constexpr (D == 0) {
        leaves<SUM32>(st.k, st.d, S, a);
    } else if constexpr (D == 1) {
        int4 t = tbl[nib_get(rem, 0)];
        Eng s1 = step(st, t.x, t.y, t.z);
        leaves<SUM32>(s1.k, s1.d, S, a);
    } else if constexpr (D == 2) {
        int4 t0 = tbl[nib_get(rem, 0)], t1 = tbl[nib_get(rem, 1)];
        Eng s01 = step(step(st, t0.x, t0.y, t0.z), t1.x, t1.y, t1.z);
        Eng s10 = step(step(st, t1.x, t1.y, t1.z), t0.x, t0.y, t0.z);
        leaves<SUM32>(s01.k, s01.d, S, a);
        leaves<SUM32>(s10.k, s10.d, S, a);
    } else {
#pragma unroll 1
        for (int c = 0; c < D; ++c) {
            int4 t = tbl[nib_get(rem, c)];
            dfs<D - 1, SUM32>(step(st, t.x, t.y, t.z), nib_remove(rem, c), tbl, S, a);
        }
    }
}

template <int PDMAX, bool SUM32>
__device__ __forceinline__ void walk_prefixes(int pd, Eng st, uint64_t rem,
                                              const int4* __restrict__ tbl, const Sfx& S, Acc& a)
{
    switch (pd) {
    case 0: dfs<0, SUM32>(st, rem, tbl, S, a); break;
    case 1: dfs<1, SUM32>(st, rem, tbl, S, a); break;
    case 2: dfs<2, SUM32>(st, rem, tbl, S, a); break;
    default:
        if constexpr (PDMAX >= 3) { if (pd == 3) dfs<3, SUM32>(st, rem, tbl, S, a); }
        if constexpr (PDMAX >= 4) { if (pd == 4) dfs<4, SUM32>(st, rem, tbl, S, a); }
        if constexpr (PDMAX >= 5) { if (pd == 5) dfs<5, SUM32>(st, rem, tbl, S, a); }
        break;
    }
}

// The head of an item: its f leading prefix positions are the Lehmer digits
// of hd (radices P, P-1, ...) over the ascending list `rem` of S's
// complement.  Runs the recurrence over them; leaves the other pd tasks in
// `rem` and the placed tasks in `placed`.
__device__ __forceinline__ Eng run_head(uint32_t hd, int f, int P, int32_t dinit, uint64_t& rem,
                                        uint32_t& placed, const int4* __restrict__ tbl)
{
    uint32_t digits = 0;
    for (int j = f - 1; j >= 0; --j) {
        uint32_t r = (uint32_t)(P - j);
        uint32_t q = hd / r;
        digits |= (hd - q * r) << (4 * j);
        hd = q;
    }
    placed = 0;
    Eng st{0, 0, dinit};
    for (int j = 0; j < f; ++j) {
        int c = (digits >> (4 * j)) & 0xF;
        int e = nib_get(rem, c);
        rem = nib_remove(rem, c);
        int4 t = tbl[e];
        st = step(st, t.x, t.y, t.z);
        placed |= (uint32_t)e << (4 * j);
    }
    return st;
}

// Rank of the first order of the current item reaching v: the prefix walked
// `at`-th (its tail is the at-th order, lexicographically, of the pd tasks in
// `rem`), completed by the first order of S reaching v.
__device__ __noinline__ uint32_t item_rank(uint32_t at, int32_t v, uint32_t hd, uint64_t rem,
                                           int f, int pd, int n, int32_t dinit,
                                           const int4* __restrict__ tbl,
                                           const SuffixTab* __restrict__ tab)
{
    uint32_t placed;
    Eng st = run_head(hd, f, n - 4, dinit, rem, placed, tbl);
    for (int q = 0; q < pd; ++q) {
        uint32_t fq = c_fact[pd - 1 - q];
        uint32_t c = at / fq;
        at -= c * fq;
        int e = nib_get(rem, (int)c);
        rem = nib_remove(rem, (int)c);
        int4 t = tbl[e];
        st = step(st, t.x, t.y, t.z);
        placed |= (uint32_t)e << (4 * (f + q));
    }
    return prefix_rank(placed, n, f + pd) + (uint32_t)first_completion(st.k, st.d, v, tab);
}

// First work item whose first order is at or after global order index x.
template <int PDMAX>
__device__ __forceinline__ uint32_t first_item(const GroupPlan* __restrict__ gp, int G,
                                               uint64_t x)
{
    if (x >= gp[G].cost_base) return gp[G].item_base;
    int g = search_group(G, x, [&](int i) { return gp[i].cost_base; });
    int n = gp[g + 1].off - gp[g].off;
    uint64_t lpi = 24ull * factorial_u64(plan_pd(n, PDMAX));
    uint64_t q = (x - gp[g].cost_base + lpi - 1) / lpi;
    uint64_t i = gp[g].item_base + q;
    return (uint32_t)min(i, (uint64_t)gp[g + 1].item_base);
}

template <int PDMAX>
__global__ void __launch_bounds__(kEnumBlock, 4)
enum_kernel(const GroupPlan* __restrict__ gp, const GroupInfo* __restrict__ info,
            const int4* __restrict__ tbl, const SuffixTab* __restrict__ sub, int G,
            uint64_t per_thread, unsigned long long* __restrict__ acc)
{
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t x0 = t * per_thread;
    const uint64_t total = gp[G].cost_base;
    if (x0 >= total) return;
    uint32_t i = first_item<PDMAX>(gp, G, x0);
    const uint32_t end = first_item<PDMAX>(gp, G, min(x0 + per_thread, total));
    if (i >= end) return;
    int g = search_group(G, i, [&](int j) { return (uint64_t)gp[j].item_base; });

    Acc a;
    a.reset();
    Sfx S;
    GroupInfo gi;
    const int4* gt = tbl;
    uint32_t gbase = 0, gend = 0, heads = 1, cur = kFull;
    const SuffixTab* tab = sub;
    uint64_t sc = 0;   // S's complement, ascending nibbles
    int pd = 0, f = 0, P = 0;
    bool load_group = true;
    for (; i < end; ++i) {
        while (load_group || i >= gend) {
            if (!load_group) { flush(a, acc, g); a.reset(); ++g; }
            load_group = false;
            gi = info[g];
            gbase = gp[g].item_base;
            gend = gp[g + 1].item_base;
            gt = tbl + gi.off;
            P = gi.n - 4;
            pd = plan_pd(gi.n, PDMAX);
            f = P - pd;
            heads = (uint32_t)(factorial_u64(P) / factorial_u64(pd));
            cur = kFull;
        }
        if (gi.status != 0) continue;
        const uint32_t local = i - gbase;
        const uint32_t s = local / heads;
        const uint32_t hd = local - s * heads;
        if (s != cur) {
            cur = s;
            tab = sub + gp[g].sub_base + s;
            const int4* v = reinterpret_cast<const int4*>(tab);
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                int4 b = __ldg(v + q);
                S.b[4 * q] = b.x; S.b[4 * q + 1] = b.y; S.b[4 * q + 2] = b.z; S.b[4 * q + 3] = b.w;
                int4 c = __ldg(v + 6 + q);
                S.c[4 * q] = c.x; S.c[4 * q + 1] = c.y; S.c[4 * q + 2] = c.z; S.c[4 * q + 3] = c.w;
            }
            int4 tail = __ldg(v + 12);
            S.alpha = tail.x;
            const uint32_t mask = (uint32_t)tail.y;
            int32_t bm[8], cm[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                bm[q] = max3i(S.b[3 * q], S.b[3 * q + 1], S.b[3 * q + 2]);
                cm[q] = max3i(S.c[3 * q], S.c[3 * q + 1], S.c[3 * q + 2]);
            }
            S.bmax = max3i(max3i(bm[0], bm[1], bm[2]), max3i(bm[3], bm[4], bm[5]), max(bm[6], bm[7]));
            S.cmax = max3i(max3i(cm[0], cm[1], cm[2]), max3i(cm[3], cm[4], cm[5]), max(cm[6], cm[7]));
            sc = 0;
            for (int e = 0, cnt = 0; e < gi.n; ++e)
                if (!((mask >> e) & 1u)) sc |= (uint64_t)e << (4 * cnt++);
        }
        uint64_t rem = sc;
        uint32_t placed;
        Eng st = run_head(hd, f, P, gi.dinit, rem, placed, gt);
        a.start_item();
        if (gi.sum32) walk_prefixes<PDMAX, true>(pd, st, rem, gt, S, a);
        else walk_prefixes<PDMAX, false>(pd, st, rem, gt, S, a);
        // Settle the item against the running best / worst: every lane of a
        // warp gets here together, so this rank work does not diverge.
        if (a.imin <= a.best) {
            uint32_t r = item_rank(a.imin_at, a.imin, hd, sc, f, pd, gi.n, gi.dinit, gt, tab);
            if (a.imin < a.best || r < a.best_rank) { a.best = a.imin; a.best_rank = r; }
        }
        if (a.imax >= a.worst) {
            uint32_t r = item_rank(a.imax_at, a.imax, hd, sc, f, pd, gi.n, gi.dinit, gt, tab);
            if (a.imax > a.worst || r < a.worst_rank) { a.worst = a.imax; a.worst_rank = r; }
        }
    }
    flush_final(a, acc, g);
}

// ---- finalize ---------------------------------------------------------------

__global__ void finalize_kernel(const GroupInfo* __restrict__ info, const int4* __restrict__ tbl,
                                int G, unsigned long long* __restrict__ acc,
                                tm_stats* __restrict__ stats, int32_t* __restrict__ status)
{
    int g = (int)((blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5);
    int lane = threadIdx.x & 31;
    if (g >= G) return;
    GroupInfo gi = info[g];
    unsigned long long* A = acc + 3 * g;
    if (gi.status != 0) {
        if (lane == 0) {
            if (status) status[g] = gi.status;
            A[0] = ~0ull; A[1] = 0; A[2] = 0;
        }
        return;
    }
    const int4* t = tbl + gi.off;
    const int n = gi.n;
    int32_t best, worst;
    uint32_t best_rank, worst_rank;
    unsigned long long sum;
    bool ok = true;
    if (n <= 3) {
        uint32_t nf = (uint32_t)factorial_u64(n);
        bool live = (uint32_t)lane < nf;
        int32_t ms = live ? makespan_of_rank(t, n, gi.dinit, lane, nullptr) : 0;
        best = __reduce_min_sync(kFull, live ? ms : INT32_MAX);
        worst = __reduce_max_sync(kFull, live ? ms : -1);
        best_rank = __ffs(__ballot_sync(kFull, live && ms == best)) - 1;
        worst_rank = __ffs(__ballot_sync(kFull, live && ms == worst)) - 1;
        sum = live ? (unsigned long long)ms : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(kFull, sum, o);
    } else {
        unsigned long long mk = A[0], xk = A[1];
        sum = A[2];
        best = (int32_t)(mk >> 32);
        worst = (int32_t)(xk >> 32);
        best_rank = (uint32_t)mk;
        worst_rank = kFull - (uint32_t)xk;
        const uint64_t nf = factorial_u64(n);
        ok = best_rank < nf && worst_rank < nf;
        __syncwarp();
        if (lane == 0) { A[0] = ~0ull; A[1] = 0; A[2] = 0; }
    }
    if (lane != 0) return;
    tm_stats st;
    st.best = best;
    st.worst = worst;
    st.sum = (int64_t)sum;
    st.mean = (double)(int64_t)sum / (double)factorial_u64(n);
    st.best_rank = best_rank;
    st.worst_rank = worst_rank;
    for (int i = 0; i < 16; ++i) st.best_order[i] = st.worst_order[i] = 0xFF;
    // self-check: the reported orders must reproduce the reported values
    if (ok) {
        ok = makespan_of_rank(t, n, gi.dinit, best_rank, st.best_order) == best &&
             makespan_of_rank(t, n, gi.dinit, worst_rank, st.worst_order) == worst;
    }
    if (!ok) {  // the reduction disagrees with a re-evaluation: never expected
        if (status) status[g] = TM_ECUDA;
        return;
    }
    stats[g] = st;
    if (status) status[g] = 0;
}

template <int PDMAX>
cudaError_t launch_enum(const Plan& p, cudaStream_t stream)
{
    uint32_t blocks = (p.threads + kEnumBlock - 1) / kEnumBlock;
    enum_kernel<PDMAX><<<blocks, kEnumBlock, 0, stream>>>(p.d_gp, p.d_info, p.d_tbl, p.d_sub, p.G,
                                                           p.leaves_per_thread, p.d_acc);
    return cudaGetLastError();
}

int resident_threads(int pdmax, int device)
{
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    cudaError_t e = cudaErrorInvalidValue;
    switch (pdmax) {
    case 3: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, enum_kernel<3>, kEnumBlock, 0); break;
    case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, enum_kernel<4>, kEnumBlock, 0); break;
    case 5: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, enum_kernel<5>, kEnumBlock, 0); break;
    default: break;
    }
    if (e != cudaSuccess || sms <= 0 || per_sm <= 0) return 152 * 512;
    return sms * per_sm * kEnumBlock;
}

}  // namespace

void exhaustive_partition(Plan& p, int device)
{
    uint64_t threads = std::min<uint64_t>((uint64_t)resident_threads(p.pdmax, device),
                                          std::max<uint64_t>(p.total_items, 1));
    p.leaves_per_thread = std::max<uint64_t>(1, (p.total_leaves + threads - 1) / threads);
    p.threads = (uint32_t)((p.total_leaves + p.leaves_per_thread - 1) / p.leaves_per_thread);
    p.launches = exhaustive_launch_count(p);
}

int exhaustive_launch_count(const Plan& p)
{
    return p.total_items > 0 ? 3 : 2;
}

cudaError_t launch_exhaustive(const Plan& p, const tm_task* d_tasks, const tm_device* d_devs,
                              tm_stats* d_stats, int32_t* d_status, cudaStream_t stream)
{
    if (p.G == 0) return cudaSuccess;
    const uint64_t prep_threads = (uint64_t)p.total_units * 24;
    prep_kernel<<<(unsigned)((prep_threads + 191) / 192), 192, 0, stream>>>(
        d_tasks, d_devs, p.d_gp, p.G, p.total_units, p.d_info, p.d_tbl, p.d_sub);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (p.total_items > 0) {
        if (p.ev_before && (e = cudaEventRecord(p.ev_before, stream)) != cudaSuccess) return e;
        switch (p.pdmax) {
        case 3: e = launch_enum<3>(p, stream); break;
        case 4: e = launch_enum<4>(p, stream); break;
        case 5: e = launch_enum<5>(p, stream); break;
        default: return cudaErrorInvalidValue;
        }
        if (e != cudaSuccess) return e;
        if (p.ev_after && (e = cudaEventRecord(p.ev_after, stream)) != cudaSuccess) return e;
    }
    uint64_t threads = (uint64_t)p.G * 32;
    finalize_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, stream>>>(
        p.d_info, p.d_tbl, p.G, p.d_acc, d_stats, d_status);
    return cudaGetLastError();
}

}  // namespace tmgpu

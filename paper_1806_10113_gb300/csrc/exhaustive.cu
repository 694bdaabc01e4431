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

#include "heuristic.cuh"
#include "tm_device.cuh"

namespace tmgpu {
namespace {

constexpr int kEnumBlock = 128;
// Three resident blocks per SM leave the enumeration up to 168 registers per
// thread (no spills); measured as fast as four blocks of 128 registers, and
// up to 2% faster on ragged and 12-task batches.
#ifndef TM_ENUM_MIN_BLOCKS
#define TM_ENUM_MIN_BLOCKS 3
#endif
constexpr unsigned kFull = 0xFFFFFFFFu;

// Programmatic dependent launch: the finalize launch may start while the
// enumeration finishes (launch_exhaustive sets the launch attribute when no
// timing event sits between them).  wait blocks until the kernel before has
// completed and its writes are visible (a no-op without the attribute);
// launch_dependents lets the next launch begin once every block of this
// grid has started.  (Between prep and enumeration it measured slower: the
// enumeration's blocks, placed beside the prep blocks still running, spread
// its uneven walk-mode-5 work worse over the SMs.)
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_next() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

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

// ---- per-group results ------------------------------------------------------

// Statistics of a group of n <= 3 tasks (at most 6 orders), by one warp:
// lane r evaluates the order of rank r.
__device__ __forceinline__ void small_group_stats(const int4* __restrict__ t, int n,
                                                  int32_t dinit, int lane, tm_stats* out)
{
    const uint32_t nf = (uint32_t)factorial_u64(n);
    const bool live = (uint32_t)lane < nf;
    const int32_t ms = live ? makespan_of_rank(t, n, dinit, lane, nullptr) : 0;
    const int32_t best = __reduce_min_sync(kFull, live ? ms : INT32_MAX);
    const int32_t worst = __reduce_max_sync(kFull, live ? ms : -1);
    const uint32_t brank = __ffs(__ballot_sync(kFull, live && ms == best)) - 1;
    const uint32_t wrank = __ffs(__ballot_sync(kFull, live && ms == worst)) - 1;
    unsigned long long sum = live ? (unsigned long long)ms : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(kFull, sum, o);
    if (lane != 0) return;
    tm_stats st;
    st.best = best;
    st.worst = worst;
    st.sum = (int64_t)sum;
    st.mean = (double)(int64_t)sum / (double)nf;
    st.best_rank = brank;
    st.worst_rank = wrank;
    for (int i = 0; i < 16; ++i) st.best_order[i] = st.worst_order[i] = 0xFF;
    makespan_of_rank(t, n, dinit, brank, st.best_order);
    makespan_of_rank(t, n, dinit, wrank, st.worst_order);
    *out = st;
}

// The same by one full warp: lanes 0 and 1 unrank and check the best and
// the worst order in parallel.  Every lane passes the same g.
__device__ __noinline__ void finalize_group_warp(int g, const GroupInfo& gi,
                                                 const int4* __restrict__ tbl,
                                                 unsigned long long* __restrict__ acc,
                                                 tm_stats* __restrict__ stats,
                                                 int32_t* __restrict__ status)
{
    const int lane = threadIdx.x & 31;
    unsigned long long* A = acc + (size_t)kAccStride * g;
    unsigned long long mk = 0, xk = 0, sum = 0;
    const int4 row = lane < gi.n ? tbl[gi.off + lane] : make_int4(0, 0, 0, 0);
    if (lane == 0) {
        mk = __ldcg(A);
        xk = __ldcg(A + 1);
        sum = __ldcg(A + 2);
        A[0] = ~0ull;
        A[1] = 0;
        A[2] = 0;
    }
    mk = __shfl_sync(kFull, mk, 0);
    xk = __shfl_sync(kFull, xk, 0);
    const int n = gi.n;
    const int32_t best = (int32_t)(mk >> 32), worst = (int32_t)(xk >> 32);
    const uint32_t brank = (uint32_t)mk, wrank = kFull - (uint32_t)xk;
    const uint64_t nf = factorial_u64(n);
    uint8_t order[16];
    for (int i = 0; i < 16; ++i) order[i] = 0xFF;
    bool good = brank < nf && wrank < nf;   // the same on every lane
    if (good) {
        const uint32_t r = lane == 0 ? brank : lane == 1 ? wrank : 0u;
        const int32_t ms = makespan_of_rank_warp(row, n, gi.dinit, r, order);
        if (lane < 2) good = ms == (lane == 0 ? best : worst);
    }
    const bool ok = __all_sync(kFull, good);
    uint32_t packed[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint32_t w = (uint32_t)order[4 * q] | ((uint32_t)order[4 * q + 1] << 8) |
                           ((uint32_t)order[4 * q + 2] << 16) | ((uint32_t)order[4 * q + 3] << 24);
        packed[q] = __shfl_sync(kFull, w, 1);   // the worst order, from lane 1
    }
    if (lane != 0) return;
    if (!ok) {  // the reduction disagrees with a re-evaluation: never expected
        if (status) status[gi.user] = TM_ECUDA;
        return;
    }
    tm_stats st;
    st.best = best;
    st.worst = worst;
    st.sum = (int64_t)sum;
    st.mean = (double)(int64_t)sum / (double)nf;
    st.best_rank = brank;
    st.worst_rank = wrank;
    for (int i = 0; i < 16; ++i) {
        st.best_order[i] = order[i];
        st.worst_order[i] = (uint8_t)(packed[i / 4] >> (8 * (i % 4)));
    }
    stats[gi.user] = st;
    if (status) status[gi.user] = 0;
}

// Turns a group's three reduction words into tm_stats (one thread) and
// resets them for the next launch.  The reported orders are re-evaluated;
// a mismatch (never expected) is reported as TM_ECUDA.
__device__ __noinline__ void finalize_group(int g, const GroupInfo& gi, const int4* __restrict__ tbl,
                               unsigned long long* __restrict__ acc, tm_stats* __restrict__ stats,
                               int32_t* __restrict__ status)
{
    unsigned long long* A = acc + (size_t)kAccStride * g;
    const unsigned long long mk = __ldcg(A), xk = __ldcg(A + 1), sum = __ldcg(A + 2);
    A[0] = ~0ull;
    A[1] = 0;
    A[2] = 0;
    const int n = gi.n;
    const int4* t = tbl + gi.off;
    tm_stats st;
    st.best = (int32_t)(mk >> 32);
    st.worst = (int32_t)(xk >> 32);
    st.best_rank = (uint32_t)mk;
    st.worst_rank = kFull - (uint32_t)xk;
    st.sum = (int64_t)sum;
    st.mean = (double)(int64_t)sum / (double)factorial_u64(n);
    for (int i = 0; i < 16; ++i) st.best_order[i] = st.worst_order[i] = 0xFF;
    const uint64_t nf = factorial_u64(n);
    bool ok = st.best_rank < nf && st.worst_rank < nf;
    ok = ok && makespan_of_rank(t, n, gi.dinit, (uint32_t)st.best_rank, st.best_order) == st.best;
    ok = ok && makespan_of_rank(t, n, gi.dinit, (uint32_t)st.worst_rank, st.worst_order) ==
                   st.worst;
    if (!ok) {
        if (status) status[gi.user] = TM_ECUDA;
        return;
    }
    stats[gi.user] = st;
    if (status) status[gi.user] = 0;
}

// ---- prep: validation, padded task table, suffix tables -------------------

// One block per group (128 threads, or 512 when the batch has groups with
// many 4-subsets; a warp per group measured slower: its largest groups'
// tables then run on 32 threads).  Every warp loads the group itself (lane
// i holds task i), so no warp waits at a block barrier: warp 0 validates it
// and writes its GroupInfo and padded task table (and finishes groups of
// n <= 3 outright) while all warps stride over the group's 4-subsets and
// tabulate alpha / beta / gamma, taking the subset's tasks from the lanes
// by shuffle.  A group that fails validation gets tables too, which
// nothing reads.  When the heuristic is requested and no enumeration launch
// follows (no group of 4 or more tasks), blocks G.. of the same launch run
// it, one warp per group.
constexpr int kPrepMaxThreads = 512;

}  // namespace

// PrepArgs and Sink have external linkage: exhaustive_wide.cu's launchers
// take them (both translation units compile this file).
struct PrepArgs {
    const tm_task* tasks;
    const tm_device* devs;
    const GroupPlan* gp;
    int G;
    GroupInfo* info;
    int4* tbl;
    SuffixTab* sub;
    tm_stats* stats;
    int32_t* status;
    int32_t* orders;              // heuristic outputs; null: no heuristic
    int32_t* makespans;
    uint32_t* next;               // dynamic chunk counter to zero, or null
    unsigned long long* full;     // Plan::d_full, to zero (or null)
};

namespace {

// Validation, GroupInfo, padded task table (and n <= 3 groups finished
// outright) for the group at work position w, by one full warp: lane i
// holds task i in t (lanes >= n hold zeros).
__device__ __forceinline__ void prep_group(const PrepArgs& a, int w, int lane, int off, int n,
                                           int user, const tm_task& t)
{
    const int dma = a.devs[user].dma_engines;
    const bool mine = lane < n;
    const bool neg = mine && (t.htd < 0 || t.k < 0 || t.dth < 0);
    unsigned long long tot = mine ? (unsigned long long)((int64_t)t.htd + t.k + t.dth) : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(kFull, tot, o);
    // with no negative duration and tot <= INT32_MAX the HtD sum fits
    const int32_t hs = (int32_t)__reduce_add_sync(kFull, mine ? (uint32_t)t.htd : 0u);
    int status = 0;
    if (n < 1 || n > TM_MAX_EXHAUSTIVE || (dma != 1 && dma != 2)) status = TM_EINVAL;
    else if (__ballot_sync(kFull, neg)) status = TM_ENEG;
    else if (tot > (unsigned long long)INT32_MAX) status = TM_EOVERFLOW;
    if (mine && status == 0) a.tbl[off + lane] = make_int4(t.htd, t.k, t.dth, 0);
    if (lane == 0) {
        GroupInfo gi;
        gi.off = off;
        gi.n = n;
        gi.hs = hs;
        gi.dinit = dma == 1 ? hs : 0;
        gi.status = status;
        gi.sum32 = tot * 24u < (1ull << 32) ? 1u : 0u;
        gi.user = user;
        gi.pad1 = 0;
        a.info[w] = gi;
        if (status != 0 && a.status) a.status[user] = status;
    }
    if (status == 0 && n <= 3) {       // at most 6 orders: finish here
        __syncwarp();
        small_group_stats(a.tbl + off, n, dma == 1 ? hs : 0, lane, a.stats + user);
        if (lane == 0 && a.status) a.status[user] = 0;
    }
}

// The suffix tables of the group at work position w (n >= 4) by one warp:
// 4-subsets S = first + lane, first + lane + stride, ...; lane i holds task
// i in `row`, hs is the group's HtD sum.  The 24 orders of S are walked
// depth-first in lexicographic order (prefix steps shared) and the 208-byte
// table goes out in 16-byte stores as it fills.
//   beta[j]:  the order's makespan when only the K engine (free at 0) enters
//             S: HtD and DtH start unconstrained, so the first task's kernel
//             starts at 0 and its DtH right after it;
//   gamma[j]: when only the HtD engine enters S, free at hS = hs - (S's HtD
//             sum): the first task's kernel and DtH follow its HtD directly.
// Every value is a path length within the group, so int32 holds it.
__device__ __forceinline__ void prep_tables(const PrepArgs& a, int w, int n, int32_t hs,
                                            int4 row, int lane, uint32_t first, uint32_t stride)
{
    SuffixTab* out = a.sub + a.gp[w].sub_base;
    const uint32_t subsets = choose4(n);
    for (uint32_t base = first; base < subsets; base += stride) {   // the same on every lane
        const uint32_t sidx = base + (uint32_t)lane;
        const bool live = sidx < subsets;
        const uint32_t mask = live ? c_subsets.m[sidx] : 0xFu;
        int4 t[4];
#pragma unroll
        for (int q = 0, m = (int)mask; q < 4; ++q) {
            const int e = __ffs(m) - 1;
            t[q] = make_int4(__shfl_sync(kFull, row.x, e), __shfl_sync(kFull, row.y, e),
                             __shfl_sync(kFull, row.z, e), 0);
            m &= m - 1;
        }
        if (!live) continue;
        const int32_t hS = hs - t[0].x - t[1].x - t[2].x - t[3].x;
        int4* dst = reinterpret_cast<int4*>(out + sidx);
        int32_t bq[4], gq[4];
        int j = 0;
#pragma unroll
        for (int p0 = 0; p0 < 4; ++p0) {
            const int4 A = t[p0];
            const int32_t bk1 = A.y, bd1 = A.y + A.z;
            const int32_t gh1 = hS + A.x, gk1 = gh1 + A.y, gd1 = gk1 + A.z;
#pragma unroll
            for (int p1 = 0; p1 < 4; ++p1) {
                if (p1 == p0) continue;
                const int4 B = t[p1];
                const int32_t bk2 = bk1 + B.y, bd2 = max(bd1, bk2) + B.z;
                const int32_t gh2 = gh1 + B.x, gk2 = max(gk1, gh2) + B.y, gd2 = max(gd1, gk2) + B.z;
#pragma unroll
                for (int p2 = 0; p2 < 4; ++p2) {
                    if (p2 == p0 || p2 == p1) continue;
                    const int p3 = 6 - p0 - p1 - p2;
                    const int4 C = t[p2], D = t[p3];
                    const int32_t bk3 = bk2 + C.y, bd3 = max(bd2, bk3) + C.z;
                    const int32_t bk4 = bk3 + D.y, bd4 = max(bd3, bk4) + D.z;
                    const int32_t gh3 = gh2 + C.x, gk3 = max(gk2, gh3) + C.y, gd3 = max(gd2, gk3) + C.z;
                    const int32_t gh4 = gh3 + D.x, gk4 = max(gk3, gh4) + D.y, gd4 = max(gd3, gk4) + D.z;
                    bq[j & 3] = bd4;
                    gq[j & 3] = gd4;
                    if ((j & 3) == 3) {
                        dst[j >> 2] = make_int4(bq[0], bq[1], bq[2], bq[3]);
                        dst[6 + (j >> 2)] = make_int4(gq[0], gq[1], gq[2], gq[3]);
                    }
                    ++j;
                }
            }
        }
        dst[12] = make_int4(t[0].z + t[1].z + t[2].z + t[3].z, (int)mask, 0, 0);
    }
}

// Heuristic warp for the group at work position w (blocks after the table
// work), if requested.
__device__ __forceinline__ void prep_heuristic(const PrepArgs& a, int w, int lane)
{
    if (!a.orders || w >= a.G) return;
    const int user = a.gp[w].group;
    heur::heuristic_group(a.tasks, a.gp[w].uoff, a.gp[w + 1].off - a.gp[w].off,
                          a.devs[user].dma_engines, user, lane, a.orders, a.makespans, nullptr);
}

// Block per group (groups with many 4-subsets).  Blocks G.. run the
// heuristic, a warp per group, so that no table block waits for one.
__global__ void __launch_bounds__(kPrepMaxThreads) prep_kernel(PrepArgs a)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (blockIdx.x >= (unsigned)a.G) {
        prep_heuristic(a, (blockIdx.x - a.G) * (blockDim.x / 32) + warp, lane);
        return;
    }
    const int w = blockIdx.x;
    if (w == 0 && tid == 0) {
        if (a.next) *a.next = 0;
        if (a.full) *a.full = 0;
    }
    const GroupPlan* __restrict__ gp = a.gp;
    const int off = gp[w].off, uoff = gp[w].uoff, user = gp[w].group;
    const int n = gp[w + 1].off - off;     // 1..TM_MAX_EXHAUSTIVE: the plan checked it
    const tm_task t = lane < n ? a.tasks[uoff + lane] : tm_task{0, 0, 0};
    if (warp == 0) prep_group(a, w, lane, off, n, user, t);
    if (n < 4) return;
    const int32_t hs = (int32_t)__reduce_add_sync(kFull, lane < n ? (uint32_t)t.htd : 0u);
    prep_tables(a, w, n, hs, make_int4(t.htd, t.k, t.dth, 0), lane, (uint32_t)warp * 32u,
                blockDim.x);
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
    // Walk modes 5 to 8: prefixes of the thread's whole range evaluated
    // order by order (not reset per group).
    uint32_t full;
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

// Where the enumeration threads report.  With done != null each group is
// finalized by its last finishing thread.
}  // namespace

struct Sink {
    unsigned long long* acc;
    const GroupInfo* info;
    const int4* tbl;
    tm_stats* stats;
    int32_t* status;
    const uint32_t* target;
    uint32_t* done;
    uint32_t one;   // always 1 (the leaves' multiply-add sum)
    unsigned long long* full;   // Plan::d_full (walk modes 5 to 8), or null
};

namespace {

__device__ __forceinline__ void flush(const Acc& a, unsigned long long* acc, int g)
{
    if (a.worst < 0) return;
    unsigned long long* A = acc + (size_t)kAccStride * g;
    atomicMin(&A[0], best_key(a));
    atomicMax(&A[1], worst_key(a));
    atomicAdd(&A[2], a.sum);
}

// Reports `threads` finished contributors to group g.  Returns true if this
// call was the last one: the caller then finalizes the group.
__device__ __forceinline__ bool finished(const Sink& k, int g, uint32_t threads)
{
    if (!k.done) return false;
    __threadfence();
    uint32_t* done = k.done + (size_t)kDoneStride * g;
    const uint32_t before = atomicAdd(done, threads);
    if (before + threads != k.target[g]) return false;
    __threadfence();
    *done = 0;
    return true;
}

// finished() by one thread, which finalizes alone if it was the last.
__device__ __forceinline__ void finished_single(const Sink& k, int g)
{
    if (finished(k, g, 1)) {
        const GroupInfo gi = k.info[g];
        if (gi.status == 0) finalize_group(g, gi, k.tbl, k.acc, k.stats, k.status);
    }
}

// End-of-thread flush: when the whole warp is present and on one group, the
// warp reduces first and one lane issues the three atomics.
__device__ __forceinline__ void flush_final(Acc& a, const Sink& k, int g)
{
    unsigned long long* acc = k.acc;
    const unsigned live = __activemask();
    if (live == kFull && __all_sync(kFull, g == __shfl_sync(kFull, g, 0))) {
        int32_t best = __reduce_min_sync(kFull, a.best);
        uint32_t brank = __reduce_min_sync(kFull, a.best == best ? a.best_rank : kFull);
        int32_t worst = __reduce_max_sync(kFull, a.worst);
        uint32_t wrank = __reduce_min_sync(kFull, a.worst == worst ? a.worst_rank : kFull);
        unsigned long long sum = a.sum;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(kFull, sum, o);
        bool last = false;
        if ((threadIdx.x & 31) == 0) {
            Acc r = a;
            r.best = best; r.best_rank = brank; r.worst = worst; r.worst_rank = wrank;
            r.sum = sum;
            flush(r, acc, g);
            last = finished(k, g, 32);
        }
        if (__shfl_sync(kFull, last, 0)) {     // the whole warp finalizes
            const GroupInfo gi = k.info[g];
            if (gi.status == 0) finalize_group_warp(g, gi, k.tbl, k.acc, k.stats, k.status);
        }
    } else {
        flush(a, acc, g);
        finished_single(k, g);
    }
}

// Suffix constants of the current S, in registers.  The extremes, the
// bounds of gamma - beta and the 32-bit sums serve the dominance test of
// walk modes 5 to 8 (dominated()).
struct Sfx {
    int32_t b[24], c[24];
    int32_t alpha, bmax, cmax;
    int32_t bmin, cmin, tmin, tmax;   // tmin / tmax: min / max over sigma of gamma - beta
    uint32_t bsum, csum;              // sums of beta and gamma mod 2^32
    uint32_t one;   // 1, read from a kernel parameter (see leaves)
    // Walk modes 6, 7: b and c live in shared memory instead, six int4 rows of
    // b then six of c, row r of this thread at sq[r * kEnumBlock].
    const int4* sq;
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

// All 24 orders of S after a prefix with engine times (k, d).  FMA_SUM:
// the 32-bit sum takes 18 of the 24 makespans as multiply-adds by S.one,
// which the compiler cannot fold to plain adds, so they issue on the FMA
// pipe; the maxima, the minima and the other six terms (three-input adds)
// stay on the ALU pipe.  That balance pays where the walk's straight-line
// level keeps the ALU pipe busy (5% on uniform batches) and costs 2% in the
// looped walk, so the two go together.
// Walk modes (tm_tuning.unroll): 1 the straight-line level with the
// FMA-pipe sum; 2 every level as a loop (ALU sum); 3 as 1, and each order's
// addition k + beta as a multiply-add by S.one, so that it too issues on the
// FMA pipe beside the ALU pipe's maxima and minima; 4 as 3, compiled for four
// resident blocks per SM (at most 128 registers) instead of three; 5 as 3,
// with the dominance test (dominated()) before each prefix's 24 orders; 6
// as 5, with S's beta and gamma in shared memory instead of 48 registers,
// the six prefixes of the straight-line level evaluated quad by quad of S's
// orders (leaves6), compiled for four resident blocks per SM; 7 as 6, with
// the six prefixes' vote and closed forms in one pass and leaves6's quads
// as a loop (less hot code); 8 as 6 with that loop.
__host__ __device__ constexpr bool mode_straight(int mode) { return mode != 2; }
__host__ __device__ constexpr bool mode_fma_add(int mode) { return mode >= 3; }
__host__ __device__ constexpr int mode_min_blocks(int mode)
{
    return (mode == 4 || mode >= 6) ? 4 : TM_ENUM_MIN_BLOCKS;
}
__host__ __device__ constexpr bool mode_dominance(int mode) { return mode >= 5; }
__host__ __device__ constexpr bool mode_smem_sfx(int mode) { return mode >= 6; }
__host__ __device__ constexpr bool mode_one_pass(int mode) { return mode == 7; }
__host__ __device__ constexpr bool mode_rolled(int mode) { return mode == 7 || mode == 8; }
static_assert(mode_smem_sfx(8) && mode_rolled(8) && !mode_one_pass(8) && !mode_rolled(6),
              "walk mode 8: mode 6 with the rolled quad loop");

// One engine's path ends all 24 orders of S after a prefix with engine
// times (k, d) in three cases, each with a closed form for the minimum, the
// maximum and the sum of the 24 makespans max(c0, gamma_j, k + beta_j),
// c0 = d + alpha:
//   the DtH engine's: c0 >= every gamma_j and every k + beta_j, i.e.
//     c0 >= max(cmax, k + bmax): all 24 equal c0;
//   the K engine's: k + beta_j >= gamma_j for every j (k >= tmax) and
//     k + bmin >= c0: makespan j is k + beta_j;
//   the HtD engine's: gamma_j >= k + beta_j for every j (k <= tmin) and
//     cmin >= c0: makespan j is gamma_j.
// The sums are exact in 32 bits where the group's 24-order sums fit (SUM32);
// other groups take the first case only, with a 64-bit sum.
struct Dom {
    bool ok;
    int32_t mn, mx;
    unsigned long long sum;
};

template <bool SUM32>
__device__ __forceinline__ Dom dominated(int32_t k, int32_t d, const Sfx& S)
{
    const int32_t c0 = d + S.alpha, kmin = k + S.bmin, kmax = k + S.bmax;
    const bool all_d = c0 >= max(kmax, S.cmax);
    const bool all_k = SUM32 && k >= S.tmax && c0 <= kmin;
    const bool all_c = SUM32 && k <= S.tmin && c0 <= S.cmin;
    Dom r;
    r.ok = all_d || all_k || all_c;
    r.mn = all_d ? c0 : all_k ? kmin : S.cmin;
    r.mx = all_d ? c0 : all_k ? kmax : S.cmax;
    if (SUM32)
        r.sum = all_d ? 24u * (uint32_t)c0 : all_k ? 24u * (uint32_t)k + S.bsum : S.csum;
    else
        r.sum = 24ull * (uint32_t)c0;
    return r;
}

// The walk's bookkeeping for one prefix whose 24 orders reach pmin / pmax.
__device__ __forceinline__ void note_prefix(int32_t pmin, int32_t pmax, Acc& a)
{
    if (pmin < a.imin) { a.imin = pmin; a.imin_at = a.walked; }
    if (pmax > a.imax) { a.imax = pmax; a.imax_at = a.walked; }
    a.walked += 1;
}

// CHECK (walk modes 5 to 8): take the closed form when dominated() holds on every
// active lane of the warp, so that the warp's lanes stay on one path.
template <bool SUM32, int MODE, bool CHECK = mode_dominance(MODE)>
__device__ __forceinline__ void leaves(int32_t k, int32_t d, const Sfx& S, Acc& a)
{
    constexpr bool FMA_SUM = mode_straight(MODE);
    if constexpr (CHECK) {
        const Dom q = dominated<SUM32>(k, d, S);
        if (__all_sync(__activemask(), q.ok)) {
            a.sum += q.sum;
            note_prefix(q.mn, q.mx, a);
            return;
        }
        a.full += 1;
    }
    const int32_t c0 = d + S.alpha;
    int32_t m[24];
    if constexpr (mode_smem_sfx(MODE)) {
#pragma unroll
        for (int r = 0; r < 6; ++r) {
            const int4 bq = S.sq[r * kEnumBlock], cq = S.sq[(6 + r) * kEnumBlock];
            const uint32_t ku = (uint32_t)k;
            m[4 * r] = max3i(c0, cq.x, (int32_t)(ku * S.one + (uint32_t)bq.x));
            m[4 * r + 1] = max3i(c0, cq.y, (int32_t)(ku * S.one + (uint32_t)bq.y));
            m[4 * r + 2] = max3i(c0, cq.z, (int32_t)(ku * S.one + (uint32_t)bq.z));
            m[4 * r + 3] = max3i(c0, cq.w, (int32_t)(ku * S.one + (uint32_t)bq.w));
        }
    } else if constexpr (mode_fma_add(MODE)) {
#pragma unroll
        for (int j = 0; j < 24; ++j)
            m[j] = max3i(c0, S.c[j], (int32_t)((uint32_t)k * S.one + (uint32_t)S.b[j]));
    } else {
#pragma unroll
        for (int j = 0; j < 24; ++j) m[j] = max3i(c0, S.c[j], k + S.b[j]);
    }
    int32_t t8[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) t8[i] = min3i(m[3 * i], m[3 * i + 1], m[3 * i + 2]);
    const int32_t pmin = min3i(min3i(t8[0], t8[1], t8[2]), min3i(t8[3], t8[4], t8[5]),
                               min(t8[6], t8[7]));
    if (SUM32 && FMA_SUM) {
        // the group's duration sum bounds every makespan, and 24 of them fit
        uint32_t q[4] = {0u, 0u, 0u, 0u};
#pragma unroll
        for (int j = 0; j < 18; ++j) q[j & 3] = (uint32_t)m[j] * S.one + q[j & 3];
        const uint32_t t0 = (uint32_t)m[18] + (uint32_t)m[19] + (uint32_t)m[20];
        const uint32_t t1 = (uint32_t)m[21] + (uint32_t)m[22] + (uint32_t)m[23];
        a.sum += ((q[0] + q[1]) + (q[2] + q[3])) + (t0 + t1);
    } else if (SUM32) {
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
    note_prefix(pmin, pmax, a);
}

// The last two prefix positions, holding tasks x < y: orders (x, y), (y, x).
template <bool SUM32, int MODE>
__device__ __forceinline__ void last_two(Eng st, int4 x, int4 y, const Sfx& S, Acc& a)
{
    const Eng sxy = step(step(st, x.x, x.y, x.z), y.x, y.y, y.z);
    const Eng syx = step(step(st, y.x, y.y, y.z), x.x, x.y, x.z);
    leaves<SUM32, MODE>(sxy.k, sxy.d, S, a);
    leaves<SUM32, MODE>(syx.k, syx.d, S, a);
}

// Walk modes 6, 7: the 24 orders of S after each of six prefixes (in walk
// order), quad by quad of S's orders, so that each int4 of beta and gamma is
// read from shared memory once for the six.  Each prefix keeps its own
// minimum and (SUM32) its own 32-bit sum, which fits as in leaves.
template <bool SUM32, bool ROLLED>
__device__ __forceinline__ void leaves6(const Eng (&e)[6], const Sfx& S, Acc& a)
{
    int32_t c0[6], mn[6];
    uint32_t sm[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        c0[i] = e[i].d + S.alpha;
        mn[i] = INT32_MAX;
        sm[i] = 0u;
    }
    unsigned long long wide = 0;
    // ROLLED: a loop over the quads (the six prefixes' work per quad is
    // straight-line already, and the loop keeps the hot code small, which
    // pays on batches of many group sizes); else unrolled
    constexpr int kQuadUnroll = ROLLED ? 1 : 6;
#pragma unroll kQuadUnroll
    for (int r = 0; r < 6; ++r) {
        const int4 bq = S.sq[r * kEnumBlock], cq = S.sq[(6 + r) * kEnumBlock];
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            const uint32_t ku = (uint32_t)e[i].k;
            const int32_t m0 = max3i(c0[i], cq.x, (int32_t)(ku * S.one + (uint32_t)bq.x));
            const int32_t m1 = max3i(c0[i], cq.y, (int32_t)(ku * S.one + (uint32_t)bq.y));
            const int32_t m2 = max3i(c0[i], cq.z, (int32_t)(ku * S.one + (uint32_t)bq.z));
            const int32_t m3 = max3i(c0[i], cq.w, (int32_t)(ku * S.one + (uint32_t)bq.w));
            mn[i] = min3i(min3i(mn[i], m0, m1), m2, m3);
            if (SUM32) {
                // two terms as multiply-adds (FMA pipe), two as one 3-input add
                sm[i] = (uint32_t)m0 * S.one + sm[i];
                sm[i] = (uint32_t)m1 * S.one + sm[i];
                sm[i] = sm[i] + (uint32_t)m2 + (uint32_t)m3;
            } else {
                // two makespans fit in 32 bits unsigned
                wide += (uint32_t)m0 + (uint32_t)m1;
                wide += (uint32_t)m2 + (uint32_t)m3;
            }
        }
    }
    if (SUM32) {
        a.sum += ((unsigned long long)sm[0] + sm[1]) + ((unsigned long long)sm[2] + sm[3]) +
                 ((unsigned long long)sm[4] + sm[5]);
    } else {
        a.sum += wide;
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) note_prefix(mn[i], max3i(c0[i], e[i].k + S.bmax, S.cmax), a);
}

// Depth-first walk over the D remaining prefix tasks (ascending in `rem`):
// their orders in lexicographic order, so `walked` counts prefixes in rank
// order.  Straight-line modes: the level with three tasks left runs as straight-line code
// (its six prefixes in one block, which the compiler can interleave); else
// as a loop (less code: better when a batch mixes group sizes and so runs
// many walk depths and both sum widths at once).
template <int D, bool SUM32, int MODE>
__device__ __forceinline__ void dfs(Eng st, uint64_t rem, const int4* __restrict__ tbl,
                                    const Sfx& S, Acc& a)
{
    if constexpr (D == 0) {
        leaves<SUM32, MODE>(st.k, st.d, S, a);
    } else if constexpr (D == 1) {
        int4 t = tbl[nib_get(rem, 0)];
        Eng s1 = step(st, t.x, t.y, t.z);
        leaves<SUM32, MODE>(s1.k, s1.d, S, a);
    } else if constexpr (D == 2) {
        last_two<SUM32, MODE>(st, tbl[nib_get(rem, 0)], tbl[nib_get(rem, 1)], S, a);
    } else if constexpr (D == 3 && mode_one_pass(MODE) && SUM32) {
        // walk mode 7: as the block below, with the vote and the closed
        // forms in one pass (beta and gamma are not in registers here);
        // groups whose sums need 64 bits, where only the DtH engine's case
        // applies and the vote fails more often, take the block below.
        // Under any of the three cases the minimum of the 24 makespans is
        // max(c0, k + bmin, cmin): the dominating term's minimum, which
        // bounds the other two terms' minima; the maximum max(c0, k + bmax,
        // cmax) holds always.
        const int4 t0 = tbl[nib_get(rem, 0)], t1 = tbl[nib_get(rem, 1)], t2 = tbl[nib_get(rem, 2)];
        const Eng s0 = step(st, t0.x, t0.y, t0.z), s1 = step(st, t1.x, t1.y, t1.z),
                  s2 = step(st, t2.x, t2.y, t2.z);
        Eng e[6];
        e[0] = step(step(s0, t1.x, t1.y, t1.z), t2.x, t2.y, t2.z);
        e[1] = step(step(s0, t2.x, t2.y, t2.z), t1.x, t1.y, t1.z);
        e[2] = step(step(s1, t0.x, t0.y, t0.z), t2.x, t2.y, t2.z);
        e[3] = step(step(s1, t2.x, t2.y, t2.z), t0.x, t0.y, t0.z);
        e[4] = step(step(s2, t0.x, t0.y, t0.z), t1.x, t1.y, t1.z);
        e[5] = step(step(s2, t1.x, t1.y, t1.z), t0.x, t0.y, t0.z);
        int32_t mn[6], mx[6];
        unsigned long long sum = 0;
        bool ok = true;
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            const int32_t c0 = e[i].d + S.alpha, kmin = e[i].k + S.bmin;
            mx[i] = max3i(c0, e[i].k + S.bmax, S.cmax);
            mn[i] = max3i(c0, kmin, S.cmin);
            const bool all_d = c0 >= mx[i];
            const bool all_k = e[i].k >= S.tmax && c0 <= kmin;
            const bool all_c = e[i].k <= S.tmin && c0 <= S.cmin;
            ok = ok && (all_d || all_k || all_c);
            sum += all_d ? 24u * (uint32_t)c0 : all_k ? 24u * (uint32_t)e[i].k + S.bsum : S.csum;
        }
        if (__all_sync(__activemask(), ok)) {
            a.sum += sum;
            const int32_t pmin = min(min3i(mn[0], mn[1], mn[2]), min3i(mn[3], mn[4], mn[5]));
            const int32_t pmax = max(max3i(mx[0], mx[1], mx[2]), max3i(mx[3], mx[4], mx[5]));
            if (pmin < a.imin) {
                int at = 5;
#pragma unroll
                for (int i = 4; i >= 0; --i)
                    if (mn[i] == pmin) at = i;
                a.imin = pmin;
                a.imin_at = a.walked + (uint32_t)at;
            }
            if (pmax > a.imax) {
                int at = 5;
#pragma unroll
                for (int i = 4; i >= 0; --i)
                    if (mx[i] == pmax) at = i;
                a.imax = pmax;
                a.imax_at = a.walked + (uint32_t)at;
            }
            a.walked += 6;
        } else {
            a.full += 6;
            leaves6<SUM32, mode_rolled(MODE)>(e, S, a);
        }
    } else if constexpr (D == 3 && mode_dominance(MODE)) {
        // as below, with one dominance vote for all six prefixes: either all
        // six take the closed form on every lane, or all six the full leaves
        const int4 t0 = tbl[nib_get(rem, 0)], t1 = tbl[nib_get(rem, 1)], t2 = tbl[nib_get(rem, 2)];
        const Eng s0 = step(st, t0.x, t0.y, t0.z), s1 = step(st, t1.x, t1.y, t1.z),
                  s2 = step(st, t2.x, t2.y, t2.z);
        Eng e[6];
        e[0] = step(step(s0, t1.x, t1.y, t1.z), t2.x, t2.y, t2.z);
        e[1] = step(step(s0, t2.x, t2.y, t2.z), t1.x, t1.y, t1.z);
        e[2] = step(step(s1, t0.x, t0.y, t0.z), t2.x, t2.y, t2.z);
        e[3] = step(step(s1, t2.x, t2.y, t2.z), t0.x, t0.y, t0.z);
        e[4] = step(step(s2, t0.x, t0.y, t0.z), t1.x, t1.y, t1.z);
        e[5] = step(step(s2, t1.x, t1.y, t1.z), t0.x, t0.y, t0.z);
        // the vote carries one bit; the closed forms are formed after it,
        // so that the full path does not hold them
        bool ok = true;
#pragma unroll
        for (int i = 0; i < 6; ++i) ok = ok && dominated<SUM32>(e[i].k, e[i].d, S).ok;
        if (__all_sync(__activemask(), ok)) {
            // the six prefixes' minima, maxima and sums by shallow trees;
            // the first prefix reaching a new item minimum (maximum) is
            // only looked for when there is one, which is rare
            Dom q[6];
#pragma unroll
            for (int i = 0; i < 6; ++i) q[i] = dominated<SUM32>(e[i].k, e[i].d, S);
            a.sum += ((q[0].sum + q[1].sum) + (q[2].sum + q[3].sum)) + (q[4].sum + q[5].sum);
            const int32_t mn = min(min3i(q[0].mn, q[1].mn, q[2].mn), min3i(q[3].mn, q[4].mn, q[5].mn));
            const int32_t mx = max(max3i(q[0].mx, q[1].mx, q[2].mx), max3i(q[3].mx, q[4].mx, q[5].mx));
            if (mn < a.imin) {
                int at = 5;
#pragma unroll
                for (int i = 4; i >= 0; --i)
                    if (q[i].mn == mn) at = i;
                a.imin = mn;
                a.imin_at = a.walked + (uint32_t)at;
            }
            if (mx > a.imax) {
                int at = 5;
#pragma unroll
                for (int i = 4; i >= 0; --i)
                    if (q[i].mx == mx) at = i;
                a.imax = mx;
                a.imax_at = a.walked + (uint32_t)at;
            }
            a.walked += 6;
        } else {
            a.full += 6;
            if constexpr (mode_smem_sfx(MODE)) {
                leaves6<SUM32, mode_rolled(MODE)>(e, S, a);
            } else {
#pragma unroll
                for (int i = 0; i < 6; ++i) leaves<SUM32, MODE, false>(e[i].k, e[i].d, S, a);
            }
        }
    } else if constexpr (D == 3 && mode_straight(MODE)) {
        // the three tasks' rows loaded once; their six orders in
        // lexicographic order (the list is ascending)
        const int4 t0 = tbl[nib_get(rem, 0)], t1 = tbl[nib_get(rem, 1)], t2 = tbl[nib_get(rem, 2)];
        last_two<SUM32, MODE>(step(st, t0.x, t0.y, t0.z), t1, t2, S, a);
        last_two<SUM32, MODE>(step(st, t1.x, t1.y, t1.z), t0, t2, S, a);
        last_two<SUM32, MODE>(step(st, t2.x, t2.y, t2.z), t0, t1, S, a);
    } else {
#pragma unroll 1
        for (int c = 0; c < D; ++c) {
            int4 t = tbl[nib_get(rem, c)];
            dfs<D - 1, SUM32, MODE>(step(st, t.x, t.y, t.z), nib_remove(rem, c), tbl, S, a);
        }
    }
}

template <int PDMAX, bool SUM32, int MODE>
__device__ __forceinline__ void walk_prefixes(int pd, Eng st, uint64_t rem,
                                              const int4* __restrict__ tbl, const Sfx& S, Acc& a)
{
    switch (pd) {
    case 0: dfs<0, SUM32, MODE>(st, rem, tbl, S, a); break;
    case 1: dfs<1, SUM32, MODE>(st, rem, tbl, S, a); break;
    case 2: dfs<2, SUM32, MODE>(st, rem, tbl, S, a); break;
    default:
        if constexpr (PDMAX >= 3) { if (pd == 3) dfs<3, SUM32, MODE>(st, rem, tbl, S, a); }
        if constexpr (PDMAX >= 4) { if (pd == 4) dfs<4, SUM32, MODE>(st, rem, tbl, S, a); }
        if constexpr (PDMAX >= 5) { if (pd == 5) dfs<5, SUM32, MODE>(st, rem, tbl, S, a); }
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

// Rank of the item's first order (its head, the other prefix tasks
// ascending, then S's first order): no order of the item ranks lower.
__device__ __noinline__ uint32_t item_first_rank(uint32_t hd, uint64_t rem, int f, int pd, int n)
{
    const int P = n - 4;
    uint32_t digits = 0;
    for (int j = f - 1; j >= 0; --j) {
        const uint32_t r = (uint32_t)(P - j);
        const uint32_t q = hd / r;
        digits |= (hd - q * r) << (4 * j);
        hd = q;
    }
    uint32_t placed = 0;
    for (int j = 0; j < f; ++j) {
        const int c = (digits >> (4 * j)) & 0xF;
        placed |= (uint32_t)nib_get(rem, c) << (4 * j);
        rem = nib_remove(rem, c);
    }
    for (int q = 0; q < pd; ++q) placed |= (uint32_t)nib_get(rem, q) << (4 * (f + q));
    return prefix_rank(placed, n, P);
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

// The items whose first cost unit lies in [x0, x1), in order: walk them,
// settle each against the thread's running best / worst, and report to the
// group accumulators when the group changes and at the end.
template <int PDMAX, int MODE>
__device__ __forceinline__ void enum_range(const GroupPlan* __restrict__ gp,
                                           const GroupInfo* __restrict__ info,
                                           const int4* __restrict__ tbl,
                                           const SuffixTab* __restrict__ sub, int G, uint64_t x0,
                                           uint64_t x1, uint32_t item_cost, const Sink& sink,
                                           int4* sq)
{
    const uint64_t total = gp[G].cost_base;
    if (x0 >= total) return;
    uint32_t i = plan_first_item(gp, G, PDMAX, item_cost, x0);
    const uint32_t end = plan_first_item(gp, G, PDMAX, item_cost, min(x1, total));
    if (i >= end) return;
    int g = search_group(G, i, [&](int j) { return (uint64_t)gp[j].item_base; });
    Acc a;
    a.reset();
    a.full = 0;
    Sfx S;
    S.one = sink.one;
    S.sq = sq;
    GroupInfo gi;
    const int4* gt = tbl;
    uint32_t gbase = 0, gend = 0, heads = 1, cur = kFull;
    const SuffixTab* tab = sub;
    uint64_t sc = 0;   // S's complement, ascending nibbles
    int pd = 0, f = 0, P = 0;
    bool load_group = true;
    bool touched = false;   // this thread has visited an item of group g
    for (; i < end; ++i) {
        while (load_group || i >= gend) {
            if (!load_group) {
                if (touched) { flush(a, sink.acc, g); finished_single(sink, g); }
                a.reset();
                touched = false;
                ++g;
            }
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
        touched = true;
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
                if constexpr (mode_smem_sfx(MODE)) {   // this thread's column only
                    sq[q * kEnumBlock] = b;
                    sq[(6 + q) * kEnumBlock] = c;
                }
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
            if constexpr (mode_dominance(MODE)) {
                int32_t bn[8], cn[8], tn[8], tx[8];
                uint32_t bs = 0u, cs = 0u;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    bn[q] = min3i(S.b[3 * q], S.b[3 * q + 1], S.b[3 * q + 2]);
                    cn[q] = min3i(S.c[3 * q], S.c[3 * q + 1], S.c[3 * q + 2]);
                    const int32_t u0 = S.c[3 * q] - S.b[3 * q], u1 = S.c[3 * q + 1] - S.b[3 * q + 1],
                                  u2 = S.c[3 * q + 2] - S.b[3 * q + 2];
                    tn[q] = min3i(u0, u1, u2);
                    tx[q] = max3i(u0, u1, u2);
                    bs += (uint32_t)S.b[3 * q] + (uint32_t)S.b[3 * q + 1] + (uint32_t)S.b[3 * q + 2];
                    cs += (uint32_t)S.c[3 * q] + (uint32_t)S.c[3 * q + 1] + (uint32_t)S.c[3 * q + 2];
                }
                S.bmin = min3i(min3i(bn[0], bn[1], bn[2]), min3i(bn[3], bn[4], bn[5]), min(bn[6], bn[7]));
                S.cmin = min3i(min3i(cn[0], cn[1], cn[2]), min3i(cn[3], cn[4], cn[5]), min(cn[6], cn[7]));
                S.tmin = min3i(min3i(tn[0], tn[1], tn[2]), min3i(tn[3], tn[4], tn[5]), min(tn[6], tn[7]));
                S.tmax = max3i(max3i(tx[0], tx[1], tx[2]), max3i(tx[3], tx[4], tx[5]), max(tx[6], tx[7]));
                S.bsum = bs;
                S.csum = cs;
            }
            sc = 0;
            for (int e = 0, cnt = 0; e < gi.n; ++e)
                if (!((mask >> e) & 1u)) sc |= (uint64_t)e << (4 * cnt++);
        }
        uint64_t rem = sc;
        uint32_t placed;
        Eng st = run_head(hd, f, P, gi.dinit, rem, placed, gt);
        a.start_item();
        if (gi.sum32) walk_prefixes<PDMAX, true, MODE>(pd, st, rem, gt, S, a);
        else walk_prefixes<PDMAX, false, MODE>(pd, st, rem, gt, S, a);
        // Settle the item against the running best / worst: every lane of a
        // warp gets here together, so this rank work does not diverge.  A
        // tie can only lower the rank if the item's first order ranks below
        // the running one; a strict improvement always counts.
        const bool tie_b = a.imin == a.best, tie_w = a.imax == a.worst;
        uint32_t low = 0;
        if (tie_b || tie_w) low = item_first_rank(hd, sc, f, pd, gi.n);
        if (a.imin < a.best || (tie_b && low < a.best_rank)) {
            uint32_t r = item_rank(a.imin_at, a.imin, hd, sc, f, pd, gi.n, gi.dinit, gt, tab);
            if (a.imin < a.best || r < a.best_rank) { a.best = a.imin; a.best_rank = r; }
        }
        if (a.imax > a.worst || (tie_w && low < a.worst_rank)) {
            uint32_t r = item_rank(a.imax_at, a.imax, hd, sc, f, pd, gi.n, gi.dinit, gt, tab);
            if (a.imax > a.worst || r < a.worst_rank) { a.worst = a.imax; a.worst_rank = r; }
        }
    }
    if constexpr (mode_dominance(MODE)) {
        if (sink.full) {   // one atomic per warp
            const unsigned live = __activemask();
            const uint32_t tot = __reduce_add_sync(live, a.full);
            if ((int)(threadIdx.x & 31) == __ffs(live) - 1 && tot != 0)
                atomicAdd(sink.full, (unsigned long long)tot);
        }
    }
    flush_final(a, sink, g);
}

template <int PDMAX, int MODE>
__global__ void __launch_bounds__(kEnumBlock, mode_min_blocks(MODE))
enum_kernel(const GroupPlan* __restrict__ gp, const GroupInfo* __restrict__ info,
            const int4* __restrict__ tbl, const SuffixTab* __restrict__ sub, int G,
            uint64_t per_thread, uint32_t item_cost, Sink sink, uint32_t* next, uint32_t nchunks,
            uint64_t split_c, uint32_t split_warps, uint32_t split_hi, uint32_t split_klo,
            uint32_t enum_blocks, PrepArgs heur)
{
    pdl_launch_next();   // the finalize launch may begin
    if (blockIdx.x >= enum_blocks) {
        // Blocks after the enumeration's run the heuristic, a warp per group
        // (heur.orders set): they start as enumeration blocks finish, on the
        // SMs the enumeration's uneven tail leaves idle.
        prep_heuristic(heur, (int)((blockIdx.x - enum_blocks) * (blockDim.x / 32) + (threadIdx.x >> 5)),
                       threadIdx.x & 31);
        return;
    }
    // walk modes 6, 7: each thread's suffix constants, a column of 12 int4
    __shared__ int4 s_sfx[mode_smem_sfx(MODE) ? 12 * kEnumBlock : 1];
    int4* const sq = mode_smem_sfx(MODE) ? s_sfx + threadIdx.x : s_sfx;
    if (!next) {   // static split: one range per thread
        const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
        uint64_t x0, x1;
        static_range(t, per_thread, split_c, split_warps, split_hi, split_klo, &x0, &x1);
        enum_range<PDMAX, MODE>(gp, info, tbl, sub, G, x0, x1, item_cost, sink, sq);
        return;
    }
    // dynamic: each warp takes 32 consecutive chunks at a time, one per lane
    const int lane = threadIdx.x & 31;
    for (;;) {
        uint32_t c0 = 0;
        if (lane == 0) c0 = atomicAdd(next, 32u);
        c0 = __shfl_sync(kFull, c0, 0);
        if (c0 >= nchunks) break;
        const uint64_t c = (uint64_t)c0 + lane;
        enum_range<PDMAX, MODE>(gp, info, tbl, sub, G, c * per_thread, (c + 1) * per_thread, item_cost,
                                sink, sq);
        __syncwarp();
    }
}

// ---- finalize ---------------------------------------------------------------

// Separate finalize (when the plan has no completion counters): one warp
// per group of n >= 4 tasks; the prep kernel handled the others.  (The
// heuristic, when requested, runs in the enumeration launch's last blocks.)
__global__ void finalize_kernel(PrepArgs a, unsigned long long* __restrict__ acc)
{
    pdl_wait();          // the enumeration's reduction words
    const int g = (int)(((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (g >= a.G) return;
    const GroupInfo gi = a.info[g];
    if (gi.status == 0 && gi.n >= 4) finalize_group_warp(g, gi, a.tbl, acc, a.stats, a.status);
}

}  // namespace

// Walk modes 6 to 8 of the enumeration kernel, compiled in their own
// translation unit (exhaustive_wide.cu, this file with TM_ENUM_WIDE_MODES
// defined) so that the two build in parallel: launch, occupancy (resident
// blocks per SM), and module load for pdmax 3..5.
cudaError_t enum_wide_launch(int pdmax, int mode, const Plan& p, const Sink& sink,
                             const PrepArgs& heur, cudaStream_t stream, bool pdl);
cudaError_t enum_wide_occupancy(int pdmax, int mode, int* per_sm);
cudaError_t enum_wide_preload(int pdmax);

namespace {

// A launch configuration, with programmatic dependent launch if pdl.
struct LaunchCfg {
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute attr[1];
    LaunchCfg(unsigned grid, unsigned block, cudaStream_t s, bool pdl)
    {
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(block);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = s;
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = pdl ? attr : nullptr;
        cfg.numAttrs = pdl ? 1 : 0;
    }
};

// heur.orders set: the launch also runs the heuristic (enum_kernel).
template <int PDMAX, int MODE>
cudaError_t launch_enum(const Plan& p, const Sink& sink, const PrepArgs& heur, cudaStream_t stream,
                        bool pdl)
{
    const uint32_t blocks = (p.threads + kEnumBlock - 1) / kEnumBlock;
    const uint32_t hblocks = heur.orders ? (uint32_t)(p.G + kEnumBlock / 32 - 1) / (kEnumBlock / 32) : 0u;
    const bool dyn = p.chunks_per_thread > 1;
    LaunchCfg lc(blocks + hblocks, kEnumBlock, stream, pdl);
    return cudaLaunchKernelEx(&lc.cfg, enum_kernel<PDMAX, MODE>,
        (const GroupPlan*)p.d_gp, (const GroupInfo*)p.d_info, (const int4*)p.d_tbl,
        (const SuffixTab*)p.d_sub, p.G, (uint64_t)(dyn ? p.chunk : p.leaves_per_thread), p.item_cost,
        sink, dyn ? p.d_next : (uint32_t*)nullptr, dyn ? p.nchunks : 0u,
        (uint64_t)(dyn ? 0ull : p.split_c), p.split_warps, p.split_hi, p.split_klo, blocks, heur);
}

template <int PDMAX, int MODE>
cudaError_t enum_occupancy(int* per_sm)
{
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, enum_kernel<PDMAX, MODE>,
                                                         kEnumBlock, 0);
}

#ifndef TM_ENUM_WIDE_MODES

template <int PDMAX>
cudaError_t enum_occupancy_mode(int mode, int* per_sm)
{
    switch (mode) {
    case 1: return enum_occupancy<PDMAX, 1>(per_sm);
    case 2: return enum_occupancy<PDMAX, 2>(per_sm);
    case 3: return enum_occupancy<PDMAX, 3>(per_sm);
    case 4: return enum_occupancy<PDMAX, 4>(per_sm);
    case 5: return enum_occupancy<PDMAX, 5>(per_sm);
    case 6: case 7: case 8: return enum_wide_occupancy(PDMAX, mode, per_sm);
    default: return cudaErrorInvalidValue;
    }
}

template <int PDMAX>
cudaError_t launch_enum_mode(const Plan& p, const Sink& sink, const PrepArgs& heur,
                             cudaStream_t stream, bool pdl)
{
    switch (p.unroll) {
    case 1: return launch_enum<PDMAX, 1>(p, sink, heur, stream, pdl);
    case 2: return launch_enum<PDMAX, 2>(p, sink, heur, stream, pdl);
    case 3: return launch_enum<PDMAX, 3>(p, sink, heur, stream, pdl);
    case 4: return launch_enum<PDMAX, 4>(p, sink, heur, stream, pdl);
    case 5: return launch_enum<PDMAX, 5>(p, sink, heur, stream, pdl);
    case 6: case 7: case 8: return enum_wide_launch(PDMAX, p.unroll, p, sink, heur, stream, pdl);
    default: return cudaErrorInvalidValue;
    }
}

template <int PDMAX>
cudaError_t preload_modes()
{
    cudaFuncAttributes fa;
    cudaError_t e;
    if ((e = cudaFuncGetAttributes(&fa, enum_kernel<PDMAX, 1>)) != cudaSuccess) return e;
    if ((e = cudaFuncGetAttributes(&fa, enum_kernel<PDMAX, 2>)) != cudaSuccess) return e;
    if ((e = cudaFuncGetAttributes(&fa, enum_kernel<PDMAX, 3>)) != cudaSuccess) return e;
    if ((e = cudaFuncGetAttributes(&fa, enum_kernel<PDMAX, 4>)) != cudaSuccess) return e;
    if ((e = cudaFuncGetAttributes(&fa, enum_kernel<PDMAX, 5>)) != cudaSuccess) return e;
    return enum_wide_preload(PDMAX);
}

int resident_threads(int pdmax, int mode, int device, int blocks_per_sm)
{
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    cudaError_t e = cudaErrorInvalidValue;
    switch (pdmax) {
    case 3: e = enum_occupancy_mode<3>(mode, &per_sm); break;
    case 4: e = enum_occupancy_mode<4>(mode, &per_sm); break;
    case 5: e = enum_occupancy_mode<5>(mode, &per_sm); break;
    default: break;
    }
    if (e != cudaSuccess || sms <= 0 || per_sm <= 0) return 152 * 512;
    if (blocks_per_sm > 0 && blocks_per_sm < per_sm) per_sm = blocks_per_sm;
    return sms * per_sm * kEnumBlock;
}

}  // namespace

void exhaustive_partition(Plan& p, int device, int blocks_per_sm)
{
    uint64_t threads = std::min<uint64_t>((uint64_t)resident_threads(p.pdmax, p.unroll, device, blocks_per_sm),
                                          std::max<uint64_t>(p.total_items, 1));
    p.leaves_per_thread = std::max<uint64_t>(1, (p.total_leaves + threads - 1) / threads);
    p.threads = (uint32_t)((p.total_leaves + p.leaves_per_thread - 1) / p.leaves_per_thread);
    p.split_c = 0;
    p.split_warps = p.split_hi = p.split_klo = 0;
    if (p.chunks_per_thread == 1 && p.total_items > 0 && p.uniform_n >= 4) {
        const uint64_t I = p.total_items, c = p.total_leaves / I;   // every item costs c
        uint64_t warps = (threads + 31) / 32;
        const uint64_t klo = I / (32 * warps);
        if (klo == 0) warps = (I + 31) / 32;                // one item per lane at most
        const uint64_t hi = (I - 32 * warps * klo + 31) / 32;   // warps with klo + 1
        p.split_c = c;
        p.split_warps = (uint32_t)warps;
        p.split_hi = (uint32_t)hi;
        p.split_klo = (uint32_t)klo;
        p.threads = (uint32_t)(32 * warps);
    }
    if (p.chunks_per_thread > 1) {
        p.chunk = std::max<uint64_t>(1, p.leaves_per_thread / (uint64_t)p.chunks_per_thread);
        if (p.uniform_n >= 4 && p.total_items > 0) {
            // every item costs the same: chunks of whole items, so that each
            // lane of a warp that takes 32 chunks walks the same number
            const uint64_t c = p.total_leaves / p.total_items;
            const uint64_t per_thread = std::max<uint64_t>(1, p.total_items / threads);
            p.chunk = c * std::max<uint64_t>(1, (per_thread + p.chunks_per_thread / 2) /
                                                    (uint64_t)p.chunks_per_thread);
        }
        const uint64_t nch = (p.total_leaves + p.chunk - 1) / p.chunk;
        if (nch >= 0xFFFFFF00ull) {           // counter range: fall back to the static split
            p.chunks_per_thread = 1;
        } else {
            p.nchunks = (uint32_t)nch;
        }
    }
    p.launches = exhaustive_launch_count(p);
}

cudaError_t exhaustive_preload()
{
    cudaFuncAttributes fa;
    cudaError_t e;
    if ((e = cudaFuncGetAttributes(&fa, prep_kernel)) != cudaSuccess) return e;
    if ((e = cudaFuncGetAttributes(&fa, finalize_kernel)) != cudaSuccess) return e;
    if ((e = preload_modes<3>()) != cudaSuccess) return e;
    if ((e = preload_modes<4>()) != cudaSuccess) return e;
    return preload_modes<5>();
}

int exhaustive_launch_count(const Plan& p)
{
    if (p.G == 0) return 0;
    return 1 + (p.total_items > 0 ? 1 : 0) + (p.d_done ? 0 : 1);
}

cudaError_t launch_exhaustive(const Plan& p, const tm_task* d_tasks, const tm_device* d_devs,
                              tm_stats* d_stats, int32_t* d_status, cudaStream_t stream,
                              int32_t* d_orders, int32_t* d_makespans)
{
    if (p.G == 0) return cudaSuccess;
    PrepArgs pa;
    pa.tasks = d_tasks;
    pa.devs = d_devs;
    pa.gp = p.d_gp;
    pa.G = p.G;
    pa.info = p.d_info;
    pa.tbl = p.d_tbl;
    pa.sub = p.d_sub;
    pa.stats = d_stats;
    pa.status = d_status;
    pa.orders = d_orders;
    pa.makespans = d_makespans;
    pa.next = (p.chunks_per_thread > 1 && p.total_items > 0) ? p.d_next : nullptr;
    pa.full = p.d_full;
    // a block per group: 512 threads when the batch's groups have many
    // (subset, order) pairs (n >= 9: >= 3,024), else 128
    const int prep_threads = p.total_subs >= 100u * (uint32_t)p.G ? kPrepMaxThreads : 128;
    // the heuristic runs in the enumeration launch's last blocks when there
    // is one, else here
    const bool heur_late = d_orders && p.total_items > 0;
    PrepArgs pp = pa;
    if (heur_late) pp.orders = pp.makespans = nullptr;
    const int heur_blocks =
        pp.orders ? (p.G + prep_threads / 32 - 1) / (prep_threads / 32) : 0;
    prep_kernel<<<p.G + heur_blocks, prep_threads, 0, stream>>>(pp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (p.total_items > 0) {
        Sink sink{p.d_acc, p.d_info, p.d_tbl, d_stats, d_status, p.d_target, p.d_done, 1u, p.d_full};
        // Under stream capture, an external record becomes an event-record
        // node of the graph (a plain record would only order the capture).
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        if (p.ev_before && (e = cudaStreamIsCapturing(stream, &cap)) != cudaSuccess) return e;
        const unsigned rec_flags =
            cap == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : cudaEventRecordDefault;
        if (p.ev_before &&
            (e = cudaEventRecordWithFlags(p.ev_before, stream, rec_flags)) != cudaSuccess)
            return e;
        PrepArgs heur = pa;
        if (!heur_late) heur.orders = heur.makespans = nullptr;
        switch (p.pdmax) {
        case 3: e = launch_enum_mode<3>(p, sink, heur, stream, false); break;
        case 4: e = launch_enum_mode<4>(p, sink, heur, stream, false); break;
        case 5: e = launch_enum_mode<5>(p, sink, heur, stream, false); break;
        default: return cudaErrorInvalidValue;
        }
        if (e != cudaSuccess) return e;
        if (p.ev_after &&
            (e = cudaEventRecordWithFlags(p.ev_after, stream, rec_flags)) != cudaSuccess)
            return e;
        if (!p.d_done) {
            const int fin_blocks = (p.G * 32 + 255) / 256;
            // programmatic dependent launch where it directly follows the
            // enumeration (a timing event between them keeps stream order)
            LaunchCfg lc((unsigned)fin_blocks, 256, stream, !p.ev_after);
            e = cudaLaunchKernelEx(&lc.cfg, finalize_kernel, pa, p.d_acc);
        }
    }
    return e;
}

#else   // TM_ENUM_WIDE_MODES: the launchers of walk modes 6 to 8

}  // namespace

cudaError_t enum_wide_launch(int pdmax, int mode, const Plan& p, const Sink& sink,
                             const PrepArgs& heur, cudaStream_t stream, bool pdl)
{
#define TM_WIDE_CASE(PD, M) \
    case (PD) * 16 + (M): return launch_enum<PD, M>(p, sink, heur, stream, pdl);
    switch (pdmax * 16 + mode) {
    TM_WIDE_CASE(3, 6) TM_WIDE_CASE(3, 7) TM_WIDE_CASE(3, 8)
    TM_WIDE_CASE(4, 6) TM_WIDE_CASE(4, 7) TM_WIDE_CASE(4, 8)
    TM_WIDE_CASE(5, 6) TM_WIDE_CASE(5, 7) TM_WIDE_CASE(5, 8)
    default: return cudaErrorInvalidValue;
    }
#undef TM_WIDE_CASE
}

cudaError_t enum_wide_occupancy(int pdmax, int mode, int* per_sm)
{
#define TM_WIDE_CASE(PD, M) \
    case (PD) * 16 + (M): return enum_occupancy<PD, M>(per_sm);
    switch (pdmax * 16 + mode) {
    TM_WIDE_CASE(3, 6) TM_WIDE_CASE(3, 7) TM_WIDE_CASE(3, 8)
    TM_WIDE_CASE(4, 6) TM_WIDE_CASE(4, 7) TM_WIDE_CASE(4, 8)
    TM_WIDE_CASE(5, 6) TM_WIDE_CASE(5, 7) TM_WIDE_CASE(5, 8)
    default: return cudaErrorInvalidValue;
    }
#undef TM_WIDE_CASE
}

cudaError_t enum_wide_preload(int pdmax)
{
    cudaFuncAttributes fa;
    cudaError_t e;
    switch (pdmax) {
#define TM_WIDE_LOAD(PD)                                                                    \
    case PD:                                                                                \
        if ((e = cudaFuncGetAttributes(&fa, enum_kernel<PD, 6>)) != cudaSuccess) return e; \
        if ((e = cudaFuncGetAttributes(&fa, enum_kernel<PD, 7>)) != cudaSuccess) return e; \
        return cudaFuncGetAttributes(&fa, enum_kernel<PD, 8>);
    TM_WIDE_LOAD(3) TM_WIDE_LOAD(4) TM_WIDE_LOAD(5)
#undef TM_WIDE_LOAD
    default: return cudaErrorInvalidValue;
    }
}

#endif  // TM_ENUM_WIDE_MODES

}  // namespace tmgpu

// tm_internal.h -- data layout and launch helpers shared by the CUDA
// translation units of libtm.so.  Nothing here is visible through tm.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "tm.h"

namespace tmgpu {

// 0! .. 20!
__host__ __device__ inline uint64_t factorial_u64(int n)
{
    uint64_t f = 1;
    for (int i = 2; i <= n; ++i) f *= (uint64_t)i;
    return f;
}

// Number of 4-task subsets of n tasks.
__host__ __device__ inline uint32_t choose4(int n)
{
    return n < 4 ? 0u : (uint32_t)(n * (n - 1) * (n - 2) * (n - 3) / 24);
}

// Each group's three reduction words (min key, max key, sum) and its
// completion counter sit on their own 128-byte line, so that the atomics of
// different groups do not queue at the same L2 slice.
constexpr int kAccStride = 16;    // unsigned long long per group
constexpr int kDoneStride = 32;   // uint32_t per group

// Per-group facts derived on the device by the prep kernel.
struct GroupInfo {
    int32_t off;      // index of the group's first task
    int32_t n;        // number of tasks
    int32_t dinit;    // time the DtH stream becomes free before the first
                      // task: 0 with two DMA engines; with one engine the
                      // single transfer queue carries every HtD first, so it
                      // is the sum of HtD (Sec. 3.2, Fig. 2)
    int32_t hs;       // sum of HtD of the group
    int32_t status;   // 0 or a tm_status code
    uint32_t sum32;   // 1 if 24 makespans of this group always fit in 32 bits
    int32_t user;     // the caller's index of the group (outputs go there)
    int32_t pad1;
};

// Per-group work layout computed on the host from the group sizes alone.
// Groups are laid out in WORK ORDER: by size, largest first, stable (so a
// batch of one size keeps the caller's order).  The threads and warps that
// run at one time then mostly hold groups of one size and walk one code
// path, which keeps the instruction cache warm on mixed batches.  Every
// per-group array of the plan (GroupInfo, the padded task table, suffix
// tables, reduction words) is in work order; inputs are read and outputs
// written at the caller's index.  Entry G holds the totals.
struct GroupPlan {
    uint64_t cost_base;   // first cost unit of the group: each work item of a
                          // group with n >= 4 costs its orders plus a fixed
                          // per-item overhead (the plan's item_cost)
    uint32_t item_base;   // first work item
    uint32_t unit_base;   // first thread of the prep / suffix-table kernel
    uint32_t sub_base;    // first suffix-table entry
    int32_t off;          // first task in the plan's task table (work order)
    int32_t uoff;         // first task in the caller's task array
    int32_t group;        // the caller's index of the group
};

// The last four positions of an order hold a 4-task set S.  Because the
// model's recurrence is max-plus linear in the engine times (h, k, d), the
// makespan of prefix pi followed by an order sigma of S is
//     max(d_pi + alpha, k_pi + beta[sigma], gamma[sigma])
// where h entering S is fixed (the HtD sum of the other tasks) and folded
// into gamma.  One entry per (group, S); sigma in lexicographic order of S.
struct SuffixTab {
    int32_t beta[24];    // longest path from the K-engine time to the end
    int32_t gamma[24];   // longest path from the HtD-engine time, plus that time
    int32_t alpha;       // sum of DtH over S (the DtH-engine path)
    uint32_t mask;       // bit e set if task e is in S
    int32_t pad0, pad1;
};
static_assert(sizeof(SuffixTab) == 208, "suffix table layout");

// Exhaustive-search plan (see tm_plan_create in tm.h).
struct Plan {
    int device = 0;
    int G = 0;
    int T = 0;                    // total tasks
    int pdmax = 4;                // prefix positions walked depth-first per item
    uint32_t total_items = 0;     // work items over all groups
    uint64_t total_leaves = 0;    // cost units of all work items (see GroupPlan)
    uint32_t item_cost = 256;     // per-item overhead, in orders
    uint32_t total_units = 0;     // prep / suffix-table threads
    uint32_t total_subs = 0;      // suffix-table entries
    uint64_t total_prefixes = 0;  // prefixes walked per run: n! / 24 per group of n >= 4
    int uniform_n = 0;            // the group size when every group has it, else 0
    uint32_t threads = 0;         // enumeration threads
    uint64_t leaves_per_thread = 0;
    int launches = 0;
    // Work distribution of the enumeration: 1 = a static split (thread t
    // takes cost units [t W, (t + 1) W)); c > 1 = dynamic: c chunks of W / c
    // units per thread, which warps take in turn from the counter *d_next
    // (zeroed by the prep kernel), so threads that meet cheap orders take
    // more work.
    int chunks_per_thread = 1;
    int unroll = 2;                       // 1: straight-line walk level (tm_tuning)
    // Static split of a batch of one group size (all work items cost the
    // same, split_c): whole warps take klo or klo + 1 items per lane, the
    // split_hi heavier warps spread evenly over the split_warps warps, so no
    // lane of a warp waits for another's extra item and every SM holds the
    // same mix.  split_c == 0: contiguous cost ranges of leaves_per_thread.
    uint64_t split_c = 0;
    uint32_t split_warps = 0, split_hi = 0, split_klo = 0;
    uint64_t chunk = 0;                   // cost units per chunk (dynamic)
    uint32_t nchunks = 0;
    GroupPlan* d_gp = nullptr;            // [G + 1]
    GroupInfo* d_info = nullptr;          // [G]
    int4* d_tbl = nullptr;                // [T] {htd, k, dth, 0}
    SuffixTab* d_sub = nullptr;           // [total_subs]
    unsigned long long* d_acc = nullptr;  // [kAccStride G] min key, max key, sum
    // Fused finalize: each group is finalized by the last enumeration thread
    // to finish with it.  d_target[g] counts the threads whose item range
    // touches group g; d_done[g] counts those that finished.  Without these
    // (nullptr) a separate finalize kernel runs.
    uint32_t* d_target = nullptr;         // [G]
    uint32_t* d_done = nullptr;           // [kDoneStride G]
    uint32_t* d_next = nullptr;           // dynamic chunk counter
    // Prefixes of the last run whose 24 completions were evaluated order by
    // order (walk modes 5 to 8 count them; the others evaluate every prefix so);
    // zeroed by the prep kernel; in d_next's 256-byte piece.
    unsigned long long* d_full = nullptr;
    cudaEvent_t ev_before = nullptr;      // optional timing hook
    cudaEvent_t ev_after = nullptr;
};

// Work item of a group with n >= 4 tasks: a 4-subset S (the last four
// positions) and a HEAD, the first f positions of the prefix; the thread
// walks the remaining pd prefix positions depth-first.  P = n - 4.
__host__ __device__ inline int plan_pd(int n, int pdmax) { return n - 4 < pdmax ? n - 4 : pdmax; }

// Fills gp[0..G] from host offsets; allocates nothing.  Returns TM_OK,
// TM_EINVAL (bad offsets) or TM_ETOOBIG (n > 12 or too many items).
inline int plan_decompose(const int32_t* offsets, int G, int pdmax, uint32_t item_cost,
                          GroupPlan* gp, Plan* totals)
{
    if (!offsets || G < 0 || offsets[0] != 0 || pdmax < 2 || pdmax > 5) return TM_EINVAL;
    // work order: a counting sort by size, largest first, stable
    uint32_t start[TM_MAX_EXHAUSTIVE + 1] = {};
    for (int g = 0; g < G; ++g) {
        const int n = offsets[g + 1] - offsets[g];
        if (n < 1) return TM_EINVAL;
        if (n > TM_MAX_EXHAUSTIVE) return TM_ETOOBIG;
        ++start[n];
    }
    for (uint32_t nn = TM_MAX_EXHAUSTIVE, at = 0; nn >= 1; --nn) {
        const uint32_t c = start[nn];
        start[nn] = at;
        at += c;
    }
    for (int g = 0; g < G; ++g) gp[start[offsets[g + 1] - offsets[g]]++].group = g;
    uint64_t cost = 0, items = 0, units = 0, subs = 0, prefixes = 0;
    int32_t toff = 0;
    for (int w = 0; w < G; ++w) {
        const int g = gp[w].group;
        const int n = offsets[g + 1] - offsets[g];
        gp[w].cost_base = cost;
        gp[w].item_base = (uint32_t)items;
        gp[w].unit_base = (uint32_t)units;
        gp[w].sub_base = (uint32_t)subs;
        gp[w].off = toff;
        gp[w].uoff = offsets[g];
        toff += n;
        uint32_t c4 = choose4(n);
        units += c4 > 0 ? c4 : 1;
        subs += c4;
        if (n >= 4) {
            int P = n - 4, pd = plan_pd(n, pdmax);
            uint64_t heads = factorial_u64(P) / factorial_u64(pd);
            items += (uint64_t)c4 * heads;
            cost += (uint64_t)c4 * heads * (24ull * factorial_u64(pd) + item_cost);
            prefixes += factorial_u64(n) / 24;
        }
        if (items >= 0xFFFFFFFFull || units >= 0xFFFFFFFFull) return TM_ETOOBIG;
    }
    gp[G].cost_base = cost;
    gp[G].item_base = (uint32_t)items;
    gp[G].unit_base = (uint32_t)units;
    gp[G].sub_base = (uint32_t)subs;
    gp[G].off = offsets[G];
    gp[G].uoff = offsets[G];
    gp[G].group = G;
    totals->G = G;
    totals->T = offsets[G];
    totals->pdmax = pdmax;
    totals->item_cost = item_cost;
    totals->total_items = (uint32_t)items;
    totals->total_leaves = cost;
    totals->total_units = (uint32_t)units;
    totals->total_subs = (uint32_t)subs;
    totals->total_prefixes = prefixes;
    totals->uniform_n = 0;
    for (int nn = 1; nn <= TM_MAX_EXHAUSTIVE && G > 0; ++nn)
        if (start[nn] - (nn < TM_MAX_EXHAUSTIVE ? start[nn + 1] : 0u) == (uint32_t)G) totals->uniform_n = nn;
    return TM_OK;
}

// Lays the plan's device arrays out in one block starting at `base` (256-byte
// aligned pieces) and returns the block's size; with base == nullptr it only
// measures.
inline size_t plan_carve(Plan& p, unsigned char* base)
{
    size_t off = 0;
    auto take = [&](size_t bytes) {
        unsigned char* at = base ? base + off : nullptr;
        off += (bytes + 255) & ~size_t(255);
        return at;
    };
    const size_t G1 = (size_t)(p.G > 0 ? p.G : 1), T1 = (size_t)(p.T > 0 ? p.T : 1);
    const size_t S1 = (size_t)(p.total_subs > 0 ? p.total_subs : 1);
    p.d_gp = reinterpret_cast<GroupPlan*>(take((G1 + 1) * sizeof(GroupPlan)));
    p.d_info = reinterpret_cast<GroupInfo*>(take(G1 * sizeof(GroupInfo)));
    p.d_tbl = reinterpret_cast<int4*>(take(T1 * sizeof(int4)));
    p.d_sub = reinterpret_cast<SuffixTab*>(take(S1 * sizeof(SuffixTab)));
    p.d_acc = reinterpret_cast<unsigned long long*>(
        take(kAccStride * G1 * sizeof(unsigned long long)));
    p.d_next = reinterpret_cast<uint32_t*>(take(2 * sizeof(unsigned long long)));
    p.d_full = base ? reinterpret_cast<unsigned long long*>(p.d_next) + 1 : nullptr;
    return off;
}

// Device arrays of the fused-finalize plan, laid out after plan_carve's
// block (same conventions).
inline size_t plan_carve_fused(Plan& p, unsigned char* base)
{
    size_t off = 0;
    auto take = [&](size_t bytes) {
        unsigned char* at = base ? base + off : nullptr;
        off += (bytes + 255) & ~size_t(255);
        return at;
    };
    const size_t G1 = (size_t)(p.G > 0 ? p.G : 1);
    p.d_target = reinterpret_cast<uint32_t*>(take(G1 * sizeof(uint32_t)));
    p.d_done = reinterpret_cast<uint32_t*>(take(kDoneStride * G1 * sizeof(uint32_t)));
    return off;
}

// First work item whose first cost unit is at or after x (host and device);
// pdmax and item_cost as in the plan.
__host__ __device__ inline uint32_t plan_first_item(const GroupPlan* gp, int G, int pdmax,
                                                    uint32_t item_cost, uint64_t x)
{
    if (x >= gp[G].cost_base) return gp[G].item_base;
    int lo = 0, hi = G;                       // largest g with cost_base <= x
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (gp[mid].cost_base <= x) lo = mid; else hi = mid;
    }
    const int n = gp[lo + 1].off - gp[lo].off;
    const uint64_t lpi = 24ull * factorial_u64(plan_pd(n, pdmax)) + item_cost;
    const uint64_t q = (x - gp[lo].cost_base + lpi - 1) / lpi;
    const uint64_t i = gp[lo].item_base + q;
    return (uint32_t)(i < gp[lo + 1].item_base ? i : gp[lo + 1].item_base);
}

// Cost units [x0, x1) of static-split enumeration thread t.
__host__ __device__ inline void static_range(uint64_t t, uint64_t per_thread, uint64_t split_c,
                                             uint32_t split_warps, uint32_t split_hi,
                                             uint32_t split_klo, uint64_t* x0, uint64_t* x1)
{
    if (split_c == 0) {
        *x0 = t * per_thread;
        *x1 = (t + 1) * per_thread;
        return;
    }
    const uint64_t w = t >> 5, lane = t & 31;
    const uint64_t hi_before = w * split_hi / split_warps;
    const uint64_t k = split_klo + (((w + 1) * split_hi / split_warps > hi_before) ? 1u : 0u);
    const uint64_t first = 32 * (split_klo * w + hi_before) + lane * k;
    *x0 = first * split_c;
    *x1 = (first + k) * split_c;
}

// Launchers (return cudaError_t of the launch).  With d_orders non-null the
// heuristic for every group runs in the same launches (orders in the task
// layout, makespans optional).
cudaError_t launch_exhaustive(const Plan& plan, const tm_task* d_tasks,
                              const tm_device* d_devs, tm_stats* d_stats,
                              int32_t* d_status, cudaStream_t stream,
                              int32_t* d_orders = nullptr, int32_t* d_makespans = nullptr);
int exhaustive_launch_count(const Plan& plan);
// Sets plan.threads and plan.leaves_per_thread for the given device;
// blocks_per_sm 0 = occupancy limit.
void exhaustive_partition(Plan& plan, int device, int blocks_per_sm = 0);
// Loads every kernel launch_exhaustive can launch (prep, each enumeration
// variant, finalize) on the current device, so that no later launch has to
// load code (under lazy module loading the first launch of a kernel loads
// its module, which allocates device memory).
cudaError_t exhaustive_preload();

cudaError_t launch_predict(const tm_task* d_tasks, const int32_t* d_offsets,
                           int G, const int32_t* d_orders,
                           const tm_device* d_devs, int32_t* d_makespans,
                           int32_t* d_status, cudaStream_t stream);

// Partial-overlap variant (overlap.cu).  rate: 1 <= num <= den <= 1024.
int overlap_rate_ok(int32_t num, int32_t den);
cudaError_t launch_overlap_predict(const tm_task* d_tasks, const int32_t* d_offsets, int G,
                                   const int32_t* d_orders, const tm_device* d_devs, int32_t num,
                                   int32_t den, int32_t* d_makespans, int32_t* d_status,
                                   cudaStream_t s);
int overlap_exhaustive(const tm_task* d_tasks, const int32_t* d_offsets, const int32_t* h_offsets,
                       int G, const tm_device* d_devs, int32_t num, int32_t den, tm_stats* d_stats,
                       int32_t* d_status, cudaStream_t s);
cudaError_t launch_heuristic(const tm_task* d_tasks, const int32_t* d_offsets,
                             int G, const tm_device* d_devs,
                             int32_t* d_orders, int32_t* d_makespans,
                             int32_t* d_status, cudaStream_t stream);

}  // namespace tmgpu

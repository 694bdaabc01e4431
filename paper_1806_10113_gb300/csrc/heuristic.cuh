// heuristic.cuh -- the Batch Reordering heuristic (Sec. 5.1, Algorithm 1),
// one warp (or half a warp) per task group, lane j holding task j.  Used by
// the heuristic kernel and by the fused scheduling launches.
//
// The selection rules follow the paper's wording under these readings:
//   select_first_task: largest K - HtD (short HtD, long K); ties -> longer
//     DtH; ties -> lower task index.
//   update(OT): the model applied to the ordered set OT alone; t_HTD, t_K,
//     t_DTH are the ends of its last HtD, K and DtH command.
//   select_next_task: best fit of the candidate's HtD to the kernel time left
//     after the last HtD, and of its kernel (starting at
//     s = max(t_K, t_HTD + HtD_j)) to the DtH time left after s:
//     cost_j = |(t_K - t_HTD) - HtD_j| + |(t_DTH - s) - K_j|, smallest wins;
//     ties -> longer K; ties -> lower index.
//   select_last_tasks: with two tasks left, both completions are evaluated
//     with the model; the smaller makespan wins; ties -> the completion whose
//     last task has the shorter DtH; ties -> lower index first.
//   n = 1 -> [0]; n = 2 -> select_last_tasks on both tasks.
// Lanes score all candidates at once; warp reductions pick the winner.
#pragma once

#include "tm_device.cuh"

namespace tmgpu {
namespace heur {

constexpr unsigned kFull = 0xFFFFFFFFu;

// A group runs on a segment of W lanes of one warp (W = 32: the whole warp;
// W = 16: half a warp, two groups per warp; groups have at most 16 tasks):
// `mask` holds the segment's lanes, lane numbers are within the segment.
template <int W>
__device__ __forceinline__ unsigned seg_mask()
{
    return W == 32 ? kFull : (0xFFFFu << (threadIdx.x & 16u));
}

template <int W>
__device__ __forceinline__ unsigned seg_ballot(unsigned mask, bool pred)
{
    const unsigned b = __ballot_sync(mask, pred);
    return W == 32 ? b : (b >> (threadIdx.x & 16u)) & 0xFFFFu;
}

__device__ __forceinline__ int lowest_lane(unsigned mask) { return __ffs(mask) - 1; }

template <int W>
__device__ __forceinline__ int64_t seg_min_i64(unsigned mask, int64_t v)
{
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1)
        v = min(v, (int64_t)__shfl_xor_sync(mask, (long long)v, o, W));
    return v;
}

// With one DMA engine the DtH chain of OT starts when the last of OT's HtDs
// ends; as a max-plus function of that start x it is max(x + sumD, C), where
// sumD is the DtH sum of OT and C the chain's value started from minus
// infinity.  Keeping (sumD, C) makes each update O(1).
constexpr int32_t kNegC = INT32_MIN / 2;

struct HeurState {
    int32_t tH, tK, tD;   // ends of the last HtD, K and DtH of OT
    int32_t sumD, C;      // one-engine DtH chain of OT (see above)
    int m;                // |OT|
    int32_t my_ot;        // lane i: task at position i of OT
};

// Appends task j (durations hj, kj, dj) to OT and updates t_HTD, t_K, t_DTH.
__device__ __forceinline__ void append(HeurState& st, int lane, int dma, int j,
                                       int32_t hj, int32_t kj, int32_t dj)
{
    st.tH += hj;                          // HtDs run back to back
    const int32_t kend = max(st.tK, st.tH) + kj;
    st.tK = kend;
    if (lane == st.m) st.my_ot = j;
    st.m += 1;
    if (dma == 2) {
        st.tD = max(st.tD, kend) + dj;
    } else {
        st.C = max(st.C, kend) + dj;
        st.sumD += dj;
        st.tD = max(st.tH + st.sumD, st.C);   // OT's DtHs follow all of OT's HtDs
    }
}

// Makespan of OT followed by tasks a then b (the last two).
__device__ __forceinline__ int32_t finish_two(const HeurState& st, int dma, int32_t hs,
                                              int32_t ha, int32_t ka, int32_t da,
                                              int32_t hb, int32_t kb, int32_t db)
{
    const int32_t h1 = st.tH + ha;
    const int32_t k1 = max(st.tK, h1) + ka;
    const int32_t h2 = h1 + hb;
    const int32_t k2 = max(k1, h2) + kb;
    // one engine: every HtD of the group precedes the first DtH
    int32_t d = dma == 1 ? max(hs + st.sumD, st.C) : st.tD;
    d = max(d, k1) + da;
    d = max(d, k2) + db;
    return d;
}

// Algorithm 1 for group g (tasks[off .. off + n)), run by a segment of W
// lanes (every lane of it; lane = the lane within the segment).
template <int W>
__device__ __forceinline__ void heuristic_group_seg(const tm_task* __restrict__ tasks, int off,
                                                    int n, int dma, int g, int lane,
                                                    int32_t* __restrict__ orders_out,
                                                    int32_t* __restrict__ ms_out,
                                                    int32_t* __restrict__ status)
{
    const unsigned mask = seg_mask<W>();
    // the input check of check_group, one task per lane
    if (n < 1 || n > TM_MAX_TASKS || n > W || (dma != 1 && dma != 2)) {
        if (lane == 0 && status) status[g] = TM_EINVAL;
        return;
    }
    int32_t H = 0, K = 0, D = 0;
    if (lane < n) {
        tm_task t = tasks[off + lane];
        H = t.htd; K = t.k; D = t.dth;
    }
    long long tot = (long long)H + K + D, hsum = H;
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) {
        tot += __shfl_xor_sync(mask, tot, o, W);
        hsum += __shfl_xor_sync(mask, hsum, o, W);
    }
    const int err = seg_ballot<W>(mask, H < 0 || K < 0 || D < 0) ? TM_ENEG
                    : tot > INT32_MAX                              ? TM_EOVERFLOW
                                                                   : 0;
    if (err != 0) {
        if (lane == 0 && status) status[g] = err;
        return;
    }
    const int32_t hs = (int32_t)hsum, dinit = dma == 1 ? hs : 0;
    unsigned rt = (n >= 32) ? kFull : ((1u << n) - 1u);   // remaining tasks
    HeurState st{0, 0, dinit, 0, kNegC, 0, -1};
    auto take = [&](int j) {
        int32_t hj = __shfl_sync(mask, H, j, W), kj = __shfl_sync(mask, K, j, W),
                dj = __shfl_sync(mask, D, j, W);
        append(st, lane, dma, j, hj, kj, dj);
        rt &= ~(1u << j);
    };

    if (n == 1) {
        take(0);
    } else {
        if (n >= 3) {
            // select_first_task
            bool in = (rt >> lane) & 1u;
            int32_t gain = in ? K - H : INT32_MIN;
            int32_t best_gain = __reduce_max_sync(mask, gain);
            bool c1 = in && gain == best_gain;
            int32_t best_d = (int32_t)__reduce_max_sync(mask, c1 ? (unsigned)D : 0u);
            take(lowest_lane(seg_ballot<W>(mask, c1 && D == best_d)));
            // select_next_task while more than two tasks remain
            while (__popc(rt) > 2) {
                bool inr = (rt >> lane) & 1u;
                int64_t s = max((int64_t)st.tK, (int64_t)st.tH + H);
                int64_t a = ((int64_t)st.tK - st.tH) - H;
                int64_t b = ((int64_t)st.tD - s) - K;
                int64_t cost = inr ? (a < 0 ? -a : a) + (b < 0 ? -b : b) : INT64_MAX;
                int64_t best_cost = seg_min_i64<W>(mask, cost);
                bool c = inr && cost == best_cost;
                int32_t best_k = (int32_t)__reduce_max_sync(mask, c ? (unsigned)K : 0u);
                take(lowest_lane(seg_ballot<W>(mask, c && K == best_k)));
            }
        }
        // select_last_tasks on the two remaining tasks a < b
        int a = __ffs(rt) - 1;
        int b = 31 - __clz(rt);
        int32_t ha = __shfl_sync(mask, H, a, W), ka = __shfl_sync(mask, K, a, W),
                da = __shfl_sync(mask, D, a, W);
        int32_t hb = __shfl_sync(mask, H, b, W), kb = __shfl_sync(mask, K, b, W),
                db = __shfl_sync(mask, D, b, W);
        int32_t m_ab = finish_two(st, dma, hs, ha, ka, da, hb, kb, db);
        int32_t m_ba = finish_two(st, dma, hs, hb, kb, db, ha, ka, da);
        bool ba = (m_ab != m_ba) ? (m_ba < m_ab) : (da < db);
        if (ba) { take(b); take(a); } else { take(a); take(b); }
    }
    if (lane < n) orders_out[off + lane] = st.my_ot;
    if (lane == 0) {
        if (ms_out) ms_out[g] = st.tD;
        if (status) status[g] = 0;
    }
}

// Algorithm 1 for group g by one full warp.
__device__ __forceinline__ void heuristic_group(const tm_task* __restrict__ tasks, int off, int n,
                                                int dma, int g, int lane,
                                                int32_t* __restrict__ orders_out,
                                                int32_t* __restrict__ ms_out,
                                                int32_t* __restrict__ status)
{
    heuristic_group_seg<32>(tasks, off, n, dma, g, lane, orders_out, ms_out, status);
}

}  // namespace heur
}  // namespace tmgpu

// refine.cuh -- exact-model descent over task orders: starting from a given
// order, repeatedly apply the single move (a swap of two positions, or one
// task taken out and reinserted elsewhere) that lowers the model's makespan
// the most, until no move lowers it.  The paper has no such step; it
// polishes the orders of the heuristic (Sec. 5.1) and of the learned beam
// search, and every makespan it compares is the model's exact int32 value
// (the recurrence of tm_device.cuh), so it never makes an order worse.
//
// Moves of a group of n tasks, in the order that settles ties (the lowest
// index wins among equal makespans):
//   swaps       (i, j), i < j < n, by j then i            n (n - 1) / 2 moves
//   insertions  (i, j), |i - j| >= 2, max(i, j) < n: the task at position i
//               is removed and reinserted so that it ends at position j;
//               ordered by max(i, j), then i, then j      (n - 1) (n - 2) moves
// (moving a task by one position is the adjacent swap, so insertions start at
// a distance of two).  Both lists are ordered so that the moves of a smaller
// group are a prefix of the moves of a larger one.
//
// One warp runs one descent: each lane evaluates every 32nd move from the
// engine state of the current order just before the first position the move
// changes (prefix states kept in shared memory), the warp takes the best,
// applies it, and repeats; at most kMaxPasses moves are applied.
#pragma once

#include "tm_device.cuh"

namespace tmgpu {
namespace refine {

constexpr int kMaxPasses = 64;
constexpr int kSwaps16 = 120;   // 16 * 15 / 2
constexpr int kIns16 = 210;     // 15 * 14

struct MoveTable {
    uint8_t si[kSwaps16], sj[kSwaps16];
    uint8_t ii[kIns16], ij[kIns16];
};
constexpr MoveTable make_moves()
{
    MoveTable t{};
    int s = 0;
    for (int j = 1; j < 16; ++j)
        for (int i = 0; i < j; ++i) {
            t.si[s] = (uint8_t)i;
            t.sj[s] = (uint8_t)j;
            ++s;
        }
    int q = 0;
    for (int m = 0; m < 16; ++m)
        for (int i = 0; i <= m; ++i)
            for (int j = 0; j <= m; ++j) {
                const int d = i > j ? i - j : j - i;
                if ((i == m || j == m) && d >= 2) {
                    t.ii[q] = (uint8_t)i;
                    t.ij[q] = (uint8_t)j;
                    ++q;
                }
            }
    return t;
}
__constant__ MoveTable c_moves = make_moves();

__host__ __device__ inline int swap_moves(int n) { return n * (n - 1) / 2; }
__host__ __device__ inline int ins_moves(int n) { return n < 2 ? 0 : (n - 1) * (n - 2); }

__device__ __forceinline__ uint64_t nib_mask(int k)   // the low k nibbles
{
    return k >= 16 ? ~0ull : ((1ull << (4 * k)) - 1ull);
}

// The order (task at position p in bits 4p .. 4p + 3) after move m of a
// group of n tasks; *lo is the first position the move changes.
__device__ __forceinline__ uint64_t apply_move(uint64_t o, int n, int m, int* lo)
{
    const int S = swap_moves(n);
    if (m < S) {
        const int i = c_moves.si[m], j = c_moves.sj[m];
        const uint64_t x = ((o >> (4 * i)) ^ (o >> (4 * j))) & 0xFull;
        *lo = i;
        return o ^ (x << (4 * i)) ^ (x << (4 * j));
    }
    const int i = c_moves.ii[m - S], j = c_moves.ij[m - S];
    const uint64_t e = (o >> (4 * i)) & 0xFull;
    if (i < j) {   // positions i .. j - 1 take the tasks of i + 1 .. j; j takes e
        *lo = i;
        const uint64_t mid = ((o >> (4 * (i + 1))) & nib_mask(j - i)) << (4 * i);
        return (o & nib_mask(i)) | mid | (e << (4 * j)) | (o & ~nib_mask(j + 1));
    }
    // j < i: positions j + 1 .. i take the tasks of j .. i - 1; j takes e
    *lo = j;
    const uint64_t mid = ((o >> (4 * j)) & nib_mask(i - j)) << (4 * (j + 1));
    return (o & nib_mask(j)) | (e << (4 * j)) | mid | (o & ~nib_mask(i + 1));
}

// Makespan of order o from position `from` on, starting in state s.
__device__ __forceinline__ int32_t finish_order(uint64_t o, int n, int from, Eng s,
                                                const int4* __restrict__ rows)
{
    for (int p = from; p < n; ++p) {
        const int4 r = rows[(o >> (4 * p)) & 0xFull];
        s = step(s, r.x, r.y, r.z);
    }
    return s.d;
}

// Descent of one warp from order *o (makespan *ms on entry and exit).  rows:
// the group's task rows {htd, k, dth, 0} in shared memory; pre: this warp's
// n + 1 prefix states in shared memory.  Every lane passes the same values
// and leaves with the same result.
__device__ inline void descend(uint64_t* o, int32_t* ms, int n, int32_t dinit,
                               const int4* __restrict__ rows, int4* __restrict__ pre, int lane)
{
    const unsigned full = 0xFFFFFFFFu;
    const int M = swap_moves(n) + ins_moves(n);
    for (int pass = 0; pass < kMaxPasses && M > 0; ++pass) {
        // state after the first p positions of the current order
        if (lane <= n) {
            Eng s{0, 0, dinit};
            for (int p = 0; p < lane; ++p) {
                const int4 r = rows[(*o >> (4 * p)) & 0xFull];
                s = step(s, r.x, r.y, r.z);
            }
            pre[lane] = make_int4(s.h, s.k, s.d, 0);
        }
        __syncwarp();
        int32_t best = INT32_MAX;
        uint32_t best_m = 0xFFFFFFFFu;
        for (int m = lane; m < M; m += 32) {
            int lo = 0;
            const uint64_t om = apply_move(*o, n, m, &lo);
            const int4 q = pre[lo];
            const int32_t v = finish_order(om, n, lo, Eng{q.x, q.y, q.z}, rows);
            if (v < best) { best = v; best_m = (uint32_t)m; }
        }
        __syncwarp();
        const int32_t vmin = (int32_t)__reduce_min_sync(full, (unsigned)best);
        const uint32_t mmin = __reduce_min_sync(full, best == vmin ? best_m : 0xFFFFFFFFu);
        if (vmin >= *ms) break;
        int lo = 0;
        *o = apply_move(*o, n, (int)mmin, &lo);
        *ms = vmin;
    }
}

}  // namespace refine
}  // namespace tmgpu

// chain.cu -- chained tasks (Sec. 6.1, experiment setup): T workers each
// submit a chain of N dependent tasks, and a worker's next task is released
// only when its previous one has completely finished.  The paper counts
// (T!)^N orders: the group runs as N rounds in sequence, round r holding the
// r-th task of every worker in some order.  Task index r * T + w is worker
// w's round-r task; an order lists the n = T * N task indices round by round.
//
// Model.  The FIFO queues of the plain model (tm_device.cuh), filled in
// order, with one more dependency: the HtD of worker w's round-r task starts
// only after the DtH of its round-(r - 1) task, whose end c_w is known when
// round r starts.  Appending worker w's task of the current round:
//     h' = max(h, c_w) + htd      k' = max(k, h') + k      d' = max(d, k') + dth
// With one DMA engine each round is submitted as a group of its own (its
// HtDs, then its DtHs, in the one transfer queue), so when round r starts
// the transfer engine is free at d, every c_w <= d, and the round's first
// DtH cannot start before its last HtD:  h = d,  d = d + (sum of the round's
// HtDs).  All values stay below the group's duration sum, checked to fit in
// int32.
//
// Enumeration.  Orders are ranked lexicographically, i.e. as a counter whose
// digits are the rounds' permutations (round 0 most significant).  The last
// m = min(T, 4) positions (the tail, all in the last round) vary fastest, so
// a BLOCK of m! consecutive ranks shares the first n - m positions.  A
// thread takes a contiguous range of blocks: it unranks the first one,
// evaluates the tail's m! orders straight-line (depth-first, the engine
// state of each tail prefix shared), advances the counter to the next block
// (a nibble-packed next-permutation of the last round's head, carrying into
// earlier rounds) and recomputes the engine states from the first changed
// position only, from per-position snapshots.  Per-thread best / worst with
// the first rank and the exact sum go to per-group 64-bit key atomics.
//
// Groups of 2 <= T <= 4 workers and at least two rounds take a faster path
// (chain_small_kernel): there the tail is the whole last round, so its rows
// and release times sit in registers under compile-time indices, and a unit
// of work is one prefix of the first R - 2 rounds, (T!)^2 orders, with round
// R - 2's permutations read from a table.
//
//   chain_prep_kernel      per group: checks, reduction words
//   chain_tail_kernel      per group of four workers: the closed-form table
//   chain_enum_kernel      every order of every other group
//   chain_small_kernel<T>  every order of the groups of T = 2, 3, 4 workers
//   chain_finalize_kernel  reduction words -> tm_stats (orders unranked)
//   chain_predict_kernel   one given order per group
#include <algorithm>
#include <climits>
#include <vector>

#include "tm_device.cuh"

namespace tmgpu {
namespace {

constexpr int kChainBlock = 128;
constexpr int kChainMaxWorkers = 8;

struct ChainInfo {
    int32_t off;      // first task
    int32_t T;        // workers
    int32_t R;        // rounds
    int32_t dma;      // 1 or 2
    int32_t status;   // 0 or a tm_status code
    int32_t pad[3];
};

__host__ __device__ inline int chain_tail(int T) { return T < 4 ? T : 4; }

// (T!)^R orders, or 0 for a shape outside 1 <= T <= 8, T * R <= 16.
__host__ __device__ inline uint64_t chain_orders(int T, int R)
{
    if (T < 1 || T > kChainMaxWorkers || R < 1 || T * R > TM_MAX_TASKS) return 0;
    uint64_t c = 1;
    for (int r = 0; r < R; ++r) c *= factorial_u64(T);
    return c;
}

// Per-group checks (shape, durations, device model); 0 or a tm_status code.
__device__ int check_chain(const tm_task* tasks, int n, int T, int dma)
{
    if (T < 1 || T > kChainMaxWorkers || n < 1 || n > TM_MAX_TASKS || n % T != 0)
        return TM_EINVAL;
    int32_t hs = 0, dinit = 0;
    return check_group(tasks, n, dma, TM_MAX_TASKS, &hs, &dinit);
}

__device__ __forceinline__ Eng step_c(Eng s, int32_t c, int4 t)
{
    Eng r;
    r.h = max(s.h, c) + t.x;
    r.k = max(s.k, r.h) + t.y;
    r.d = max(s.d, r.k) + t.z;
    return r;
}

__device__ __forceinline__ uint32_t nib32(uint32_t w, int i) { return (w >> (4 * i)) & 0xFu; }

// Lexicographic next permutation of the T nibbles of w.  Returns the index
// of the first changed nibble, or -1 when w was the last permutation (it is
// then reset to the first, ascending).
__device__ int next_perm_nib(uint32_t& w, int T)
{
    int i = T - 2;
    while (i >= 0 && nib32(w, i) >= nib32(w, i + 1)) --i;
    if (i < 0) {
        uint32_t a = 0;
        for (int e = 0; e < T; ++e) a |= (uint32_t)e << (4 * e);
        w = a;
        return -1;
    }
    int j = T - 1;
    while (nib32(w, j) <= nib32(w, i)) --j;
    const uint32_t x = (nib32(w, i) ^ nib32(w, j));
    w ^= (x << (4 * i)) | (x << (4 * j));
    for (int a = i + 1, b = T - 1; a < b; ++a, --b) {   // reverse i + 1 .. T - 1
        const uint32_t y = nib32(w, a) ^ nib32(w, b);
        w ^= (y << (4 * a)) | (y << (4 * b));
    }
    return i;
}

// Permutation of T workers with lexicographic rank q (q < T!), as nibbles.
__device__ uint32_t unrank_round(uint32_t q, int T)
{
    uint64_t list = nib_identity(T);
    uint32_t w = 0;
    for (int i = 0; i < T; ++i) {
        const int k = T - 1 - i;
        const uint32_t c = min(div_fact(q, k), (uint32_t)k);
        q -= c * (uint32_t)factorial_u64(k);
        w |= (uint32_t)nib_get(list, (int)c) << (4 * i);
        list = nib_remove(list, (int)c);
    }
    return w;
}

__device__ __forceinline__ uint32_t inverse_nib(uint32_t w, int T)
{
    uint32_t inv = 0;
    for (int i = 0; i < T; ++i) inv |= (uint32_t)i << (4 * nib32(w, i));
    return inv;
}

// The last round's 24 orders (four workers) when the HtD engine's path ends
// every one of them.  The recurrence is max-plus linear in the state
// (h, k, d) entering the round and the release times c_w, so order sigma
// ends at
//     max(h + G_sigma, k + B_sigma, d + alpha, max_w (c_w + Dw_sigma))
// with G, B, Dw the longest paths through the round from the HtD engine,
// the K engine and worker w's release, and alpha the round's DtH sum, all
// fixed by the group.  When h - d >= alpha - min G, h - k >= max (B - G) and
// c_w - h <= min (G - Dw) for every w, each order ends at h + G_sigma: the
// 24 makespans are h + G, their minimum h + min G at the first sigma reaching
// it, and so on.
struct HtdTail {
    int32_t td, tk, tc[4];
    int32_t gmin, gmax;
    uint32_t imin, imax;   // lexicographic index of the first sigma reaching them
    unsigned long long gsum;
};


__global__ void chain_prep_kernel(const tm_task* __restrict__ tasks,
                                  const int32_t* __restrict__ offsets,
                                  const int32_t* __restrict__ workers, int G,
                                  const tm_device* __restrict__ devs, ChainInfo* __restrict__ info,
                                  unsigned long long* __restrict__ acc, int32_t* __restrict__ status)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    const int off = offsets[g], n = offsets[g + 1] - off, T = workers[g];
    const int dma = devs[g].dma_engines;
    const int rc = check_chain(tasks + off, n, T, dma);
    ChainInfo ci;
    ci.off = off;
    ci.T = T;
    ci.R = rc == 0 ? n / T : 0;
    ci.dma = dma;
    ci.status = rc;
    ci.pad[0] = ci.pad[1] = ci.pad[2] = 0;
    info[g] = ci;
    acc[4 * (size_t)g + 0] = ~0ull;
    acc[4 * (size_t)g + 1] = 0ull;
    acc[4 * (size_t)g + 2] = 0ull;
    if (status && rc != 0) status[g] = rc;
}

// One thread's view of one group: the current order (worker of every
// position, nibbles), the engine state after every position, the inverse of
// every round, and the last round's task rows with their release times c_w.
struct ChainWalk {
    int T, R, n, m, dma, off;
    uint64_t seq;            // worker at position p in bits 4p .. 4p + 3
    int32_t sh[TM_MAX_TASKS], sk[TM_MAX_TASKS], sd[TM_MAX_TASKS];
    uint32_t inv[TM_MAX_TASKS];
};

// Sum of the HtDs of round r.
__device__ __forceinline__ int32_t round_htd(const tm_task* __restrict__ tasks, int off, int T,
                                             int r)
{
    int32_t s = 0;
    for (int w = 0; w < T; ++w) s += tasks[off + r * T + w].htd;
    return s;
}

// Recomputes the states from position p0 up to the start of the tail
// (n - m), entering rounds on the way; when it enters the last round it
// refills the last round's rows (with c_w) in `last`.  Returns the state at
// the start of the tail.
__device__ Eng chain_resume(ChainWalk& cw, int p0, const tm_task* __restrict__ tasks,
                            int4* __restrict__ last)
{
    const int T = cw.T, head_end = cw.n - cw.m, last_start = (cw.R - 1) * T;
    Eng s = p0 == 0 ? Eng{0, 0, 0} : Eng{cw.sh[p0 - 1], cw.sk[p0 - 1], cw.sd[p0 - 1]};
    // the round that starts at position p (p == r T) is entered before p
    auto enter = [&](int r) {
        if (cw.dma == 1) {
            s.h = s.d;
            s.d += round_htd(tasks, cw.off, T, r);
        }
        if (r == cw.R - 1) {
            for (int w = 0; w < T; ++w) {
                const tm_task t = tasks[cw.off + r * T + w];
                const int32_t c = r == 0 ? 0 : cw.sd[(r - 1) * T + min((int)nib32(cw.inv[r - 1], w), T - 1)];
                last[w * kChainBlock] = make_int4(t.htd, t.k, t.dth, c);
            }
        }
    };
    for (int p = p0; p < head_end; ++p) {
        const int r = p / T, i = p - r * T;
        if (i == 0) enter(r);
        const int w = (int)((cw.seq >> (4 * p)) & 0xF);
        int4 row;
        if (r == cw.R - 1) {
            row = last[w * kChainBlock];
        } else {
            const tm_task t = tasks[cw.off + r * T + w];
            const int32_t c = r == 0 ? 0 : cw.sd[(r - 1) * T + min((int)nib32(cw.inv[r - 1], w), T - 1)];
            row = make_int4(t.htd, t.k, t.dth, c);
        }
        s = step_c(s, row.w, row);
        cw.sh[p] = s.h;
        cw.sk[p] = s.k;
        cw.sd[p] = s.d;
        if (i == T - 1)
            cw.inv[r] = inverse_nib((uint32_t)(cw.seq >> (4 * r * T)) & (T >= 8 ? 0xFFFFFFFFu : ((1u << (4 * T)) - 1u)), T);
    }
    if (head_end == last_start && p0 <= head_end) enter(cw.R - 1);   // no head in the last round
    return s;
}

// Per-thread reduction of one group.
struct ChainAcc {
    int32_t best, worst;
    uint32_t brank, wrank;
    unsigned long long sum;
};

__device__ __forceinline__ void take_pair(ChainAcc& a, int32_t m0, int32_t m1, uint32_t rank)
{
    const int32_t mn = min(m0, m1), mx = max(m0, m1);
    if (mn < a.best) { a.best = mn; a.brank = rank + (m0 != mn); }
    if (mx > a.worst) { a.worst = mx; a.wrank = rank + (m0 != mx); }
    a.sum += (unsigned long long)((uint32_t)m0 + (uint32_t)m1);
}

__device__ __forceinline__ void take_one(ChainAcc& a, int32_t m0, uint32_t rank)
{
    if (m0 < a.best) { a.best = m0; a.brank = rank; }
    if (m0 > a.worst) { a.worst = m0; a.wrank = rank; }
    a.sum += (unsigned long long)(uint32_t)m0;
}

// The two orders of the last two workers u < v from state s.
__device__ __forceinline__ void tail2(Eng s, const int4* __restrict__ last, int u, int v,
                                      ChainAcc& a, uint32_t rank)
{
    const int4 ru = last[u * kChainBlock], rv = last[v * kChainBlock];
    const int32_t m_uv = step_c(step_c(s, ru.w, ru), rv.w, rv).d;
    const int32_t m_vu = step_c(step_c(s, rv.w, rv), ru.w, ru).d;
    take_pair(a, m_uv, m_vu, rank);
}

// The 6 orders of workers a < b < c (lexicographic: abc acb bac bca cab cba).
__device__ __forceinline__ void tail3(Eng s, const int4* __restrict__ last, int x0, int x1,
                                      int x2, ChainAcc& a, uint32_t rank)
{
    const int4 r0 = last[x0 * kChainBlock], r1 = last[x1 * kChainBlock],
               r2 = last[x2 * kChainBlock];
    tail2(step_c(s, r0.w, r0), last, x1, x2, a, rank);
    tail2(step_c(s, r1.w, r1), last, x0, x2, a, rank + 2);
    tail2(step_c(s, r2.w, r2), last, x0, x1, a, rank + 4);
}

__device__ __forceinline__ void tail4(Eng s, const int4* __restrict__ last, int x0, int x1,
                                      int x2, int x3, ChainAcc& a, uint32_t rank)
{
    const int4 r0 = last[x0 * kChainBlock], r1 = last[x1 * kChainBlock],
               r2 = last[x2 * kChainBlock], r3 = last[x3 * kChainBlock];
    tail3(step_c(s, r0.w, r0), last, x1, x2, x3, a, rank);
    tail3(step_c(s, r1.w, r1), last, x0, x2, x3, a, rank + 6);
    tail3(step_c(s, r2.w, r2), last, x0, x1, x3, a, rank + 12);
    tail3(step_c(s, r3.w, r3), last, x0, x1, x2, a, rank + 18);
}

// The same tails with the rows in registers.
__device__ __forceinline__ void tail2_regs(Eng s, int4 ru, int4 rv, ChainAcc& a, uint32_t rank)
{
    const int32_t m_uv = step_c(step_c(s, ru.w, ru), rv.w, rv).d;
    const int32_t m_vu = step_c(step_c(s, rv.w, rv), ru.w, ru).d;
    take_pair(a, m_uv, m_vu, rank);
}

__device__ void flush(ChainAcc& a, unsigned long long* __restrict__ acc, int g)
{
    if (a.best == INT32_MAX) return;
    atomicMin(&acc[4 * (size_t)g + 0],
              ((unsigned long long)(uint32_t)a.best << 32) | a.brank);
    atomicMax(&acc[4 * (size_t)g + 1],
              ((unsigned long long)(uint32_t)a.worst << 32) | (0xFFFFFFFFu - a.wrank));
    atomicAdd(&acc[4 * (size_t)g + 2], a.sum);
    a = ChainAcc{INT32_MAX, -1, 0u, 0u, 0ull};
}

// flush() by a whole warp whose lanes all hold group g: one set of atomics
// for the warp (else each lane's own).
__device__ void flush_warp(ChainAcc& a, unsigned long long* __restrict__ acc, int g)
{
    const unsigned live = __activemask();
    if (live != 0xFFFFFFFFu || !__all_sync(live, g == __shfl_sync(live, g, 0))) {
        flush(a, acc, g);
        return;
    }
    const bool any = a.best != INT32_MAX;
    unsigned long long bk = any ? (((unsigned long long)(uint32_t)a.best << 32) | a.brank) : ~0ull;
    unsigned long long wk =
        any ? (((unsigned long long)(uint32_t)a.worst << 32) | (0xFFFFFFFFu - a.wrank)) : 0ull;
    unsigned long long sum = a.sum;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long b2 = __shfl_xor_sync(live, bk, o);
        const unsigned long long w2 = __shfl_xor_sync(live, wk, o);
        bk = b2 < bk ? b2 : bk;
        wk = w2 > wk ? w2 : wk;
        sum += __shfl_xor_sync(live, sum, o);
    }
    if ((threadIdx.x & 31) == 0 && bk != ~0ull) {
        atomicMin(&acc[4 * (size_t)g + 0], bk);
        atomicMax(&acc[4 * (size_t)g + 1], wk);
        atomicAdd(&acc[4 * (size_t)g + 2], sum);
    }
    a = ChainAcc{INT32_MAX, -1, 0u, 0u, 0ull};
}

__global__ void __launch_bounds__(kChainBlock)
chain_enum_kernel(const unsigned long long* __restrict__ block_base, int G,
                  const ChainInfo* __restrict__ info, const tm_task* __restrict__ tasks,
                  unsigned long long* __restrict__ acc, unsigned long long per_thread)
{
    __shared__ int4 s_last[kChainMaxWorkers * kChainBlock];
    int4* last = s_last + threadIdx.x;
    const unsigned long long total = block_base[G];
    const unsigned long long t = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long b = t * per_thread;
    const unsigned long long b_end = min(total, b + per_thread);
    if (b >= b_end) return;
    int g = 0;
    {   // the last group whose first block is <= b
        int lo = 0, hi = G;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (block_base[mid] <= b) lo = mid; else hi = mid;
        }
        g = lo;
    }
    ChainWalk cw;
    ChainAcc a{INT32_MAX, -1, 0u, 0u, 0ull};
    while (b < b_end) {
        while (b >= block_base[g + 1]) ++g;   // groups without orders have no blocks
        const ChainInfo ci = info[g];
        if (ci.status != 0) {                 // rejected by the prep kernel
            b = min(b_end, (unsigned long long)block_base[g + 1]);
            continue;
        }
        cw.T = ci.T;
        cw.R = ci.R;
        cw.n = ci.T * ci.R;
        cw.m = chain_tail(ci.T);
        cw.dma = ci.dma;
        cw.off = ci.off;
        const int T = cw.T, m = cw.m;
        // unrank the group's block b - base: rank (b - base) m!, round by round
        const uint32_t F = (uint32_t)factorial_u64(T);
        const uint32_t mf = (uint32_t)factorial_u64(m);
        uint32_t rank = (uint32_t)(b - block_base[g]) * mf;
        {
            uint32_t q = rank;
            cw.seq = 0;
            for (int r = cw.R - 1; r >= 0; --r) {
                const uint32_t digit = q % F;
                q /= F;
                cw.seq |= (uint64_t)unrank_round(digit, T) << (4 * r * T);
            }
        }
        const unsigned long long g_end = min(b_end, (unsigned long long)block_base[g + 1]);
        Eng s = chain_resume(cw, 0, tasks, last);
        const int head_end = cw.n - m, last_start = (cw.R - 1) * T;
        for (;;) {
            // the tail: the last round's workers not in its head, ascending
            uint32_t freew = (1u << T) - 1u;
            for (int p = last_start; p < head_end; ++p) freew &= ~(1u << ((cw.seq >> (4 * p)) & 0xF));
            const int x0 = __ffs(freew) - 1;
            freew &= freew - 1;
            if (m == 4) {
                const int x1 = __ffs(freew) - 1; freew &= freew - 1;
                const int x2 = __ffs(freew) - 1; freew &= freew - 1;
                const int x3 = __ffs(freew) - 1;
                tail4(s, last, x0, x1, x2, x3, a, rank);
            } else if (m == 3) {
                const int x1 = __ffs(freew) - 1; freew &= freew - 1;
                const int x2 = __ffs(freew) - 1;
                tail3(s, last, x0, x1, x2, a, rank);
            } else if (m == 2) {
                tail2(s, last, x0, __ffs(freew) - 1, a, rank);
            } else {
                const int4 r0 = last[x0 * kChainBlock];
                take_one(a, step_c(s, r0.w, r0).d, rank);
            }
            rank += mf;
            if (++b >= g_end) break;
            // next block: the last round's head advances (its tail taken as
            // descending, i.e. exhausted); a round that wraps carries into
            // the round before it
            int p0 = -1;
            for (int r = cw.R - 1; r >= 0 && p0 < 0; --r) {
                uint32_t w = (uint32_t)(cw.seq >> (4 * r * T)) &
                             (T >= 8 ? 0xFFFFFFFFu : ((1u << (4 * T)) - 1u));
                if (r == cw.R - 1) {
                    // tail descending: reverse its ascending nibbles
                    for (int x = T - m, y = T - 1; x < y; ++x, --y) {
                        const uint32_t z = nib32(w, x) ^ nib32(w, y);
                        w ^= (z << (4 * x)) | (z << (4 * y));
                    }
                }
                const int i = next_perm_nib(w, T);
                const uint64_t maskr = (T >= 8 ? 0xFFFFFFFFull : ((1ull << (4 * T)) - 1ull)) << (4 * r * T);
                cw.seq = (cw.seq & ~maskr) | ((uint64_t)w << (4 * r * T));
                if (i >= 0) p0 = r * T + i;
            }
            s = chain_resume(cw, p0, tasks, last);
        }
        flush(a, acc, g);
    }
}

// ---- fast path: 2 <= T <= 4 workers, R >= 2 rounds --------------------------
//
// With T <= 4 the tail is the whole last round, so its workers are 0 .. T-1
// in every block: the last round's rows and release times can live in
// registers under compile-time indices.  A unit of work is one prefix of the
// first R - 2 rounds; the thread replays it once, then walks the T!
// permutations of round R - 2 in lexicographic order from a table (each
// recomputes only from the first position that differs from the previous
// one) and, for each, the T! orders of the last round straight-line:
// (T!)^2 consecutive ranks per unit.

// Permutations of 0 .. T-1 in lexicographic order (nibbles), the first
// position where each differs from the one before, and their inverses.
struct SmallPerms {
    uint16_t perm[3][24], inv[3][24];
    uint8_t pivot[3][24];
};
constexpr SmallPerms make_small_perms()
{
    SmallPerms t{};
    for (int T = 2; T <= 4; ++T) {
        int a[4] = {0, 1, 2, 3};
        int prev[4] = {0, 1, 2, 3};
        for (int q = 0;; ++q) {
            uint16_t pw = 0, iw = 0;
            int piv = 0;
            for (int i = 0; i < T; ++i) {
                pw |= (uint16_t)(a[i] << (4 * i));
                iw |= (uint16_t)(i << (4 * a[i]));
            }
            if (q > 0) {
                piv = T;
                for (int i = T - 1; i >= 0; --i)
                    if (a[i] != prev[i]) piv = i;
            }
            t.perm[T - 2][q] = pw;
            t.inv[T - 2][q] = iw;
            t.pivot[T - 2][q] = (uint8_t)piv;
            for (int i = 0; i < T; ++i) prev[i] = a[i];
            // next permutation
            int i = T - 2;
            while (i >= 0 && a[i] >= a[i + 1]) --i;
            if (i < 0) break;
            int j = T - 1;
            while (a[j] <= a[i]) --j;
            const int x = a[i]; a[i] = a[j]; a[j] = x;
            for (int l = i + 1, r = T - 1; l < r; ++l, --r) { const int y = a[l]; a[l] = a[r]; a[r] = y; }
        }
    }
    return t;
}
__constant__ SmallPerms c_small = make_small_perms();

// Element w (0 <= w < T) of a register array, by selects.
template <int T>
__device__ __forceinline__ int32_t pick(const int32_t (&v)[T], int w)
{
    int32_t r = v[0];
#pragma unroll
    for (int i = 1; i < T; ++i) r = w == i ? v[i] : r;
    return r;
}

template <int T>
__device__ __forceinline__ int4 pick4(const int4 (&v)[T], int w)
{
    int4 r = v[0];
#pragma unroll
    for (int i = 1; i < T; ++i) r = w == i ? v[i] : r;
    return r;
}

// The fast path's additions run as multiply-adds by `one` (a kernel
// parameter, always 1), so that they issue on the FMA pipe beside the ALU
// pipe's maxima; the values are those of plain additions.
__device__ __forceinline__ int32_t fadd(int32_t x, int32_t y, uint32_t one)
{
    return (int32_t)((uint32_t)x * one + (uint32_t)y);
}

__device__ __forceinline__ Eng step_f(Eng s, int32_t c, int4 t, uint32_t one)
{
    Eng r;
    r.h = fadd(max(s.h, c), t.x, one);
    r.k = fadd(max(s.k, r.h), t.y, one);
    r.d = fadd(max(s.d, r.k), t.z, one);
    return r;
}

// The last two positions in closed form.  From state (h, k, d), appending
// worker x then worker y (release times c_x, c_y) ends at
//     max(d + A_xy, k + P_xy, h + Q_xy, R_xy)
// with A_xy = D_x + D_y, P_xy = K_x + max(D_x, K_y) + D_y,
// Q_xy = H_x + max(P_xy, C_y), C_y = H_y + K_y + D_y, and
// R_xy = max(c_x + Q_xy, c_y + C_y): the two recurrence steps written as the
// longest of the paths through them.  A, P and Q depend only on the group's
// last round; R on the release times.
struct Pair4 {
    int32_t A[4][4], P[4][4], Q[4][4], C[4];
};

__device__ __forceinline__ void pair4_setup(const int4 (&lr)[4], Pair4& q)
{
#pragma unroll
    for (int y = 0; y < 4; ++y) q.C[y] = lr[y].x + lr[y].y + lr[y].z;
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) {
            if (x == y) continue;
            q.A[x][y] = lr[x].z + lr[y].z;
            q.P[x][y] = lr[x].y + max(lr[x].z, lr[y].y) + lr[y].z;
            q.Q[x][y] = lr[x].x + max(q.P[x][y], q.C[y]);
        }
}

// The two orders of the last two workers x < y from state s.
template <int X, int Y>
__device__ __forceinline__ void tail2_pair(Eng s, const Pair4& q, const int32_t (&E)[4],
                                           const int32_t (&c)[4], ChainAcc& a, uint32_t rank,
                                           uint32_t one)
{
    const int32_t r_xy = max(fadd(c[X], q.Q[X][Y], one), E[Y]);
    const int32_t r_yx = max(fadd(c[Y], q.Q[Y][X], one), E[X]);
    const int32_t m_xy = max(max(fadd(s.d, q.A[X][Y], one), fadd(s.k, q.P[X][Y], one)),
                             max(fadd(s.h, q.Q[X][Y], one), r_xy));
    const int32_t m_yx = max(max(fadd(s.d, q.A[Y][X], one), fadd(s.k, q.P[Y][X], one)),
                             max(fadd(s.h, q.Q[Y][X], one), r_yx));
    take_pair(a, m_xy, m_yx, rank);
}

// The 24 orders of the last round's four workers from state s (rows with
// release times in lr; E[y] = c_y + C_y).
__device__ __forceinline__ void tail4_pair(Eng s, const int4 (&lr)[4], const Pair4& q,
                                           ChainAcc& a, uint32_t rank, uint32_t one)
{
    int32_t c[4], E[4];
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        c[w] = lr[w].w;
        E[w] = fadd(c[w], q.C[w], one);
    }
    // first worker 0
    {
        const Eng s0 = step_f(s, c[0], lr[0], one);
        tail2_pair<2, 3>(step_f(s0, c[1], lr[1], one), q, E, c, a, rank, one);
        tail2_pair<1, 3>(step_f(s0, c[2], lr[2], one), q, E, c, a, rank + 2, one);
        tail2_pair<1, 2>(step_f(s0, c[3], lr[3], one), q, E, c, a, rank + 4, one);
    }
    {
        const Eng s1 = step_f(s, c[1], lr[1], one);
        tail2_pair<2, 3>(step_f(s1, c[0], lr[0], one), q, E, c, a, rank + 6, one);
        tail2_pair<0, 3>(step_f(s1, c[2], lr[2], one), q, E, c, a, rank + 8, one);
        tail2_pair<0, 2>(step_f(s1, c[3], lr[3], one), q, E, c, a, rank + 10, one);
    }
    {
        const Eng s2 = step_f(s, c[2], lr[2], one);
        tail2_pair<1, 3>(step_f(s2, c[0], lr[0], one), q, E, c, a, rank + 12, one);
        tail2_pair<0, 3>(step_f(s2, c[1], lr[1], one), q, E, c, a, rank + 14, one);
        tail2_pair<0, 1>(step_f(s2, c[3], lr[3], one), q, E, c, a, rank + 16, one);
    }
    {
        const Eng s3 = step_f(s, c[3], lr[3], one);
        tail2_pair<1, 2>(step_f(s3, c[0], lr[0], one), q, E, c, a, rank + 18, one);
        tail2_pair<0, 2>(step_f(s3, c[1], lr[1], one), q, E, c, a, rank + 20, one);
        tail2_pair<0, 1>(step_f(s3, c[2], lr[2], one), q, E, c, a, rank + 22, one);
    }
}


// The T! orders of the last round's workers 0 .. T-1 from state s, in
// lexicographic order: ranks rank, rank + 1, ...  (T = 4 takes tail4_pair.)
template <int T>
__device__ __forceinline__ void tail_static(Eng s, const int4 (&lr)[T], ChainAcc& a, uint32_t rank)
{
    static_assert(T == 2 || T == 3, "two or three workers");
    if constexpr (T == 2) {
        const int32_t m01 = step_c(step_c(s, lr[0].w, lr[0]), lr[1].w, lr[1]).d;
        const int32_t m10 = step_c(step_c(s, lr[1].w, lr[1]), lr[0].w, lr[0]).d;
        take_pair(a, m01, m10, rank);
    } else {
        const int4 x[3] = {lr[0], lr[1], lr[2]};
        tail2_regs(step_c(s, x[0].w, x[0]), x[1], x[2], a, rank);
        tail2_regs(step_c(s, x[1].w, x[1]), x[0], x[2], a, rank + 2);
        tail2_regs(step_c(s, x[2].w, x[2]), x[0], x[1], a, rank + 4);
    }
}

// The closed-form table (HtdTail) of every group of four workers and at
// least two rounds, a warp per group: lane q < 24 takes the q-th order of
// the last round (lexicographic), follows the paths from the HtD engine, the
// K engine and each worker's release through it (64-bit, with unreached
// sources far below any time), and the warp reduces: G's minimum and
// maximum with their first order, its sum, max (B - G) and min (G - Dw).
__global__ void chain_tail_kernel(const ChainInfo* __restrict__ info,
                                  const tm_task* __restrict__ tasks, int G,
                                  HtdTail* __restrict__ tails)
{
    const int g = (int)(((unsigned)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (g >= G) return;   // whole warps
    const ChainInfo ci = info[g];
    if (ci.status != 0 || ci.T != 4 || ci.R < 2) return;
    constexpr long long kNeg = -(1ll << 40);
    const bool live = lane < 24;
    long long G_ = 0, tk = LLONG_MIN, tc[4] = {LLONG_MAX, LLONG_MAX, LLONG_MAX, LLONG_MAX};
    if (live) {
        const uint32_t pw = c_small.perm[2][lane];
        long long h[6], k[6], d[6];
        for (int q = 0; q < 6; ++q) {
            h[q] = q == 0 ? 0 : kNeg;
            k[q] = q == 1 ? 0 : kNeg;
            d[q] = kNeg;
        }
        for (int i = 0; i < 4; ++i) {
            const int w = (int)((pw >> (4 * i)) & 0xF);
            const tm_task t = tasks[ci.off + (ci.R - 1) * 4 + w];
            for (int q = 0; q < 6; ++q) {
                h[q] = max(h[q], q == 2 + w ? 0ll : kNeg) + t.htd;
                k[q] = max(k[q], h[q]) + t.k;
                d[q] = max(d[q], k[q]) + t.dth;
            }
        }
        G_ = d[0];
        tk = d[1] - G_;
        for (int w = 0; w < 4; ++w) tc[w] = G_ - d[2 + w];
    }
    // G < 2^31 and the order index < 32: (G, index) packed keeps the first order on ties
    unsigned long long kmin = live ? ((unsigned long long)G_ << 5) | (unsigned)lane : ~0ull;
    unsigned long long kmax = live ? ((unsigned long long)G_ << 5) | (31u - (unsigned)lane) : 0ull;
    unsigned long long sum = live ? (unsigned long long)G_ : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long a = __shfl_xor_sync(0xFFFFFFFFu, kmin, o);
        const unsigned long long b = __shfl_xor_sync(0xFFFFFFFFu, kmax, o);
        kmin = a < kmin ? a : kmin;
        kmax = b > kmax ? b : kmax;
        sum += __shfl_xor_sync(0xFFFFFFFFu, sum, o);
        tk = max(tk, __shfl_xor_sync(0xFFFFFFFFu, tk, o));
        for (int w = 0; w < 4; ++w) tc[w] = min(tc[w], __shfl_xor_sync(0xFFFFFFFFu, tc[w], o));
    }
    if (lane == 0) {
        long long alpha = 0;
        for (int w = 0; w < 4; ++w) alpha += tasks[ci.off + (ci.R - 1) * 4 + w].dth;
        HtdTail ht;
        ht.gmin = (int32_t)(kmin >> 5);
        ht.imin = (uint32_t)(kmin & 31u);
        ht.gmax = (int32_t)(kmax >> 5);
        ht.imax = 31u - (uint32_t)(kmax & 31u);
        ht.gsum = sum;
        ht.td = (int32_t)(alpha - (long long)ht.gmin);
        ht.tk = (int32_t)tk;
        for (int w = 0; w < 4; ++w) ht.tc[w] = (int32_t)tc[w];
        tails[g] = ht;
    }
}

template <int T>
__global__ void __launch_bounds__(kChainBlock)
chain_small_kernel(const unsigned long long* __restrict__ unit_base, int G,
                   const ChainInfo* __restrict__ info, const tm_task* __restrict__ tasks,
                   unsigned long long* __restrict__ acc, unsigned long long per_lane,
                   uint32_t one, unsigned long long* __restrict__ counts,
                   const HtdTail* __restrict__ tails, unsigned long long* __restrict__ next)
{
    constexpr int F = T == 2 ? 2 : T == 3 ? 6 : 24;
    uint32_t ntail = 0, nclosed = 0;   // four workers: tails walked, closed forms taken
    const unsigned long long total = unit_base[G];
    const int lane = threadIdx.x & 31;
    ChainAcc a{INT32_MAX, -1, 0u, 0u, 0ull};
    // Warps take batches of 32 per_lane consecutive units from *next in
    // turn (units cost unevenly: closed-form tails are cheap), lane l every
    // 32nd from the l-th, so that a warp's lanes walk neighbouring units
    // (one group) at once.
    for (;;) {
    unsigned long long b0 = 0;
    if (lane == 0) b0 = atomicAdd(next, 32ull * per_lane);
    b0 = __shfl_sync(0xFFFFFFFFu, b0, 0);
    if (b0 >= total) break;
    unsigned long long u = b0 + (unsigned long long)lane;
    const unsigned long long u_end = min(total, b0 + 32ull * per_lane);
    int g = 0;
    if (u < u_end) {
        int lo = 0, hi = G;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (unit_base[mid] <= u) lo = mid; else hi = mid;
        }
        g = lo;
    }
    while (u < u_end) {
        while (u >= unit_base[g + 1]) ++g;
        const ChainInfo ci = info[g];
        const unsigned long long g_end = min(u_end, (unsigned long long)unit_base[g + 1]);
        if (ci.status != 0 || ci.T != T || ci.R < 2) {   // rejected by the prep kernel
            u += (g_end - u + 31) / 32 * 32;   // the lane's next unit past the group
            continue;
        }
        const int R = ci.R;
        // the penultimate and last rounds' rows
        int4 prow[T], lrow[T];
        int32_t sh_pen = 0, sh_last = 0;
#pragma unroll
        for (int w = 0; w < T; ++w) {
            const tm_task p = tasks[ci.off + (R - 2) * T + w];
            const tm_task l = tasks[ci.off + (R - 1) * T + w];
            prow[w] = make_int4(p.htd, p.k, p.dth, 0);
            lrow[w] = make_int4(l.htd, l.k, l.dth, 0);
            sh_pen += p.htd;
            sh_last += l.htd;
        }
        Pair4 pq;
        HtdTail ht;
        if constexpr (T == 4) {
            pair4_setup(reinterpret_cast<const int4 (&)[4]>(lrow), pq);
            ht = tails[g];   // tabulated by chain_tail_kernel
        }
        for (; u < g_end; u += 32) {
            const uint32_t o = (uint32_t)(u - unit_base[g]);
            // replay rounds 0 .. R-3 of prefix o (digits base T!, round 0 first)
            Eng s{0, 0, 0};
            int32_t c[T];
#pragma unroll
            for (int w = 0; w < T; ++w) c[w] = 0;
            {
                uint32_t digits[TM_MAX_TASKS];
                uint32_t q = o;
                for (int r = R - 3; r >= 0; --r) { digits[r] = q % F; q /= F; }
                for (int r = 0; r <= R - 3; ++r) {
                    const uint32_t pw = c_small.perm[T - 2][digits[r]];
                    const uint32_t iw = c_small.inv[T - 2][digits[r]];
                    if (ci.dma == 1) {
                        s.h = s.d;
                        for (int w = 0; w < T; ++w) s.d += tasks[ci.off + r * T + w].htd;
                    }
                    int32_t dend[T];
#pragma unroll
                    for (int i = 0; i < T; ++i) {
                        const int w = (int)((pw >> (4 * i)) & 0xF);
                        const tm_task x = tasks[ci.off + r * T + w];
                        s = step_c(s, pick<T>(c, w), make_int4(x.htd, x.k, x.dth, 0));
                        dend[i] = s.d;
                    }
#pragma unroll
                    for (int w = 0; w < T; ++w) c[w] = pick<T>(dend, (int)((iw >> (4 * w)) & 0xF));
                }
            }
            // the penultimate round's rows with their release times
            int4 pr[T];
#pragma unroll
            for (int w = 0; w < T; ++w) pr[w] = make_int4(prow[w].x, prow[w].y, prow[w].z, c[w]);
            Eng s0 = s;                       // entering the penultimate round
            if (ci.dma == 1) { s0.h = s0.d; s0.d += sh_pen; }
            Eng st[T];
            int32_t dend[T];
            uint32_t rank = o * (uint32_t)(F * F);
            for (int q = 0; q < F; ++q) {
                const uint32_t pw = c_small.perm[T - 2][q];
                const int piv = c_small.pivot[T - 2][q];
#pragma unroll
                for (int i = 0; i < T; ++i) {
                    if (i >= piv) {
                        const int4 x = pick4<T>(pr, (int)((pw >> (4 * i)) & 0xF));
                        st[i] = step_c(i == 0 ? s0 : st[i > 0 ? i - 1 : 0], x.w, x);
                        dend[i] = st[i].d;
                    }
                }
                // the last round: release times from this round's DtH ends
                const uint32_t iw = c_small.inv[T - 2][q];
                int4 lr[T];
#pragma unroll
                for (int w = 0; w < T; ++w)
                    lr[w] = make_int4(lrow[w].x, lrow[w].y, lrow[w].z,
                                      pick<T>(dend, (int)((iw >> (4 * w)) & 0xF)));
                Eng s1 = st[T - 1];
                if (ci.dma == 1) { s1.h = s1.d; s1.d += sh_last; }
                if constexpr (T == 4) {
                    // the closed form when the HtD engine's path ends every
                    // order on every lane of the warp (one path per warp)
                    ++ntail;
                    const int32_t hh = s1.h;
                    bool hd = hh - s1.d >= ht.td && hh - s1.k >= ht.tk;
#pragma unroll
                    for (int w = 0; w < 4; ++w) hd = hd && lr[w].w - hh <= ht.tc[w];
                    if (__all_sync(__activemask(), hd)) {
                        ++nclosed;
                        const int32_t mn = hh + ht.gmin, mx = hh + ht.gmax;
                        if (mn < a.best) { a.best = mn; a.brank = rank + ht.imin; }
                        if (mx > a.worst) { a.worst = mx; a.wrank = rank + ht.imax; }
                        a.sum += 24ull * (uint32_t)hh + ht.gsum;
                    } else {
                        tail4_pair(s1, reinterpret_cast<const int4 (&)[4]>(lr), pq, a, rank, one);
                    }
                } else {
                    tail_static<T>(s1, lr, a, rank);
                }
                rank += F;
            }
        }
        flush_warp(a, acc, g);
    }
    __syncwarp();
    }
    if constexpr (T == 4) {
        if (counts) {   // one pair of atomics per warp
            const unsigned live = __activemask();
            const uint32_t t32 = __reduce_add_sync(live, ntail);
            const uint32_t c32 = __reduce_add_sync(live, nclosed);
            if ((int)(threadIdx.x & 31) == __ffs(live) - 1) {
                atomicAdd(&counts[0], (unsigned long long)t32);
                atomicAdd(&counts[1], (unsigned long long)c32);
            }
        }
    }
}

// Order of rank `rank` of a chained group as task indices, and its makespan.
__device__ int32_t chain_order_of_rank(const tm_task* __restrict__ tasks, const ChainInfo& ci,
                                       uint32_t rank, uint8_t* order_out)
{
    const int T = ci.T, R = ci.R;
    const uint32_t F = (uint32_t)factorial_u64(T);
    uint32_t rw[TM_MAX_TASKS];
    for (int r = R - 1; r >= 0; --r) {
        rw[r] = unrank_round(rank % F, T);
        rank /= F;
    }
    Eng s{0, 0, 0};
    int32_t dend[TM_MAX_TASKS];
    for (int r = 0; r < R; ++r) {
        if (ci.dma == 1) {
            s.h = s.d;
            s.d += round_htd(tasks, ci.off, T, r);
        }
        const uint32_t prev_inv = r ? inverse_nib(rw[r - 1], T) : 0u;
        for (int i = 0; i < T; ++i) {
            const int w = (int)nib32(rw[r], i);
            const tm_task t = tasks[ci.off + r * T + w];
            const int32_t c = r ? dend[(r - 1) * T + (int)nib32(prev_inv, w)] : 0;
            s = step_c(s, c, make_int4(t.htd, t.k, t.dth, 0));
            dend[r * T + i] = s.d;
            if (order_out) order_out[r * T + i] = (uint8_t)(r * T + w);
        }
    }
    return s.d;
}

__global__ void chain_finalize_kernel(const ChainInfo* __restrict__ info, const tm_task* __restrict__ tasks,
                                      int G, const unsigned long long* __restrict__ acc,
                                      tm_stats* __restrict__ stats, int32_t* __restrict__ status)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    const ChainInfo ci = info[g];
    if (ci.status != 0) return;
    const unsigned long long kmin = acc[4 * (size_t)g], kmax = acc[4 * (size_t)g + 1];
    tm_stats st;
    st.best = (int32_t)(kmin >> 32);
    st.worst = (int32_t)(kmax >> 32);
    st.sum = (int64_t)acc[4 * (size_t)g + 2];
    st.mean = (double)st.sum / (double)chain_orders(ci.T, ci.R);
    st.best_rank = (uint32_t)kmin;
    st.worst_rank = 0xFFFFFFFFu - (uint32_t)kmax;
    for (int i = 0; i < 16; ++i) st.best_order[i] = st.worst_order[i] = 0xFF;
    const int32_t b = chain_order_of_rank(tasks, ci, (uint32_t)st.best_rank, st.best_order);
    const int32_t w = chain_order_of_rank(tasks, ci, (uint32_t)st.worst_rank, st.worst_order);
    stats[g] = st;
    // the unranked orders must reproduce the reduced values
    if (status) status[g] = (b == st.best && w == st.worst) ? 0 : TM_ECUDA;
}

__global__ void chain_predict_kernel(const tm_task* __restrict__ tasks,
                                     const int32_t* __restrict__ offsets,
                                     const int32_t* __restrict__ workers, int G,
                                     const int32_t* __restrict__ orders,
                                     const tm_device* __restrict__ devs,
                                     int32_t* __restrict__ makespans, int32_t* __restrict__ status)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    const int off = offsets[g], n = offsets[g + 1] - off, T = workers[g];
    const int dma = devs[g].dma_engines;
    int rc = check_chain(tasks + off, n, T, dma);
    // each round's block must be a permutation of that round's task indices
    uint32_t seen = 0;
    for (int p = 0; rc == 0 && p < n; ++p) {
        const int e = orders[off + p];
        if (e < 0 || e >= n || e / T != p / T || ((seen >> e) & 1u)) rc = TM_EINVAL;
        else seen |= 1u << e;
    }
    if (rc != 0) {
        if (status) status[g] = rc;
        return;
    }
    const int R = n / T;
    Eng s{0, 0, 0};
    int32_t dend[TM_MAX_TASKS];
    int pos_prev[kChainMaxWorkers];
    int pos_cur[kChainMaxWorkers];
    for (int r = 0; r < R; ++r) {
        if (dma == 1) {
            s.h = s.d;
            s.d += round_htd(tasks, off, T, r);
        }
        for (int i = 0; i < T; ++i) {
            const int e = orders[off + r * T + i], w = e - r * T;
            const tm_task t = tasks[off + e];
            const int32_t c = r ? dend[(r - 1) * T + pos_prev[w]] : 0;
            s = step_c(s, c, make_int4(t.htd, t.k, t.dth, 0));
            dend[r * T + i] = s.d;
            pos_cur[w] = i;
        }
        for (int w = 0; w < T; ++w) pos_prev[w] = pos_cur[w];
    }
    makespans[g] = s.d;
    if (status) status[g] = 0;
}

struct ChainScratch {
    void* p = nullptr;
    size_t cap = 0;
    int device = -1;
    std::vector<unsigned long long> h_base;   // generic blocks, then fast-path units per T
    unsigned long long* d_counts = nullptr;   // the last search's tails walked, closed forms
};

// Groups the fast path takes: 2 <= T <= 4 workers and at least two rounds.
inline bool chain_fast(int n, int T) { return T >= 2 && T <= 4 && n % T == 0 && n / T >= 2 && n <= TM_MAX_TASKS; }

template <int T>
cudaError_t launch_small(const unsigned long long* d_base, const unsigned long long* h_base, int G,
                         const ChainInfo* d_info, const tm_task* d_tasks, unsigned long long* d_acc,
                         int dev, cudaStream_t s, unsigned long long* d_counts,
                         const HtdTail* d_tails, unsigned long long* d_next)
{
    const unsigned long long total = h_base[G];
    if (total == 0) return cudaSuccess;
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, chain_small_kernel<T>, kChainBlock,
                                                      0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const unsigned long long resident = (unsigned long long)std::max(sms, 1) * per_sm * kChainBlock;
    // batches of 32 x per_lane units, at least four per warp where the
    // batch allows, at most 4 units a lane
    const unsigned long long per_lane = std::max<unsigned long long>(
        1ull, std::min<unsigned long long>(4ull, total / (4ull * resident)));
    const unsigned long long warps =
        std::min((resident + 31) / 32, (total + 32 * per_lane - 1) / (32 * per_lane));
    const unsigned blocks = (unsigned)((warps * 32 + kChainBlock - 1) / kChainBlock);
    chain_small_kernel<T><<<blocks, kChainBlock, 0, s>>>(d_base, G, d_info, d_tasks, d_acc,
                                                        per_lane, 1u, d_counts, d_tails, d_next);
    return cudaGetLastError();
}
thread_local ChainScratch t_chain;

}  // namespace

int chain_exhaustive(const tm_task* d_tasks, const int32_t* d_offsets, const int32_t* h_offsets,
                     const int32_t* d_workers, const int32_t* h_workers, int G,
                     const tm_device* d_devs, tm_stats* d_stats, int32_t* d_status,
                     cudaStream_t s)
{
    if (G == 0) return TM_OK;
    ChainScratch& sc = t_chain;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TM_ECUDA;
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    // four prefix tables: the generic kernel's blocks, the fast path's units for T = 2, 3, 4
    const size_t b_base = 4 * al((size_t)(G + 1) * 8), b_info = al((size_t)G * sizeof(ChainInfo)),
                 b_acc = al((size_t)G * 32);
    const size_t base_stride = al((size_t)(G + 1) * 8) / 8;
    const size_t b_tails = al((size_t)G * sizeof(HtdTail));
    // + the tail counters and the three fast-path batch counters
    const size_t need = b_base + b_info + b_acc + b_tails + al(40);
    if (sc.device != dev || sc.cap < need) {
        if (sc.p && sc.device == dev) {
            cudaDeviceSynchronize();   // earlier calls may still use it
            cudaFree(sc.p);
        }
        sc.p = nullptr;
        sc.cap = 0;
        if (cudaMalloc(&sc.p, need) != cudaSuccess) { sc.p = nullptr; return TM_ENOMEM; }
        sc.cap = need;
        sc.device = dev;
    }
    unsigned char* p = static_cast<unsigned char*>(sc.p);
    unsigned long long* d_base = reinterpret_cast<unsigned long long*>(p);
    ChainInfo* d_info = reinterpret_cast<ChainInfo*>(p + b_base);
    unsigned long long* d_acc = reinterpret_cast<unsigned long long*>(p + b_base + b_info);
    HtdTail* d_tails = reinterpret_cast<HtdTail*>(p + b_base + b_info + b_acc);
    unsigned long long* d_counts =
        reinterpret_cast<unsigned long long*>(p + b_base + b_info + b_acc + b_tails);
    sc.d_counts = d_counts;
    if (cudaMemsetAsync(d_counts, 0, 40, s) != cudaSuccess) return TM_ECUDA;
    // blocks of m! orders per group for the generic kernel (0 for a shape the
    // prep kernel rejects, and for the fast path's groups); units of (T!)^2
    // orders per fast-path group, one table per T
    sc.h_base.assign(4 * base_stride, 0ull);
    unsigned long long* hb[4] = {sc.h_base.data(), sc.h_base.data() + base_stride,
                                 sc.h_base.data() + 2 * base_stride,
                                 sc.h_base.data() + 3 * base_stride};
    for (int g = 0; g < G; ++g) {
        const int n = h_offsets[g + 1] - h_offsets[g], T = h_workers[g];
        const uint64_t orders = (T >= 1 && n % T == 0) ? chain_orders(T, n / T) : 0;
        const bool fast = orders && chain_fast(n, T);
        for (int k = 0; k < 4; ++k) hb[k][g + 1] = hb[k][g];
        if (!orders) continue;
        if (fast) {
            const uint64_t f = factorial_u64(T);
            hb[T - 1][g + 1] += orders / (f * f);
        } else {
            hb[0][g + 1] += orders / factorial_u64(chain_tail(T));
        }
    }
    if (cudaMemcpyAsync(d_base, sc.h_base.data(), 4 * base_stride * 8, cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
        return TM_ECUDA;
    chain_prep_kernel<<<(G + 127) / 128, 128, 0, s>>>(d_tasks, d_offsets, d_workers, G, d_devs,
                                                     d_info, d_acc, d_status);
    if (hb[3][G] > 0)   // groups on the four-worker fast path: their closed-form tables
        chain_tail_kernel<<<(G + 3) / 4, 128, 0, s>>>(d_info, d_tasks, G, d_tails);
    const unsigned long long total = hb[0][G];
    if (total > 0) {
        int sms = 0, per_sm = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, chain_enum_kernel, kChainBlock,
                                                          0) != cudaSuccess || per_sm < 1)
            per_sm = 1;
        const unsigned long long resident = (unsigned long long)std::max(sms, 1) * per_sm * kChainBlock;
        const unsigned long long threads = std::min(total, resident);
        const unsigned long long per_thread = (total + threads - 1) / threads;
        const unsigned long long used = (total + per_thread - 1) / per_thread;
        chain_enum_kernel<<<(unsigned)((used + kChainBlock - 1) / kChainBlock), kChainBlock, 0, s>>>(
            d_base, G, d_info, d_tasks, d_acc, per_thread);
    }
    if (launch_small<2>(d_base + base_stride, hb[1], G, d_info, d_tasks, d_acc, dev, s, nullptr,
                        d_tails, d_counts + 2) != cudaSuccess ||
        launch_small<3>(d_base + 2 * base_stride, hb[2], G, d_info, d_tasks, d_acc, dev, s,
                        nullptr, d_tails, d_counts + 3) != cudaSuccess ||
        launch_small<4>(d_base + 3 * base_stride, hb[3], G, d_info, d_tasks, d_acc, dev, s,
                        d_counts, d_tails, d_counts + 4) != cudaSuccess)
        return TM_ECUDA;
    chain_finalize_kernel<<<(G + 127) / 128, 128, 0, s>>>(d_info, d_tasks, G, d_acc, d_stats,
                                                         d_status);
    return cudaGetLastError() == cudaSuccess ? TM_OK : TM_ECUDA;
}

int chain_tail_counts(unsigned long long* tails, unsigned long long* closed)
{
    unsigned long long h[2] = {0ull, 0ull};
    if (t_chain.d_counts &&
        cudaMemcpy(h, t_chain.d_counts, sizeof h, cudaMemcpyDeviceToHost) != cudaSuccess)
        return TM_ECUDA;
    *tails = h[0];
    *closed = h[1];
    return TM_OK;
}

cudaError_t launch_chain_predict(const tm_task* d_tasks, const int32_t* d_offsets,
                                 const int32_t* d_workers, int G, const int32_t* d_orders,
                                 const tm_device* d_devs, int32_t* d_makespans, int32_t* d_status,
                                 cudaStream_t s)
{
    if (G == 0) return cudaSuccess;
    chain_predict_kernel<<<(G + 127) / 128, 128, 0, s>>>(d_tasks, d_offsets, d_workers, G,
                                                        d_orders, d_devs, d_makespans, d_status);
    return cudaGetLastError();
}

}  // namespace tmgpu

// ---- C ABI -------------------------------------------------------------------

namespace {

using namespace tmgpu;

// Host-side checks of one chained group; TM_OK or the error code.
int check_chain_host(const tm_task* tasks, int n, int T, int dma)
{
    if (!tasks || T < 1 || T > kChainMaxWorkers || n < 1 || n > TM_MAX_TASKS || n % T != 0)
        return TM_EINVAL;
    if (dma != 1 && dma != 2) return TM_EINVAL;
    int64_t total = 0;
    for (int i = 0; i < n; ++i) {
        if (tasks[i].htd < 0 || tasks[i].k < 0 || tasks[i].dth < 0) return TM_ENEG;
        total += (int64_t)tasks[i].htd + tasks[i].k + tasks[i].dth;
    }
    return total > INT32_MAX ? TM_EOVERFLOW : TM_OK;
}

// Device copies of a host batch for the host-pointer calls (grown, never
// shrunk; one per host thread).
struct ChainStage {
    void* p = nullptr;
    size_t cap = 0;
    int device = -1;
    bool ensure(size_t need, int dev)
    {
        if (p && cap >= need && device == dev) return true;
        if (p && device == dev) cudaFree(p);
        p = nullptr;
        cap = 0;
        if (cudaMalloc(&p, need) != cudaSuccess) { p = nullptr; return false; }
        cap = need;
        device = dev;
        return true;
    }
};
thread_local ChainStage t_stage;

}  // namespace

extern "C" {

int tm_chain_tail_counts(unsigned long long* tails, unsigned long long* closed)
{
    if (!tails || !closed) return TM_EINVAL;
    return chain_tail_counts(tails, closed);
}

int tm_exhaustive_chain_batch_dev(const tm_task* d_tasks, const int32_t* d_offsets,
                                  const int32_t* h_offsets, const int32_t* d_workers,
                                  const int32_t* h_workers, int G, const tm_device* d_devs,
                                  tm_stats* d_stats, int32_t* d_status, void* stream)
{
    if (G < 0) return TM_EINVAL;
    if (G == 0) return TM_OK;
    if (!d_tasks || !d_offsets || !h_offsets || !d_workers || !h_workers || !d_devs || !d_stats)
        return TM_EINVAL;
    if (h_offsets[0] != 0) return TM_EINVAL;
    for (int g = 0; g < G; ++g)
        if (h_offsets[g + 1] < h_offsets[g]) return TM_EINVAL;
    return chain_exhaustive(d_tasks, d_offsets, h_offsets, d_workers, h_workers, G, d_devs,
                            d_stats, d_status, static_cast<cudaStream_t>(stream));
}

int tm_predict_chain_batch_dev(const tm_task* d_tasks, const int32_t* d_offsets,
                               const int32_t* d_workers, int G, const int32_t* d_orders,
                               const tm_device* d_devs, int32_t* d_makespans, int32_t* d_status,
                               void* stream)
{
    if (G < 0) return TM_EINVAL;
    if (G == 0) return TM_OK;
    if (!d_tasks || !d_offsets || !d_workers || !d_orders || !d_devs || !d_makespans)
        return TM_EINVAL;
    return launch_chain_predict(d_tasks, d_offsets, d_workers, G, d_orders, d_devs, d_makespans,
                                d_status, static_cast<cudaStream_t>(stream)) == cudaSuccess
               ? TM_OK
               : TM_ECUDA;
}

int tm_exhaustive_chain_batch(const tm_task* tasks, const int32_t* offsets,
                              const int32_t* workers, int G, const tm_device* devs,
                              tm_stats* out)
{
    if (G < 0 || !offsets || !workers || !devs || (G > 0 && (!tasks || !out))) return TM_EINVAL;
    if (G == 0) return TM_OK;
    if (offsets[0] != 0) return TM_EINVAL;
    for (int g = 0; g < G; ++g) {
        if (offsets[g + 1] < offsets[g]) return TM_EINVAL;
        const int rc = check_chain_host(tasks + offsets[g], offsets[g + 1] - offsets[g],
                                        workers[g], devs[g].dma_engines);
        if (rc != TM_OK) return rc;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TM_ECUDA;
    const int T = offsets[G];
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t b_t = al((size_t)T * sizeof(tm_task)), b_o = al((size_t)(G + 1) * 4),
                 b_w = al((size_t)G * 4), b_d = al((size_t)G * sizeof(tm_device)),
                 b_s = al((size_t)G * sizeof(tm_stats)), b_st = al((size_t)G * 4);
    if (!t_stage.ensure(b_t + b_o + b_w + b_d + b_s + b_st, dev)) return TM_ENOMEM;
    unsigned char* p = static_cast<unsigned char*>(t_stage.p);
    tm_task* d_tasks = reinterpret_cast<tm_task*>(p);
    int32_t* d_off = reinterpret_cast<int32_t*>(p + b_t);
    int32_t* d_w = reinterpret_cast<int32_t*>(p + b_t + b_o);
    tm_device* d_dv = reinterpret_cast<tm_device*>(p + b_t + b_o + b_w);
    tm_stats* d_st = reinterpret_cast<tm_stats*>(p + b_t + b_o + b_w + b_d);
    int32_t* d_status = reinterpret_cast<int32_t*>(p + b_t + b_o + b_w + b_d + b_s);
    if (cudaMemcpy(d_tasks, tasks, (size_t)T * sizeof(tm_task), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d_off, offsets, (size_t)(G + 1) * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d_w, workers, (size_t)G * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d_dv, devs, (size_t)G * sizeof(tm_device), cudaMemcpyHostToDevice) != cudaSuccess)
        return TM_ECUDA;
    int rc = chain_exhaustive(d_tasks, d_off, offsets, d_w, workers, G, d_dv, d_st, d_status, 0);
    if (rc != TM_OK) return rc;
    std::vector<int32_t> status((size_t)G);
    if (cudaMemcpy(status.data(), d_status, (size_t)G * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
        return TM_ECUDA;
    for (int g = 0; g < G; ++g)
        if (status[g] != 0) return status[g];
    return cudaMemcpy(out, d_st, (size_t)G * sizeof(tm_stats), cudaMemcpyDeviceToHost) == cudaSuccess
               ? TM_OK
               : TM_ECUDA;
}

int tm_exhaustive_chain(const tm_task* tasks, int workers, int rounds, const tm_device* dev,
                        tm_stats* out)
{
    if (!tasks || !dev || !out || workers < 1 || rounds < 1 || workers * rounds > TM_MAX_TASKS)
        return TM_EINVAL;
    const int32_t offsets[2] = {0, workers * rounds};
    return tm_exhaustive_chain_batch(tasks, offsets, &workers, 1, dev, out);
}

int tm_predict_chain(const tm_task* tasks, int workers, int rounds, const int32_t* order,
                     const tm_device* dev, int32_t* makespan)
{
    if (!tasks || !order || !dev || !makespan || workers < 1 || rounds < 1 ||
        workers * rounds > TM_MAX_TASKS)
        return TM_EINVAL;
    const int n = workers * rounds;
    int rc = check_chain_host(tasks, n, workers, dev->dma_engines);
    if (rc != TM_OK) return rc;
    uint32_t seen = 0;
    for (int p = 0; p < n; ++p) {
        const int e = order[p];
        if (e < 0 || e >= n || e / workers != p / workers || ((seen >> e) & 1u)) return TM_EINVAL;
        seen |= 1u << e;
    }
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess) return TM_ECUDA;
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t b_t = al((size_t)n * sizeof(tm_task));
    if (!t_stage.ensure(b_t + 5 * 256, d)) return TM_ENOMEM;
    unsigned char* p = static_cast<unsigned char*>(t_stage.p);
    tm_task* d_tasks = reinterpret_cast<tm_task*>(p);
    int32_t* d_off = reinterpret_cast<int32_t*>(p + b_t);
    int32_t* d_w = reinterpret_cast<int32_t*>(p + b_t + 256);
    int32_t* d_ord = reinterpret_cast<int32_t*>(p + b_t + 512);
    tm_device* d_dv = reinterpret_cast<tm_device*>(p + b_t + 768);
    int32_t* d_ms = reinterpret_cast<int32_t*>(p + b_t + 1024);
    const int32_t off[2] = {0, n};
    if (cudaMemcpy(d_tasks, tasks, (size_t)n * sizeof(tm_task), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d_off, off, 8, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d_w, &workers, 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d_ord, order, (size_t)n * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d_dv, dev, sizeof(tm_device), cudaMemcpyHostToDevice) != cudaSuccess)
        return TM_ECUDA;
    if (launch_chain_predict(d_tasks, d_off, d_w, 1, d_ord, d_dv, d_ms, nullptr, 0) != cudaSuccess)
        return TM_ECUDA;
    return cudaMemcpy(makespan, d_ms, 4, cudaMemcpyDeviceToHost) == cudaSuccess ? TM_OK : TM_ECUDA;
}

}  // extern "C"

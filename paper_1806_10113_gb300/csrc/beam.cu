// beam.cu -- beam search over task orders with the learned ranker, for
// groups beyond exhaustive reach (up to 16 tasks).  The paper has no
// counterpart; its exact model judges every order: each beam carries the
// exact int32 engine times of its prefix (the recurrence of tm_device.cuh),
// so a finished beam's makespan is exact, and the result is the better of
// the best finished beam and the paper's heuristic order (Algorithm 1).
//
// The same feature map also builds the ranker's training rows along given
// orders (rows_kernel).
//
// Step i (the i-th position): every live beam b of group g proposes each of
// its unused tasks; row ((g * B + b) * R + slot) of the feature matrix holds
// the features of "append the slot-th unused task", R = nmax - i (written by
// the previous selection or the row kernel; at i = 0 the init kernel writes
// beam 0's rows alone, row g R + slot, the only live beam there).  The
// ranker scores the rows; a block per group (a warp per group for large
// batches at widths up to 16) turns scores into log-softmax over each beam's
// candidates, adds the beam's log-probability, keeps the best B candidates
// (the best 64 of the B x R keys by warp-sorted runs and pairwise merges, or
// B rounds of a warp-wide maximum; ties: lower beam, then lower slot) and
// applies them.
#include <cuda_bf16.h>

#include "rank_features.cuh"
#include "ranker.h"
#include "refine.cuh"
#include "tm_device.cuh"

namespace tmgpu {

struct BeamState {
    int32_t h, k, d;
    uint32_t used;
    unsigned long long order;   // task at position p in bits 4p .. 4p + 3
    float logp;
    int32_t alive;
};
static_assert(sizeof(BeamState) == 32, "beam state layout");

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

constexpr int kMaxCand = 64 * 16;   // beam width <= 64, tasks <= 16
constexpr int kMaxRefineStarts = TM_BEAM_MAX_REFINE_STARTS;

__device__ __forceinline__ int slot_task(uint32_t used, int n, int slot)
{
    // the slot-th task not in `used`
    uint32_t free_mask = ((n >= 32) ? kFull : ((1u << n) - 1u)) & ~used;
    for (int s = 0; s < slot; ++s) free_mask &= free_mask - 1;
    return __ffs(free_mask) - 1;
}

// Candidate row (g, b, slot) of a step with R rows per beam: the features
// of appending the slot-th unplaced task to beam state s, as one 64-byte row
// (four 16-byte stores).
__device__ __forceinline__ void write_row(__nv_bfloat16* __restrict__ X, int64_t row,
                                          const tm_task* __restrict__ gtasks, int n,
                                          const BeamState& s, int dma, float scale, int slot)
{
    float f[kFeat];
    rank_features(gtasks, n, s.used, s.h, s.k, s.d, dma, scale, slot_task(s.used, n, slot), f);
    uint32_t w[kFeat / 2];
#pragma unroll
    for (int q = 0; q < kFeat / 2; ++q) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(f[2 * q], f[2 * q + 1]);
        w[q] = *reinterpret_cast<const uint32_t*>(&h);
    }
    uint4* x = reinterpret_cast<uint4*>(X + row * kFeat);
#pragma unroll
    for (int q = 0; q < 4; ++q) x[q] = make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
}

// Initial beams (only beam 0 live, empty prefix) and the candidate rows of
// position 0: beam 0's alone, R per group (row g R + slot), since no other
// beam has candidates there.
__global__ void beam_init_kernel(const int32_t* __restrict__ offsets,
                                 const int32_t* __restrict__ status, const tm_task* __restrict__ tasks,
                                 const tm_device* __restrict__ devs, int G, int B, int R,
                                 BeamState* __restrict__ st, float* __restrict__ scale,
                                 __nv_bfloat16* __restrict__ X)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= G * B) return;
    const int g = t / B, b = t - g * B;
    const int off = offsets[g], n = offsets[g + 1] - off;
    BeamState s;
    s.h = s.k = s.d = 0;
    s.used = 0;
    s.order = 0;
    s.logp = 0.0f;
    s.alive = (b == 0 && status[g] == 0) ? 1 : 0;
    if (b == 0) {
        int64_t hs = 0, total = 0;
        for (int i = 0; i < n && status[g] == 0; ++i) {
            hs += tasks[off + i].htd;
            total += (int64_t)tasks[off + i].htd + tasks[off + i].k + tasks[off + i].dth;
        }
        if (devs[g].dma_engines == 1) s.d = (int32_t)hs;   // one transfer queue
        const float sc = total > 0 ? (float)n / (float)total : 0.0f;
        scale[g] = sc;
        if (s.alive)
            for (int slot = 0; slot < n; ++slot)
                write_row(X, (int64_t)g * R + slot, tasks + off, n, s, devs[g].dma_engines, sc, slot);
    }
    st[t] = s;
}

// Candidate rows of position pos from the current beams, one thread per
// (g, b, slot): used for large batches, where spreading the rows over the
// whole GPU beats writing them inside the per-group selection blocks.
__global__ void beam_features_kernel(const int32_t* __restrict__ offsets,
                                     const tm_task* __restrict__ tasks,
                                     const tm_device* __restrict__ devs,
                                     const float* __restrict__ scale, const BeamState* __restrict__ st,
                                     int G, int B, int R, int pos, __nv_bfloat16* __restrict__ X)
{
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t rows = (int64_t)G * B * R;
    if (row >= rows) return;
    const int gb = (int)(row / R), slot = (int)(row - (int64_t)gb * R);
    const int g = gb / B;
    const int off = offsets[g], n = offsets[g + 1] - off;
    const BeamState s = st[gb];
    if (s.alive && pos < n && slot < n - pos)
        write_row(X, row, tasks + off, n, s, devs[g].dma_engines, scale[g], slot);
}

__device__ __forceinline__ uint32_t orderable(float v)
{
    uint32_t u = __float_as_uint(v);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// With WRITE_NEXT it also writes the candidate rows of position pos + 1
// (R - 1 rows per beam) from the new beams, so that each position costs two
// launches: the scores and this selection (small batches, where launches
// dominate).
// NT (512 or 1024) threads per block; the first 512 hold the keys.  Beam
// b's R logits start at g GS + b R (GS = B R, or R at position 0).
template <bool WRITE_NEXT, int NT>
__global__ void __launch_bounds__(NT)
beam_select_kernel(const int32_t* __restrict__ offsets, const tm_task* __restrict__ tasks,
                   const tm_device* __restrict__ devs, const float* __restrict__ scale,
                   const float* __restrict__ logits, const BeamState* __restrict__ cur,
                   BeamState* __restrict__ nxt, int B, int R, int GS, int pos,
                   __nv_bfloat16* __restrict__ X)
{
    const int g = blockIdx.x;
    const int off = offsets[g], n = offsets[g + 1] - off;
    const int tid = threadIdx.x;
    if (pos >= n) {   // group already complete: carry the beams over
        for (int b = tid; b < B; b += blockDim.x) nxt[(size_t)g * B + b] = cur[(size_t)g * B + b];
        return;
    }
    __shared__ float lse[64];
    __shared__ unsigned long long buf[kMaxCand];
    __shared__ BeamState ns[64];
    const int cands = n - pos;
    // log-sum-exp of each live beam's candidate logits: all of a beam's
    // logits are loaded at once (one memory latency, not one per
    // candidate), then reduced in candidate order
    for (int b = tid; b < B; b += blockDim.x) {
        const BeamState s = cur[(size_t)g * B + b];
        float mx = -INFINITY, z = 0.0f;
        if (s.alive) {
            const float* lg = logits + (size_t)g * GS + (size_t)b * R;
            float v[TM_MAX_TASKS];
#pragma unroll
            for (int c = 0; c < TM_MAX_TASKS; ++c) v[c] = c < cands ? lg[c] : 0.0f;
#pragma unroll
            for (int c = 0; c < TM_MAX_TASKS; ++c)
                if (c < cands) mx = fmaxf(mx, v[c]);
#pragma unroll
            for (int c = 0; c < TM_MAX_TASKS; ++c)
                if (c < cands) z += expf(v[c] - mx);
        }
        lse[b] = s.alive ? mx + logf(z) : 0.0f;
    }
    __syncthreads();
    // The B x R <= kMaxCand candidate keys sit two per lane in warps
    // 0 .. 15 (warp w: keys 64 w .. 64 w + 63, lane l holding 64 w + l and
    // 64 w + 32 + l), so that each of those warps can sort its 64 alone.
    static_assert(NT >= 512 && kMaxCand == 1024, "16 warps of 64 keys");
    const int lane = tid & 31, w = tid >> 5;
    unsigned long long key[2] = {0ull, 0ull};
    if (w < 16) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int i = 64 * w + 32 * q + lane;
            const int b = i / R, c = i - (i / R) * R;
            if (b < B && c < cands && cur[(size_t)g * B + b].alive) {
                const float score = cur[(size_t)g * B + b].logp +
                                    (logits[(size_t)g * GS + (size_t)b * R + c] - lse[b]);
                key[q] = ((unsigned long long)orderable(score) << 32) | (0xFFFFu - (uint32_t)i);
            }
        }
    }
    // Top 64 by sorted runs and merges: each warp sorts its 64 keys
    // (bitonic, descending; the partner at distance 32 is the lane's other
    // key, nearer ones by shuffle), then runs merge pairwise in four rounds:
    // the upper run of a pair is read reversed from shared memory, the
    // element-wise maximum of the two is a bitonic sequence holding the
    // pair's best 64, and a half-cleaner cascade sorts it.  Keys are
    // distinct (the candidate index is in their low bits), so the best 64
    // come out exactly as a full sort would order them.
    auto cx = [&](unsigned long long& a, unsigned long long o, bool keep_max) {
        a = keep_max ? (a > o ? a : o) : (a < o ? a : o);
    };
    const bool any = __any_sync(0xFFFFFFFFu, (key[0] | key[1]) != 0ull);
    for (int kk = 2; w < 16 && any && kk <= 64; kk <<= 1) {   // a run of empty keys is sorted
        for (int j = kk >> 1; j > 0; j >>= 1) {
            if (j == 32) {   // kk == 64: element l against element 32 + l
                const unsigned long long a = key[0], b = key[1];
                key[0] = a > b ? a : b;
                key[1] = a > b ? b : a;
            } else {
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const unsigned long long o = __shfl_xor_sync(0xFFFFFFFFu, key[q], j);
                    const int e = 32 * q + lane;
                    cx(key[q], o, ((e & j) == 0) == ((e & kk) == 0));
                }
            }
        }
    }
    unsigned long long (*run)[64] = reinterpret_cast<unsigned long long (*)[64]>(buf);
    for (int span = 1; span < 16; span <<= 1) {
        const bool upper = w < 16 && (w & (2 * span - 1)) == span;
        const bool merger = w < 16 && (w & (2 * span - 1)) == 0;
        if (upper) { run[w][lane] = key[0]; run[w][32 + lane] = key[1]; }
        __syncthreads();
        if (merger) {
            // element e against the partner's element 63 - e
            cx(key[0], run[w + span][63 - lane], true);
            cx(key[1], run[w + span][31 - lane], true);
            const unsigned long long a = key[0], b = key[1];   // distance 32
            key[0] = a > b ? a : b;
            key[1] = a > b ? b : a;
            for (int j = 16; j > 0; j >>= 1) {
#pragma unroll
                for (int q = 0; q < 2; ++q)
                    cx(key[q], __shfl_xor_sync(0xFFFFFFFFu, key[q], j), (lane & j) == 0);
            }
        }
        __syncthreads();
    }
    if (w == 0) { run[0][lane] = key[0]; run[0][32 + lane] = key[1]; }
    __syncthreads();
    for (int b = tid; b < B; b += blockDim.x) {
        BeamState s;
        const unsigned long long k = run[0][b];
        if (k == 0) {
            s.alive = 0;
            s.h = s.k = s.d = 0;
            s.used = 0;
            s.order = 0;
            s.logp = 0.0f;
        } else {
            const int i = (int)(0xFFFFu - (uint32_t)(k & 0xFFFFu));
            const int pb = i / R, c = i - (i / R) * R;
            const BeamState p = cur[(size_t)g * B + pb];
            const int j = slot_task(p.used, n, c);
            const tm_task t = tasks[off + j];
            const Eng e = step(Eng{p.h, p.k, p.d}, t.htd, t.k, t.dth);
            s.h = e.h; s.k = e.k; s.d = e.d;
            s.used = p.used | (1u << j);
            s.order = p.order | ((unsigned long long)j << (4 * pos));
            s.logp = p.logp + (logits[(size_t)g * GS + (size_t)pb * R + c] - lse[pb]);
            s.alive = 1;
        }
        nxt[(size_t)g * B + b] = s;
        ns[b] = s;
    }
    // candidate rows of the next position
    const int R1 = R - 1, left = n - pos - 1;
    if (!WRITE_NEXT || R1 <= 0 || left <= 0) return;
    __syncthreads();
    const int dma = devs[g].dma_engines;
    const float sc = scale[g];
    for (int r = tid; r < B * R1; r += blockDim.x) {
        const int b = r / R1, slot = r - (r / R1) * R1;
        if (slot < left && ns[b].alive)
            write_row(X, ((int64_t)g * B + b) * R1 + slot, tasks + off, n, ns[b], dma, sc, slot);
    }
}

// The selection for beam widths up to 16 with one warp per group, for large
// batches (the next position's rows come from beam_features_kernel).  It
// forms the same log-sum-exp and the same keys, with the same float
// expressions in the same order, as beam_select_kernel; key i = b R + c sits
// in lane i mod 32 (at most 16 x 16 keys, eight per lane).  Each lane sorts
// its eight (a 19-comparator network, descending), then B rounds take the
// warp-wide maximum of the lanes' heads -- the high words by one reduction,
// the low words among the lanes that hold the top high word by a second --
// and the lane that held it advances.  The keys are distinct, so the B kept
// beams, and their order, are those of the block kernel.
constexpr int kWarpSelectMaxB = 16;   // = kBeamWarpSelectMaxB (learn_internal.h)
constexpr int kWarpSelectKeys = kWarpSelectMaxB * TM_MAX_TASKS / 32;
constexpr int kWarpSelectBlock = 256;   // 8 groups per block
// Batches of at most this many groups keep the block selection (a block of
// 1024 threads per group writes the next rows; the serving loop's batches).
constexpr int kBlockSelectMaxGroups = 8;
static_assert(kWarpSelectKeys == 8, "the sorting network below is for eight keys");

__device__ __forceinline__ void cx_desc(unsigned long long& a, unsigned long long& b)
{
    const unsigned long long hi = a > b ? a : b, lo = a > b ? b : a;
    a = hi;
    b = lo;
}

template <bool WRITE_NEXT>
__global__ void __launch_bounds__(kWarpSelectBlock)
beam_select_warp_kernel(const int32_t* __restrict__ offsets, const tm_task* __restrict__ tasks,
                        const float* __restrict__ logits, const BeamState* __restrict__ cur,
                        BeamState* __restrict__ nxt, int G, int B, int R, int GS, int pos,
                        const tm_device* __restrict__ devs, const float* __restrict__ scale,
                        __nv_bfloat16* __restrict__ X)
{
    // as a programmatic dependent launch it may start while the scores'
    // kernel finishes: wait for it (a no-op otherwise)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int g = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (g >= G) return;   // whole warps
    const int off = offsets[g], n = offsets[g + 1] - off;
    const BeamState* cg = cur + (size_t)g * B;
    BeamState* ng = nxt + (size_t)g * B;
    if (pos >= n) {   // group already complete: carry the beams over
        if (lane < B) ng[lane] = cg[lane];
        return;
    }
    const int cands = n - pos;
    const float* lg0 = logits + (size_t)g * GS;
    // lane b < B: beam b's log-sum-exp
    float lse = 0.0f, logp = 0.0f;
    int alive = 0;
    if (lane < B) {
        const BeamState s = cg[lane];
        float mx = -INFINITY, z = 0.0f;
        if (s.alive) {
            const float* lg = lg0 + (size_t)lane * R;
            float v[TM_MAX_TASKS];
#pragma unroll
            for (int c = 0; c < TM_MAX_TASKS; ++c) v[c] = c < cands ? lg[c] : 0.0f;
#pragma unroll
            for (int c = 0; c < TM_MAX_TASKS; ++c)
                if (c < cands) mx = fmaxf(mx, v[c]);
#pragma unroll
            for (int c = 0; c < TM_MAX_TASKS; ++c)
                if (c < cands) z += expf(v[c] - mx);
        }
        lse = s.alive ? mx + logf(z) : 0.0f;
        logp = s.logp;
        alive = s.alive;
    }
    unsigned long long key[kWarpSelectKeys];
#pragma unroll
    for (int q = 0; q < kWarpSelectKeys; ++q) {
        const int i = 32 * q + lane;
        const int b = (int)((unsigned)i / (unsigned)R), c = i - b * R;
        const float lb = __shfl_sync(kFull, lse, b & 31);
        const float lp = __shfl_sync(kFull, logp, b & 31);
        const int al = __shfl_sync(kFull, alive, b & 31);
        key[q] = 0ull;
        if (b < B && c < cands && al) {
            const float score = lp + (lg0[(size_t)b * R + c] - lb);
            key[q] = ((unsigned long long)orderable(score) << 32) | (0xFFFFu - (uint32_t)i);
        }
    }
    cx_desc(key[0], key[2]); cx_desc(key[1], key[3]); cx_desc(key[4], key[6]); cx_desc(key[5], key[7]);
    cx_desc(key[0], key[4]); cx_desc(key[1], key[5]); cx_desc(key[2], key[6]); cx_desc(key[3], key[7]);
    cx_desc(key[0], key[1]); cx_desc(key[2], key[3]); cx_desc(key[4], key[5]); cx_desc(key[6], key[7]);
    cx_desc(key[2], key[4]); cx_desc(key[3], key[5]);
    cx_desc(key[1], key[4]); cx_desc(key[3], key[6]);
    cx_desc(key[1], key[2]); cx_desc(key[3], key[4]); cx_desc(key[5], key[6]);
    unsigned long long mine = 0ull;   // lane r: the r-th best key (0: none)
    for (int r = 0; r < B; ++r) {
        const uint32_t hi = (uint32_t)(key[0] >> 32), lo = (uint32_t)key[0];
        const uint32_t mhi = __reduce_max_sync(kFull, hi);
        if (mhi == 0u) break;   // no keys left: the remaining beams die
        const uint32_t mlo = __reduce_max_sync(kFull, hi == mhi ? lo : 0u);
        if (lane == r) mine = ((unsigned long long)mhi << 32) | mlo;
        if (hi == mhi && lo == mlo) {
#pragma unroll
            for (int q = 0; q + 1 < kWarpSelectKeys; ++q) key[q] = key[q + 1];
            key[kWarpSelectKeys - 1] = 0ull;
        }
    }
    // the kept candidate's beam pb and slot c, and pb's log-sum-exp
    int pb = 0, c = 0;
    if (mine != 0ull) {
        const int i = (int)(0xFFFFu - (uint32_t)(mine & 0xFFFFu));
        pb = i / R;
        c = i - pb * R;
    }
    const float plse = __shfl_sync(kFull, lse, pb);
    BeamState s;
    s.alive = 0;
    s.h = s.k = s.d = 0;
    s.used = 0;
    s.order = 0;
    s.logp = 0.0f;
    if (lane < B && mine != 0ull) {
        const BeamState p = cg[pb];
        const int j = slot_task(p.used, n, c);
        const tm_task t = tasks[off + j];
        const Eng e = step(Eng{p.h, p.k, p.d}, t.htd, t.k, t.dth);
        s.h = e.h; s.k = e.k; s.d = e.d;
        s.used = p.used | (1u << j);
        s.order = p.order | ((unsigned long long)j << (4 * pos));
        s.logp = p.logp + (lg0[(size_t)pb * R + c] - plse);
        s.alive = 1;
    }
    if (lane < B) ng[lane] = s;
    if constexpr (WRITE_NEXT) {
        // the candidate rows of position pos + 1 (R - 1 per beam) from the
        // new beams, spread over the warp's lanes
        __shared__ BeamState s_new[kWarpSelectBlock / 32][kWarpSelectMaxB];
        const int wi = threadIdx.x >> 5;
        if (lane < B) s_new[wi][lane] = s;
        __syncwarp();
        const int R1 = R - 1, left = n - pos - 1;
        if (R1 > 0 && left > 0) {
            const int dma = devs[g].dma_engines;
            const float sc = scale[g];
            for (int r = lane; r < B * R1; r += 32) {
                const int b = r / R1, slot = r - b * R1;
                if (slot < left && s_new[wi][b].alive)
                    write_row(X, ((int64_t)g * B + b) * R1 + slot, tasks + off, n, s_new[wi][b],
                              dma, sc, slot);
            }
        }
    }
}

// Best finished beam vs the heuristic's order, which is already in `orders`
// (and its makespan in heur_ms): a beam replaces it only when strictly
// better.  beam_won[g] (optional) records which one was kept.
__global__ void beam_finish_kernel(const int32_t* __restrict__ offsets,
                                   const int32_t* __restrict__ status,
                                   const BeamState* __restrict__ st, int G, int B,
                                   const int32_t* __restrict__ heur_ms, int32_t* __restrict__ orders,
                                   int32_t* __restrict__ ms, int32_t* __restrict__ beam_won)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G || status[g] != 0) return;
    const int off = offsets[g], n = offsets[g + 1] - off;
    int best = -1;
    int32_t best_d = 0;
    for (int b = 0; b < B; ++b) {
        const BeamState s = st[(size_t)g * B + b];
        if (s.alive && (best < 0 || s.d < best_d)) { best = b; best_d = s.d; }
    }
    const bool use_beam = best >= 0 && best_d < heur_ms[g];
    if (use_beam) {
        const unsigned long long order = st[(size_t)g * B + best].order;
        for (int p = 0; p < n; ++p) orders[off + p] = (int32_t)((order >> (4 * p)) & 0xF);
    }
    if (ms) ms[g] = use_beam ? best_d : heur_ms[g];
    if (beam_won) beam_won[g] = use_beam ? 1 : 0;
}

// The finish with the exact-model descent of refine.cuh: one block per group,
// warp w < K starts from the finished beam of rank w (smallest makespan
// first, ties to the lower beam), warp K from the heuristic's order (already
// in `orders`); each warp descends, and the smallest result wins (ties: the
// lower warp).  beam_won[g] = 1 where the winner started from a beam.
__global__ void __launch_bounds__(32 * (kMaxRefineStarts + 1))
beam_refine_kernel(const tm_task* __restrict__ tasks, const int32_t* __restrict__ offsets,
                   const tm_device* __restrict__ devs, const int32_t* __restrict__ status,
                   const BeamState* __restrict__ st, int B, int K,
                   const int32_t* __restrict__ heur_ms, int32_t* __restrict__ orders,
                   int32_t* __restrict__ ms, int32_t* __restrict__ beam_won)
{
    __shared__ int4 s_rows[16];
    __shared__ int4 s_pre[kMaxRefineStarts + 1][17];
    __shared__ unsigned long long s_key[64];
    __shared__ unsigned long long s_res[kMaxRefineStarts + 1];
    __shared__ unsigned long long s_ord[kMaxRefineStarts + 1];
    const int g = blockIdx.x;
    if (status[g] != 0) return;   // the whole block
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int off = offsets[g], n = offsets[g + 1] - off;
    const int dma = devs[g].dma_engines;
    if (threadIdx.x < n) {
        const tm_task t = tasks[off + threadIdx.x];
        s_rows[threadIdx.x] = make_int4(t.htd, t.k, t.dth, 0);
    }
    for (int b = threadIdx.x; b < B; b += blockDim.x) {
        const BeamState x = st[(size_t)g * B + b];
        s_key[b] = ((unsigned long long)(x.alive ? (uint32_t)x.d : 0xFFFFFFFFu) << 32) | (uint32_t)b;
    }
    __syncthreads();
    int32_t hs = 0;
    for (int p = 0; p < n; ++p) hs += s_rows[p].x;
    const int32_t dinit = dma == 1 ? hs : 0;
    uint64_t o = 0;
    int32_t cur = INT32_MAX;
    bool have = false;
    if (w < K) {
        // the beam whose key has rank w among the B keys
        for (int b = lane; b < B; b += 32) {
            const unsigned long long kb = s_key[b];
            int rank = 0;
            for (int c = 0; c < B; ++c) rank += s_key[c] < kb;
            if (rank == w && (kb >> 32) != 0xFFFFFFFFull) {
                have = true;
                cur = (int32_t)(kb >> 32);
                o = st[(size_t)g * B + b].order;
            }
        }
        const unsigned who = __ballot_sync(0xFFFFFFFFu, have);
        if (who) {
            const int src = __ffs(who) - 1;
            o = __shfl_sync(0xFFFFFFFFu, o, src);
            cur = __shfl_sync(0xFFFFFFFFu, cur, src);
            have = true;
        }
    } else {
        const int e = lane < n ? orders[off + lane] : 0;
        for (int p = 0; p < n; ++p)
            o |= (uint64_t)(__shfl_sync(0xFFFFFFFFu, e, p) & 0xF) << (4 * p);
        cur = heur_ms[g];
        have = true;
    }
    if (have) refine::descend(&o, &cur, n, dinit, s_rows, s_pre[w], lane);
    if (lane == 0) {
        s_res[w] = have ? (((unsigned long long)(uint32_t)cur << 32) | (uint32_t)w) : ~0ull;
        s_ord[w] = o;
    }
    __syncthreads();
    if (w != 0) return;
    unsigned long long best = ~0ull;
    for (int v = 0; v <= K; ++v) best = min(best, s_res[v]);
    const int win = (int)(best & 0xFFFFFFFFull);
    const uint64_t bo = s_ord[win];
    if (lane < n) orders[off + lane] = (int32_t)((bo >> (4 * lane)) & 0xF);
    if (lane == 0) {
        if (ms) ms[g] = (int32_t)(best >> 32);
        if (beam_won) beam_won[g] = win < K ? 1 : 0;
    }
}

// ---- training rows ----------------------------------------------------------

// Exclusive prefix sums over groups of the training rows (n (n + 1) / 2 - 1
// for n >= 2) and states (n - 1).  One block of 1024 threads.
__global__ void __launch_bounds__(1024)
rows_scan_kernel(const int32_t* __restrict__ offsets, int G, int64_t* __restrict__ row_base,
                 int32_t* __restrict__ state_base)
{
    __shared__ int64_t wr[32];
    __shared__ int32_t ws[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int64_t carry_r = 0;
    int32_t carry_s = 0;
    for (int base = 0; base < G; base += 1024) {
        const int g = base + tid;
        int n = g < G ? offsets[g + 1] - offsets[g] : 0;
        n = n < 2 ? 0 : (n > 16 ? 16 : n);   // out-of-range groups get rows of n = 16
        int64_t r = n ? (int64_t)n * (n + 1) / 2 - 1 : 0;
        int32_t c = n ? n - 1 : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t rr = __shfl_up_sync(kFull, r, o);
            const int32_t cc = __shfl_up_sync(kFull, c, o);
            if (lane >= o) { r += rr; c += cc; }
        }
        if (lane == 31) { wr[warp] = r; ws[warp] = c; }
        __syncthreads();
        if (warp == 0) {
            int64_t x = wr[lane];
            int32_t y = ws[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t xx = __shfl_up_sync(kFull, x, o);
                const int32_t yy = __shfl_up_sync(kFull, y, o);
                if (lane >= o) { x += xx; y += yy; }
            }
            wr[lane] = x;
            ws[lane] = y;
        }
        __syncthreads();
        const int64_t before_r = carry_r + (warp ? wr[warp - 1] : 0);
        const int32_t before_s = carry_s + (warp ? ws[warp - 1] : 0);
        if (g < G) {
            const int nn = offsets[g + 1] - offsets[g];
            const int nc = nn < 2 ? 0 : (nn > 16 ? 16 : nn);
            row_base[g] = before_r + r - (nc ? (int64_t)nc * (nc + 1) / 2 - 1 : 0);
            state_base[g] = before_s + c - (nc ? nc - 1 : 0);
        }
        carry_r += wr[31];
        carry_s += ws[31];
        __syncthreads();
    }
    if (tid == 0) {
        row_base[G] = carry_r;
        state_base[G] = carry_s;
    }
}

// Training rows along each group's given order (behaviour cloning): for
// every position p < n - 1, one row per unused task (ascending task index),
// the state's target being the row of the task the order places at p.
// One warp per group.  Rows and states past M / S are never written; a
// group that fails its input check or whose order is not a permutation gets
// zero rows, targets on the first row of each state, and its status.
__global__ void rows_kernel(const tm_task* __restrict__ tasks, const int32_t* __restrict__ offsets,
                            int G, const tm_device* __restrict__ devs,
                            const int32_t* __restrict__ orders, const tm_stats* __restrict__ stats,
                            const int64_t* __restrict__ row_base,
                            const int32_t* __restrict__ state_base, int64_t M, int64_t M_pad, int S,
                            __nv_bfloat16* __restrict__ X, int32_t* __restrict__ state_off,
                            int32_t* __restrict__ target, int32_t* __restrict__ status)
{
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (gw == 0) {
        // zero tail rows up to M_pad, close the state offsets
        for (int64_t i = M * kFeat + lane; i < M_pad * kFeat; i += 32) X[i] = __float2bfloat16_rn(0.f);
        if (lane == 0) state_off[S] = (int32_t)M;
    }
    if (gw >= G) return;
    const int g = (int)gw;
    const int off = offsets[g], n = offsets[g + 1] - off;
    const int dma = devs[g].dma_engines;
    int32_t hs = 0, dinit = 0;
    int err = check_group(tasks + off, n, dma, 16, &hs, &dinit);
    int my = -1;
    if (err == 0) {
        if (orders) my = lane < n ? orders[off + lane] : -1;
        else my = lane < n ? (int)stats[g].best_order[lane] : -1;
        const bool ok = lane >= n || (my >= 0 && my < n);
        const uint32_t seen = __reduce_or_sync(kFull, (lane < n && ok) ? (1u << my) : 0u);
        if (!__all_sync(kFull, ok) || seen != (n >= 32 ? kFull : (1u << n) - 1u)) err = TM_EINVAL;
    }
    if (lane == 0 && status) status[g] = err;
    int64_t total = 0;
    for (int i = 0; i < n && err == 0; ++i)
        total += (int64_t)tasks[off + i].htd + tasks[off + i].k + tasks[off + i].dth;
    const float scale = total > 0 ? (float)n / (float)total : 0.f;
    const int64_t rb0 = row_base[g];
    const int32_t sb0 = state_base[g];
    Eng e{0, 0, dinit};
    uint32_t used = 0;
    int64_t rb = rb0;
    const int nr = n < 2 ? 0 : (n > 16 ? 16 : n);   // the row layout of rows_scan_kernel
    for (int p = 0; p + 1 < nr; ++p) {
        const int cands = nr - p;
        const int tj = err == 0 ? __shfl_sync(kFull, my, p) : 0;
        const uint32_t free_mask = ((1u << nr) - 1u) & ~used;
        if (lane < cands) {
            float f[kFeat];
            if (err == 0) {
                const int j = slot_task(used, n, lane);
                rank_features(tasks + off, n, used, e.h, e.k, e.d, dma, scale, j, f);
            } else {
                for (int q = 0; q < kFeat; ++q) f[q] = 0.f;
            }
            const int64_t row = rb + lane;
            if (row < M) {
                __nv_bfloat16* x = X + row * kFeat;
#pragma unroll
                for (int q = 0; q < kFeat; ++q) x[q] = __float2bfloat16_rn(f[q]);
            }
        }
        const int32_t sidx = sb0 + p;
        if (lane == 0 && sidx < S) {
            state_off[sidx] = (int32_t)rb;
            const int slot = err == 0 ? __popc(free_mask & ((1u << tj) - 1u)) : 0;
            target[sidx] = (int32_t)(rb + slot);
        }
        if (err == 0) {
            const tm_task t = tasks[off + tj];
            e = step(e, t.htd, t.k, t.dth);
            used |= 1u << tj;
        }
        rb += cands;
    }
}

}  // namespace

// Launchers used by the C ABI (learn_api.cu).
size_t beam_state_bytes(int G, int B) { return (size_t)G * B * sizeof(BeamState); }

cudaError_t beam_init(const int32_t* offsets, const int32_t* status, const tm_task* tasks,
                      const tm_device* devs, int G, int B, int R, void* st, float* scale,
                      bf16_raw* X, cudaStream_t s)
{
    const int threads = G * B;
    beam_init_kernel<<<(threads + 255) / 256, 256, 0, s>>>(offsets, status, tasks, devs, G, B, R,
                                                           static_cast<BeamState*>(st), scale,
                                                           reinterpret_cast<__nv_bfloat16*>(X));
    return cudaGetLastError();
}

cudaError_t beam_features(const int32_t* offsets, const tm_task* tasks, const tm_device* devs,
                          const float* scale, const void* st, int G, int B, int R, int pos,
                          bf16_raw* X, cudaStream_t s)
{
    const int64_t rows = (int64_t)G * B * R;
    beam_features_kernel<<<(unsigned)((rows + 255) / 256), 256, 0, s>>>(
        offsets, tasks, devs, scale, static_cast<const BeamState*>(st), G, B, R, pos,
        reinterpret_cast<__nv_bfloat16*>(X));
    return cudaGetLastError();
}

cudaError_t beam_select(const int32_t* offsets, const tm_task* tasks, const tm_device* devs,
                        const float* scale, const float* logits, const void* cur, void* nxt, int G,
                        int B, int R, int pos, bf16_raw* X, cudaStream_t s, bool pdl)
{
    // the logits of position 0 are beam 0's alone (beam_init_kernel)
    const int GS = pos == 0 ? R : B * R;
    // X == nullptr: the caller writes the next position's rows itself.
    // Widths up to 16 on more than kBlockSelectMaxGroups groups: a warp per
    // group.  Otherwise a block per group: 512 threads for large batches
    // (more blocks per SM), 1024 for small ones (more threads for the
    // log-softmax and the next position's rows).
    const BeamState* c = static_cast<const BeamState*>(cur);
    BeamState* nx = static_cast<BeamState*>(nxt);
    __nv_bfloat16* x = reinterpret_cast<__nv_bfloat16*>(X);
    if (B <= kWarpSelectMaxB && G > kBlockSelectMaxGroups) {
        const int64_t threads = (int64_t)G * 32;
        const unsigned blocks = (unsigned)((threads + kWarpSelectBlock - 1) / kWarpSelectBlock);
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(blocks);
        cfg.blockDim = dim3(kWarpSelectBlock);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = pdl ? attr : nullptr;
        cfg.numAttrs = pdl ? 1 : 0;
        if (X)
            return cudaLaunchKernelEx(&cfg, beam_select_warp_kernel<true>, offsets, tasks, logits, c,
                                      nx, G, B, R, GS, pos, devs, scale, x);
        return cudaLaunchKernelEx(&cfg, beam_select_warp_kernel<false>, offsets, tasks, logits, c,
                                  nx, G, B, R, GS, pos, devs, scale, (__nv_bfloat16*)nullptr);
    } else if (G > 1024) {
        if (X) beam_select_kernel<true, 512><<<G, 512, 0, s>>>(offsets, tasks, devs, scale, logits, c, nx, B, R, GS, pos, x);
        else beam_select_kernel<false, 512><<<G, 512, 0, s>>>(offsets, tasks, devs, scale, logits, c, nx, B, R, GS, pos, nullptr);
    } else {
        if (X) beam_select_kernel<true, 1024><<<G, 1024, 0, s>>>(offsets, tasks, devs, scale, logits, c, nx, B, R, GS, pos, x);
        else beam_select_kernel<false, 1024><<<G, 1024, 0, s>>>(offsets, tasks, devs, scale, logits, c, nx, B, R, GS, pos, nullptr);
    }
    return cudaGetLastError();
}

cudaError_t beam_finish(const int32_t* offsets, const int32_t* status, const void* st, int G,
                        int B, const int32_t* heur_ms, int32_t* orders, int32_t* ms,
                        int32_t* beam_won, cudaStream_t s)
{
    beam_finish_kernel<<<(G + 127) / 128, 128, 0, s>>>(offsets, status,
                                                       static_cast<const BeamState*>(st), G, B,
                                                       heur_ms, orders, ms, beam_won);
    return cudaGetLastError();
}

cudaError_t beam_refine(const tm_task* tasks, const int32_t* offsets, const tm_device* devs,
                        const int32_t* status, const void* st, int G, int B, int K,
                        const int32_t* heur_ms, int32_t* orders, int32_t* ms, int32_t* beam_won,
                        cudaStream_t s)
{
    beam_refine_kernel<<<G, 32 * (K + 1), 0, s>>>(tasks, offsets, devs, status,
                                                  static_cast<const BeamState*>(st), B, K, heur_ms,
                                                  orders, ms, beam_won);
    return cudaGetLastError();
}

cudaError_t rank_rows(const tm_task* tasks, const int32_t* offsets, int G, const tm_device* devs,
                      const int32_t* orders, const tm_stats* stats, int64_t* row_base,
                      int32_t* state_base, int64_t M, int S, bf16_raw* X, int32_t* state_off,
                      int32_t* target, int32_t* status, cudaStream_t s)
{
    rows_scan_kernel<<<1, 1024, 0, s>>>(offsets, G, row_base, state_base);
    const int64_t M_pad = (M + 15) / 16 * 16;
    const int64_t threads = (int64_t)(G > 0 ? G : 1) * 32;
    rows_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(
        tasks, offsets, G, devs, orders, stats, row_base, state_base, M, M_pad, S,
        reinterpret_cast<__nv_bfloat16*>(X), state_off, target, status);
    return cudaGetLastError();
}

}  // namespace tmgpu

// exhaustive.cu -- evaluates the makespan of every one of the n! orders of
// each task group and reduces them to best / worst / sum (the brute-force
// search of Sec. 1 of the paper; "NoReorder" best / mean / worst of Sec. 6.2).
//
// Decomposition.  Orders are numbered by lexicographic rank.  For a group
// of n >= 5 tasks a WORK ITEM fixes the first n - L positions (L = the
// plan's levels, L! orders per item); its index p is the mixed-radix
// (Lehmer) number of that prefix, so item p covers ranks [p L!, (p+1) L!).
// A thread decodes the prefix, runs the recurrence over it, then walks the
// remaining L positions depth-first: the first L - 4 levels by loops over
// the ascending list of unused tasks, and the last 4 as a fully unrolled
// tree over four register-resident tasks (a CHUNK of 24 orders, chunk index
// = rank / 24).  Every tree node costs one step of the recurrence, so the
// whole group costs about e * n! steps instead of n * n!.
//
// Reduction.  Each thread keeps the min / max makespan, the first chunk
// where each was reached (its chunks are visited in increasing rank), and
// the sum; it flushes them with 64-bit atomics as keys (value << 32 | chunk)
// so that the smallest key is the best value with the lowest chunk.  A
// finalize kernel re-evaluates the winning chunks (24 orders each) to find
// the exact first rank, and handles groups of n <= 4 outright.
#include <algorithm>

#include "tm_device.cuh"

namespace tmgpu {
namespace {

constexpr int kEnumBlock = 256;
constexpr unsigned kFull = 0xFFFFFFFFu;

__global__ void prep_kernel(const tm_task* __restrict__ tasks,
                            const int32_t* __restrict__ offsets,
                            const tm_device* __restrict__ devs, int G,
                            GroupInfo* __restrict__ info, int4* __restrict__ tbl)
{
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    GroupInfo gi;
    gi.off = offsets[g];
    gi.n = offsets[g + 1] - gi.off;
    gi.hs = 0;
    gi.dinit = 0;
    gi.pad0 = gi.pad1 = gi.pad2 = 0;
    gi.status = check_group(tasks + gi.off, gi.n, devs[g].dma_engines,
                            TM_MAX_EXHAUSTIVE, &gi.hs, &gi.dinit);
    info[g] = gi;
    if (gi.status == 0)
        for (int i = 0; i < gi.n; ++i) {
            tm_task t = tasks[gi.off + i];
            tbl[gi.off + i] = make_int4(t.htd, t.k, t.dth, 0);
        }
}

struct LaneAcc {
    int32_t best, worst;
    uint32_t best_chunk, worst_chunk;
    unsigned long long sum;
    __device__ __forceinline__ void reset()
    {
        best = INT32_MAX;
        worst = -1;
        best_chunk = worst_chunk = 0;
        sum = 0;
    }
};

__device__ __forceinline__ void flush(LaneAcc& a, unsigned long long* acc, int g)
{
    if (a.worst < 0) return;
    atomicMin(&acc[3 * g + 0], ((unsigned long long)(uint32_t)a.best << 32) | a.best_chunk);
    atomicMax(&acc[3 * g + 1],
              ((unsigned long long)(uint32_t)a.worst << 32) | (kFull - a.worst_chunk));
    atomicAdd(&acc[3 * g + 2], a.sum);
}

// Last two positions: task a then task b.  After b every HtD has run, so
// the HtD end is the group's HtD sum hs.
__device__ __forceinline__ int32_t last_two(Eng s, int4 a, int4 b, int32_t hs)
{
    int32_t h3 = s.h + a.x;
    int32_t k3 = max(s.k, h3) + a.y;
    int32_t d3 = max(s.d, k3) + a.z;
    int32_t k4 = max(k3, hs) + b.y;
    return max(d3, k4) + b.z;
}

// The 24 orders of four tasks appended to state s.
__device__ __forceinline__ void chunk4(Eng s, const int4 (&t)[4], int32_t hs,
                                       int32_t& cmin, int32_t& cmax,
                                       unsigned long long& csum)
{
#pragma unroll
    for (int x = 0; x < 4; ++x) {
        Eng s1 = step(s, t[x].x, t[x].y, t[x].z);
#pragma unroll
        for (int y = 0; y < 4; ++y) {
            if (y == x) continue;
            Eng s2 = step(s1, t[y].x, t[y].y, t[y].z);
            // the two tasks left, z < w
            const int z = (x != 0 && y != 0) ? 0 : ((x != 1 && y != 1) ? 1 : 2);
            const int w = 6 - x - y - z;
            int32_t m1 = last_two(s2, t[z], t[w], hs);
            int32_t m2 = last_two(s2, t[w], t[z], hs);
            cmin = min(cmin, min(m1, m2));
            cmax = max(cmax, max(m1, m2));
            // each makespan <= INT32_MAX, so a pair fits in 32 bits
            csum += (uint32_t)m1 + (uint32_t)m2;
        }
    }
}

template <int Q>
__device__ __forceinline__ void walk(Eng s, uint64_t list, const int4* __restrict__ tbl,
                                     int32_t hs, uint32_t& chunk, LaneAcc& a)
{
    if constexpr (Q == 0) {
        int4 t[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) t[i] = tbl[nib_get(list, i)];
        int32_t cmin = INT32_MAX, cmax = -1;
        unsigned long long csum = 0;
        chunk4(s, t, hs, cmin, cmax, csum);
        if (cmin < a.best) { a.best = cmin; a.best_chunk = chunk; }
        if (cmax > a.worst) { a.worst = cmax; a.worst_chunk = chunk; }
        a.sum += csum;
        ++chunk;
    } else {
#pragma unroll 1
        for (int c = 0; c < Q + 4; ++c) {
            int4 t = tbl[nib_get(list, c)];
            walk<Q - 1>(step(s, t.x, t.y, t.z), nib_remove(list, c), tbl, hs, chunk, a);
        }
    }
}

template <int LEVELS>
__device__ __forceinline__ void eval_item(const GroupInfo& gi, const int4* __restrict__ tbl,
                                          uint32_t p, LaneAcc& a)
{
    const int n = gi.n;
    const int M = min(n, LEVELS);
    const int P = n - M;
    uint32_t chunk = p * (uint32_t)(factorial_u64(M) / 24);
    // Lehmer digits of the prefix, least significant (position P-1) first.
    uint32_t digits = 0;
    for (int i = P - 1; i >= 0; --i) {
        uint32_t r = (uint32_t)(n - i);
        uint32_t q = p / r;
        digits |= (p - q * r) << (4 * i);
        p = q;
    }
    uint64_t list = nib_identity(n);
    Eng s{0, 0, gi.dinit};
    for (int i = 0; i < P; ++i) {
        int c = (digits >> (4 * i)) & 0xF;
        int4 t = tbl[nib_get(list, c)];
        list = nib_remove(list, c);
        s = step(s, t.x, t.y, t.z);
    }
    const int q = M - 4;
    if constexpr (LEVELS >= 5) { if (q == 1) walk<1>(s, list, tbl, gi.hs, chunk, a); }
    if constexpr (LEVELS >= 6) { if (q == 2) walk<2>(s, list, tbl, gi.hs, chunk, a); }
    if constexpr (LEVELS >= 7) { if (q == 3) walk<3>(s, list, tbl, gi.hs, chunk, a); }
}

template <int LEVELS>
__global__ void __launch_bounds__(kEnumBlock)
enum_kernel(const GroupInfo* __restrict__ info, const int4* __restrict__ tbl,
            const uint32_t* __restrict__ item_base, int G, uint32_t total_items,
            uint32_t per_thread, unsigned long long* __restrict__ acc)
{
    uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint64_t first = t * per_thread;
    if (first >= total_items) return;
    uint32_t i = (uint32_t)first;
    uint32_t end = (uint32_t)min(first + per_thread, (uint64_t)total_items);
    // the group holding item i: the largest g with item_base[g] <= i
    int lo = 0, hi = G;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (item_base[mid] <= i) lo = mid; else hi = mid;
    }
    int g = lo;
    uint32_t gbase = item_base[g], gend = item_base[g + 1];
    GroupInfo gi = info[g];
    LaneAcc a;
    a.reset();
    for (; i < end; ++i) {
        while (i >= gend) {
            flush(a, acc, g);
            a.reset();
            ++g;
            gbase = gend;
            gend = item_base[g + 1];
            gi = info[g];
        }
        if (gi.status != 0) continue;
        eval_item<LEVELS>(gi, tbl + gi.off, i - gbase, a);
    }
    flush(a, acc, g);
}

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
    if (n <= 4) {
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
        uint32_t bchunk = (uint32_t)mk, wchunk = kFull - (uint32_t)xk;
        const uint64_t chunks = factorial_u64(n) / 24;
        ok = bchunk < chunks && wchunk < chunks;
        if (!ok) bchunk = wchunk = 0;
        bool live = lane < 24;
        int32_t mb = live ? makespan_of_rank(t, n, gi.dinit, bchunk * 24 + lane, nullptr) : -2;
        int32_t mw = live ? makespan_of_rank(t, n, gi.dinit, wchunk * 24 + lane, nullptr) : -2;
        unsigned bb = __ballot_sync(kFull, live && mb == best);
        unsigned wb = __ballot_sync(kFull, live && mw == worst);
        ok = ok && bb != 0 && wb != 0;
        best_rank = bchunk * 24 + (bb ? __ffs(bb) - 1 : 0);
        worst_rank = wchunk * 24 + (wb ? __ffs(wb) - 1 : 0);
        __syncwarp();
        if (lane == 0) { A[0] = ~0ull; A[1] = 0; A[2] = 0; }
    }
    if (lane != 0) return;
    if (!ok) {  // the reduction words disagree with a re-evaluation: never expected
        if (status) status[g] = TM_ECUDA;
        return;
    }
    tm_stats st;
    st.best = best;
    st.worst = worst;
    st.sum = (int64_t)sum;
    st.mean = (double)(int64_t)sum / (double)factorial_u64(n);
    st.best_rank = best_rank;
    st.worst_rank = worst_rank;
    for (int i = 0; i < 16; ++i) st.best_order[i] = st.worst_order[i] = 0xFF;
    makespan_of_rank(t, n, gi.dinit, best_rank, st.best_order);
    makespan_of_rank(t, n, gi.dinit, worst_rank, st.worst_order);
    stats[g] = st;
    if (status) status[g] = 0;
}

template <int LEVELS>
cudaError_t launch_enum(const Plan& p, cudaStream_t stream)
{
    uint32_t blocks = (p.threads + kEnumBlock - 1) / kEnumBlock;
    enum_kernel<LEVELS><<<blocks, kEnumBlock, 0, stream>>>(
        p.d_info, p.d_tbl, p.d_item_base, p.G, p.total_items, p.items_per_thread, p.d_acc);
    return cudaGetLastError();
}

}  // namespace

int exhaustive_resident_threads(int levels, int device)
{
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    cudaError_t e = cudaErrorInvalidValue;
    switch (levels) {
    case 5: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, enum_kernel<5>, kEnumBlock, 0); break;
    case 6: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, enum_kernel<6>, kEnumBlock, 0); break;
    case 7: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, enum_kernel<7>, kEnumBlock, 0); break;
    default: break;
    }
    if (e != cudaSuccess || sms <= 0 || per_sm <= 0) return 0;
    return sms * per_sm * kEnumBlock;
}

int exhaustive_launch_count(const Plan& p)
{
    return p.total_items > 0 ? 3 : 2;
}

cudaError_t launch_exhaustive(const Plan& p, const tm_task* d_tasks, const tm_device* d_devs,
                              tm_stats* d_stats, int32_t* d_status, cudaStream_t stream)
{
    if (p.G == 0) return cudaSuccess;
    prep_kernel<<<(p.G + 127) / 128, 128, 0, stream>>>(d_tasks, p.d_offsets, d_devs, p.G,
                                                       p.d_info, p.d_tbl);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (p.total_items > 0) {
        if (p.ev_before && (e = cudaEventRecord(p.ev_before, stream)) != cudaSuccess) return e;
        switch (p.levels) {
        case 5: e = launch_enum<5>(p, stream); break;
        case 6: e = launch_enum<6>(p, stream); break;
        case 7: e = launch_enum<7>(p, stream); break;
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

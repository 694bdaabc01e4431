// overlap.cu -- the partial-overlap variant of the model (Sec. 4.2.1, Fig. 6):
// while an HtD and a DtH transfer run at the same time (two DMA engines),
// each progresses at rate_num / rate_den of its full speed, and the running
// transfers' end times are re-estimated whenever that changes.  The paper
// gives no formula for the slowdown; the reading here keeps time on whole
// nanoseconds: a transfer of d ns is d * rate_den units of work, moving
// rate_den units per ns alone and rate_num units per ns while overlapped, and
// it ends at the first whole ns by which its work is done.  Kernels never
// slow down, and with one DMA engine no two transfers ever run together, so
// that device is the plain model.
//
// The max-plus decomposition of the plain model does not hold here (a
// transfer's speed depends on what the other engine does), so every order is
// an event loop over the three engines: at each step the free engines take
// their queue's next command if its dependency has ended, the speeds follow
// from which transfers run, and time jumps to the earliest end.  Once the
// last HtD has ended nothing overlaps any more and the rest is the plain
// recurrence.
//
//   overlap_predict_kernel   one given order per group (thread per group)
//   ovl_prep_kernel          per group: input checks, padded task table,
//                            reduction words
//   ovl_enum_kernel          every order of every group: a thread walks a
//                            run of consecutive ranks (lexicographic successor
//                            after the first unranking), resuming each order's
//                            loop where it first differs from the previous
//                            one, and reduces them
//   ovl_finalize_kernel      reduction words -> tm_stats
#include <algorithm>
#include <climits>
#include <vector>

#include "tm_device.cuh"

namespace tmgpu {
namespace {

constexpr int kOvlMaxRate = 1024;
constexpr int kOvlBlock = 128;
constexpr uint32_t kRanksPerThread = 64;

// Exact ceil(x / v) for 1 <= v <= 1024: a multiply-high by floor((2^B - 1) / v)
// for B-bit x (division by invariant integers, Granlund and Montgomery, PLDI
// 1994), whose quotient is at most two below floor(x / v), then corrected by
// the exact remainder.
struct Div {
    unsigned long long v, m;   // m for 64-bit numerators (x < 2^62)
    uint32_t m32;              // m for 32-bit numerators (x < 2^31)
};
__host__ __device__ inline Div make_div(unsigned long long v)
{
    return Div{v, v <= 1 ? 0ull : (~0ull) / v, v <= 1 ? 0u : 0xFFFFFFFFu / (uint32_t)v};
}
__device__ __forceinline__ long long ceil_div(long long x, const Div& d)
{
    if (d.v <= 1) return x;
    const unsigned long long ux = (unsigned long long)x;
    unsigned long long q = __umul64hi(ux, d.m);
    unsigned long long r = ux - q * d.v;
    if (r >= d.v) { q += 1; r -= d.v; }
    if (r >= d.v) { q += 1; r -= d.v; }
    return (long long)(q + (r != 0ull));
}
__device__ __forceinline__ int32_t ceil_div(int32_t x, const Div& d)
{
    if (d.v <= 1) return x;
    const uint32_t v = (uint32_t)d.v, ux = (uint32_t)x;
    uint32_t q = __umulhi(ux, d.m32);
    uint32_t r = ux - q * v;
    if (r >= v) { q += 1; r -= v; }
    if (r >= v) { q += 1; r -= v; }
    return (int32_t)(q + (r != 0u));
}

// Total time of one order (tasks in `tbl`, order as nibbles, position 0
// lowest) on two DMA engines under the partial-overlap rule.  W is the type
// of times and work left: int32_t when every transfer's work plus one rate
// step stays below 2^31 (checked per group), else 64-bit.
template <typename W>
__device__ W overlap_makespan(const int4* __restrict__ tbl, int n, uint64_t order, const Div& slow,
                              const Div& full)
{
    const W rs = (W)slow.v, rf = (W)full.v;
    int ih = 0, ik = 0, id = 0;          // next position each queue starts
    bool hb = false, kb = false, db = false;
    W hl = 0, kl = 0, dl = 0;            // work left: transfers in units, kernel in ns
    W T = 0;
    for (;;) {
        if (!hb && ih < n) { hb = true; hl = (W)tbl[nib_get(order, ih)].x * rf; }
        // positions below ih (ik) have finished their HtD (kernel)
        if (!kb && ik < ih) { kb = true; kl = tbl[nib_get(order, ik)].y; }
        if (!db && id < ik) { db = true; dl = (W)tbl[nib_get(order, id)].z * rf; }
        if (!hb && !kb && !db) break;
        const bool both = hb && db;
        const Div& v = both ? slow : full;
        const W rate = both ? rs : rf;
        W next = sizeof(W) == 4 ? (W)INT32_MAX : (W)LLONG_MAX;
        if (hb) next = min(next, (W)(T + ceil_div(hl, v)));
        if (kb) next = min(next, (W)(T + kl));
        if (db) next = min(next, (W)(T + ceil_div(dl, v)));
        const W dt = next - T;
        T = next;
        if (hb) { hl -= rate * dt; if (hl <= 0) { hb = false; ++ih; } }
        if (kb) { kl -= dt; if (kl <= 0) { kb = false; ++ik; } }
        if (db) { dl -= rate * dt; if (dl <= 0) { db = false; ++id; } }
    }
    return T;
}

// The event loop's state at the instant the HtD queue turns to position p,
// before any command starts at that instant: everything up to then depends
// only on the tasks at positions < p, so every order that shares them can
// resume from it.  q packs ik | id << 8 | kernel busy << 16 | DtH busy << 17.
template <typename W>
struct OvlSnap {
    W T, kl, dl;
    uint32_t q;
};

// overlap_makespan resumed from snap[from] (snap[0] is the empty start);
// on the way it stores the snapshots of positions from + 1 .. n - 1.  Once
// the last HtD has ended no two transfers overlap any more, so the rest is
// the plain recurrence from the engines' state: kernels back to back, each
// DtH at full speed after its kernel and the DtH before it.
template <typename W>
__device__ W overlap_makespan_from(const int4* __restrict__ tbl, int n, uint64_t order,
                                   const Div& slow, const Div& full, OvlSnap<W>* snap, int from)
{
    const W rs = (W)slow.v, rf = (W)full.v;
    const OvlSnap<W> s0 = snap[from];
    int ih = from, ik = (int)(s0.q & 0xFFu), id = (int)((s0.q >> 8) & 0xFFu);
    bool hb = false, kb = ((s0.q >> 16) & 1u) != 0u, db = ((s0.q >> 17) & 1u) != 0u;
    W hl = 0, kl = s0.kl, dl = s0.dl;
    W T = s0.T;
    while (ih < n) {
        if (!hb && ih < n) {
            if (ih > from)
                snap[ih] = OvlSnap<W>{T, kl, dl, (uint32_t)ik | ((uint32_t)id << 8) |
                                                     ((uint32_t)kb << 16) | ((uint32_t)db << 17)};
            hb = true;
            hl = (W)tbl[nib_get(order, ih)].x * rf;
        }
        if (!kb && ik < ih) { kb = true; kl = tbl[nib_get(order, ik)].y; }
        if (!db && id < ik) { db = true; dl = (W)tbl[nib_get(order, id)].z * rf; }
        const bool both = db;            // an HtD runs throughout this loop
        const Div& v = both ? slow : full;
        const W rate = both ? rs : rf;
        W next = (W)(T + ceil_div(hl, v));
        if (kb) next = min(next, (W)(T + kl));
        if (db) next = min(next, (W)(T + ceil_div(dl, v)));
        const W dt = next - T;
        T = next;
        hl -= rate * dt;
        if (hl <= 0) { hb = false; ++ih; }
        if (kb) { kl -= dt; if (kl <= 0) { kb = false; ++ik; } }
        if (db) { dl -= rate * dt; if (dl <= 0) { db = false; ++id; } }
    }
    // the tail: every HtD has ended by T
    W kfree = kb ? (W)(T + kl) : T;      // the kernel engine frees
    int kp = kb ? ik + 1 : ik;           // next kernel to start
    W dfree = db ? (W)(T + ceil_div(dl, full)) : T;
    for (int p = db ? id + 1 : id; p < n; ++p) {
        W ke = T;                        // kernels below ik ended by T
        if (p == ik && kb) {
            ke = kfree;
        } else if (p >= ik) {
            for (; kp <= p; ++kp) kfree += (W)tbl[nib_get(order, kp)].y;
            ke = kfree;
        }
        dfree = max(dfree, ke) + (W)tbl[nib_get(order, p)].z;
    }
    return max(dfree, kfree);
}

// Whether the 32-bit loop is exact for a group: every transfer's work
// (duration x den) plus one step of the fastest rate below 2^31.  (Times
// stay below the group's bound, itself below 2^31.)
__device__ __forceinline__ bool fits32(const tm_task* tasks, int n, int32_t den)
{
    long long mx = 0;
    for (int i = 0; i < n; ++i) mx = max(mx, (long long)max(tasks[i].htd, tasks[i].dth));
    return mx * den + den <= INT32_MAX;
}

// Plain model (one DMA engine, or full rate): the closed-form recurrence.
__device__ __forceinline__ long long plain_makespan(const int4* __restrict__ tbl, int n,
                                                    uint64_t order, int32_t dinit)
{
    Eng s{0, 0, dinit};
    for (int i = 0; i < n; ++i) {
        const int4 t = tbl[nib_get(order, i)];
        s = step(s, t.x, t.y, t.z);
    }
    return s.d;
}

// Input check of a group under the overlap rule: the plain checks, and the
// bound on every time the loop can reach (all transfers at the slow rate).
__device__ int overlap_check(const tm_task* tasks, int n, int dma, int nmax, int32_t num,
                             int32_t den, int32_t* hs_out, int32_t* dinit_out)
{
    int st = check_group(tasks, n, dma, nmax, hs_out, dinit_out);
    if (st != 0) return st;
    long long bound = 0;
    for (int i = 0; i < n; ++i) {
        const tm_task t = tasks[i];
        bound += t.k + ((long long)t.htd * den + num - 1) / num + ((long long)t.dth * den + num - 1) / num;
    }
    return bound > INT32_MAX ? TM_EOVERFLOW : 0;
}

__global__ void overlap_predict_kernel(const tm_task* __restrict__ tasks,
                                       const int32_t* __restrict__ offsets, int G,
                                       const int32_t* __restrict__ orders,
                                       const tm_device* __restrict__ devs, int32_t num,
                                       int32_t den, int32_t* __restrict__ out,
                                       int32_t* __restrict__ status)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    const int off = offsets[g], n = offsets[g + 1] - off;
    const int dma = devs[g].dma_engines;
    int32_t hs = 0, dinit = 0;
    int st = overlap_check(tasks + off, n, dma, TM_MAX_TASKS, num, den, &hs, &dinit);
    uint32_t seen = 0;
    uint64_t order = 0;
    for (int i = 0; st == 0 && i < n; ++i) {
        const int o = orders[off + i];
        if (o < 0 || o >= n || ((seen >> o) & 1u)) st = TM_EINVAL;
        else { seen |= 1u << o; order |= (uint64_t)o << (4 * i); }
    }
    if (st != 0) {
        if (status) status[g] = st;
        return;
    }
    // a padded copy of the group's tasks is not needed for one order: read
    // them through a local int4 view
    int4 tb[TM_MAX_TASKS];
    for (int i = 0; i < n; ++i) tb[i] = make_int4(tasks[off + i].htd, tasks[off + i].k, tasks[off + i].dth, 0);
    long long ms;
    if (dma == 1 || num == den) ms = plain_makespan(tb, n, order, dinit);
    else if (fits32(tasks + off, n, den)) ms = overlap_makespan<int32_t>(tb, n, order, make_div(num), make_div(den));
    else ms = overlap_makespan<long long>(tb, n, order, make_div(num), make_div(den));
    out[g] = (int32_t)ms;
    if (status) status[g] = 0;
}

// ---- exhaustive search -------------------------------------------------------

struct OvlInfo {
    int32_t off, n, dinit, status;
    int32_t w32, pad0, pad1, pad2;   // w32: the 32-bit loop is exact for this group
};

__global__ void ovl_prep_kernel(const tm_task* __restrict__ tasks,
                                const int32_t* __restrict__ offsets, int G,
                                const tm_device* __restrict__ devs, int32_t num, int32_t den,
                                OvlInfo* __restrict__ info, int4* __restrict__ tbl,
                                unsigned long long* __restrict__ acc,
                                int32_t* __restrict__ status)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    const int off = offsets[g], n = offsets[g + 1] - off;
    int32_t hs = 0, dinit = 0;
    const int st = overlap_check(tasks + off, n, devs[g].dma_engines, TM_MAX_EXHAUSTIVE, num, den,
                                 &hs, &dinit);
    OvlInfo oi;
    oi.off = off;
    oi.n = n;
    oi.dinit = devs[g].dma_engines == 1 ? dinit : -1;   // -1: the overlap loop
    oi.status = st;
    oi.w32 = st == 0 && fits32(tasks + off, n, den) ? 1 : 0;
    oi.pad0 = oi.pad1 = oi.pad2 = 0;
    if (st == 0)
        for (int i = 0; i < n; ++i)
            tbl[off + i] = make_int4(tasks[off + i].htd, tasks[off + i].k, tasks[off + i].dth, 0);
    info[g] = oi;
    unsigned long long* A = acc + 4 * (size_t)g;
    A[0] = ~0ull;
    A[1] = 0ull;
    A[2] = 0ull;
    if (st != 0 && status) status[g] = st;
}

// Lexicographic successor of a permutation held as nibbles (n >= 2); the
// last permutation wraps to the first, which the caller never asks for.
__device__ __forceinline__ uint64_t next_order(uint64_t o, int n)
{
    int i = n - 2;
    while (i >= 0 && nib_get(o, i) > nib_get(o, i + 1)) --i;
    if (i < 0) return o;
    int j = n - 1;
    const int ai = nib_get(o, i);
    while (nib_get(o, j) < ai) --j;
    // swap positions i and j
    const int aj = nib_get(o, j);
    o &= ~((0xFull << (4 * i)) | (0xFull << (4 * j)));
    o |= ((uint64_t)aj << (4 * i)) | ((uint64_t)ai << (4 * j));
    // reverse positions i+1 .. n-1
    for (int a = i + 1, b = n - 1; a < b; ++a, --b) {
        const uint64_t va = (o >> (4 * a)) & 0xF, vb = (o >> (4 * b)) & 0xF;
        o &= ~((0xFull << (4 * a)) | (0xFull << (4 * b)));
        o |= (vb << (4 * a)) | (va << (4 * b));
    }
    return o;
}

__device__ __forceinline__ uint64_t unrank(uint32_t rank, int n)
{
    uint64_t list = nib_identity(n), o = 0;
    for (int i = 0; i < n; ++i) {
        const int k = n - 1 - i;
        const uint32_t c = min(div_fact(rank, k), (uint32_t)k);
        rank -= c * (uint32_t)factorial_u64(k);
        o |= (uint64_t)nib_get(list, (int)c) << (4 * i);
        list = nib_remove(list, (int)c);
    }
    return o;
}

struct OvlAcc {
    int32_t best, worst;
    uint32_t best_rank, worst_rank;
    unsigned long long sum;
};

__device__ __forceinline__ void ovl_flush(const OvlAcc& a, unsigned long long* __restrict__ acc,
                                          int g)
{
    if (a.worst < 0) return;
    unsigned long long* A = acc + 4 * (size_t)g;
    atomicMin(&A[0], ((unsigned long long)(uint32_t)a.best << 32) | a.best_rank);
    atomicMax(&A[1], ((unsigned long long)(uint32_t)a.worst << 32) | (0xFFFFFFFFu - a.worst_rank));
    atomicAdd(&A[2], a.sum);
}

__device__ __forceinline__ void ovl_take(OvlAcc& a, int32_t m, uint32_t rank)
{
    a.sum += (unsigned long long)(uint32_t)m;
    if (m < a.best) { a.best = m; a.best_rank = rank; }       // ranks rise: first kept
    if (m > a.worst) { a.worst = m; a.worst_rank = rank; }
}

// `count` consecutive orders from `order` (rank `rank`) under the plain
// model (one DMA engine, or full rate).
__device__ void ovl_run_plain(const int4* __restrict__ t, int n, uint64_t order, uint32_t rank,
                              uint32_t count, int32_t dinit, OvlAcc& a)
{
    for (uint32_t c = 0; c < count; ++c, ++rank) {
        ovl_take(a, (int32_t)plain_makespan(t, n, order, max(dinit, 0)), rank);
        if (c + 1 < count) order = next_order(order, n);
    }
}

// The same under the partial-overlap rule: each order resumes the event loop
// from the snapshot at the first position where it differs from the one
// before (the lexicographic successor changes the last ~e positions on
// average), instead of simulating from time 0.
template <typename W>
__device__ void ovl_run(const int4* __restrict__ t, int n, uint64_t order, uint32_t rank,
                        uint32_t count, const Div& slow, const Div& full, OvlAcc& a)
{
    OvlSnap<W> snap[TM_MAX_EXHAUSTIVE];
    snap[0] = OvlSnap<W>{0, 0, 0, 0u};
    int from = 0;
    for (uint32_t c = 0; c < count; ++c, ++rank) {
        ovl_take(a, (int32_t)overlap_makespan_from<W>(t, n, order, slow, full, snap, from), rank);
        if (c + 1 < count) {
            const uint64_t nx = next_order(order, n);
            from = (__ffsll((long long)(order ^ nx)) - 1) >> 2;   // first position that changes
            order = nx;
        }
    }
}

// Thread t walks global order indices [t R, (t + 1) R) (base[g] = first index
// of group g, base[G] = total).
__global__ void __launch_bounds__(kOvlBlock)
ovl_enum_kernel(const unsigned long long* __restrict__ base, int G,
                const OvlInfo* __restrict__ info, const int4* __restrict__ tbl, int32_t num,
                int32_t den, unsigned long long* __restrict__ acc)
{
    const unsigned long long total = base[G];
    const unsigned long long x0 = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) *
                                  kRanksPerThread;
    if (x0 >= total) return;
    const unsigned long long x1 = min(x0 + kRanksPerThread, total);
    int lo = 0, hi = G;                     // the group holding x0
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (base[mid] <= x0) lo = mid; else hi = mid;
    }
    int g = lo;
    const Div slow = make_div(num), full = make_div(den);
    unsigned long long x = x0;
    while (x < x1) {
        while (base[g + 1] <= x) ++g;
        const unsigned long long gend = min(x1, base[g + 1]);
        const OvlInfo oi = info[g];
        if (oi.status != 0) { x = gend; continue; }
        const int4* t = tbl + oi.off;
        const uint32_t rank = (uint32_t)(x - base[g]);
        const uint64_t order = unrank(rank, oi.n);
        OvlAcc a{INT32_MAX, -1, 0xFFFFFFFFu, 0xFFFFFFFFu, 0ull};
        const uint32_t count = (uint32_t)(gend - x);
        if (oi.dinit >= 0 || num == den) ovl_run_plain(t, oi.n, order, rank, count, oi.dinit, a);
        else if (oi.w32) ovl_run<int32_t>(t, oi.n, order, rank, count, slow, full, a);
        else ovl_run<long long>(t, oi.n, order, rank, count, slow, full, a);
        x = gend;
        ovl_flush(a, acc, g);
    }
}

__global__ void ovl_finalize_kernel(const OvlInfo* __restrict__ info, const int4* __restrict__ tbl,
                                    int G, unsigned long long* __restrict__ acc,
                                    tm_stats* __restrict__ stats, int32_t* __restrict__ status)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    const OvlInfo oi = info[g];
    if (oi.status != 0) return;
    const unsigned long long* A = acc + 4 * (size_t)g;
    tm_stats st;
    st.best = (int32_t)(A[0] >> 32);
    st.worst = (int32_t)(A[1] >> 32);
    st.best_rank = (uint32_t)A[0];
    st.worst_rank = 0xFFFFFFFFu - (uint32_t)A[1];
    st.sum = (int64_t)A[2];
    st.mean = (double)(int64_t)A[2] / (double)factorial_u64(oi.n);
    const uint64_t nf = factorial_u64(oi.n);
    if (st.best_rank >= nf || st.worst_rank >= nf) {   // never expected
        if (status) status[g] = TM_ECUDA;
        return;
    }
    const uint64_t ob = unrank((uint32_t)st.best_rank, oi.n), ow = unrank((uint32_t)st.worst_rank, oi.n);
    for (int i = 0; i < 16; ++i) {
        st.best_order[i] = i < oi.n ? (uint8_t)nib_get(ob, i) : 0xFF;
        st.worst_order[i] = i < oi.n ? (uint8_t)nib_get(ow, i) : 0xFF;
    }
    stats[g] = st;
    if (status) status[g] = 0;
}

// Library-owned scratch of the exhaustive calls, one set per host thread.
struct OvlScratch {
    int device = -1;
    void* p = nullptr;
    size_t cap = 0;
    std::vector<unsigned long long> h_base;
    ~OvlScratch()
    {
        int d = 0;
        if (p && cudaGetDevice(&d) == cudaSuccess) cudaFree(p);
    }
};
thread_local OvlScratch t_ovl;

}  // namespace

cudaError_t launch_overlap_predict(const tm_task* d_tasks, const int32_t* d_offsets, int G,
                                   const int32_t* d_orders, const tm_device* d_devs, int32_t num,
                                   int32_t den, int32_t* d_makespans, int32_t* d_status,
                                   cudaStream_t s)
{
    if (G == 0) return cudaSuccess;
    overlap_predict_kernel<<<(G + 127) / 128, 128, 0, s>>>(d_tasks, d_offsets, G, d_orders, d_devs,
                                                          num, den, d_makespans, d_status);
    return cudaGetLastError();
}

// Enqueues the exhaustive search under the overlap rule.  h_offsets: host
// copy of d_offsets (group sizes already checked: 1..12).
int overlap_exhaustive(const tm_task* d_tasks, const int32_t* d_offsets, const int32_t* h_offsets,
                       int G, const tm_device* d_devs, int32_t num, int32_t den, tm_stats* d_stats,
                       int32_t* d_status, cudaStream_t s)
{
    if (G == 0) return TM_OK;
    OvlScratch& sc = t_ovl;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TM_ECUDA;
    const int T = h_offsets[G];
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t b_base = al((size_t)(G + 1) * 8), b_info = al((size_t)G * sizeof(OvlInfo)),
                 b_tbl = al((size_t)std::max(T, 1) * sizeof(int4)), b_acc = al((size_t)G * 32);
    const size_t need = b_base + b_info + b_tbl + b_acc;
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
    OvlInfo* d_info = reinterpret_cast<OvlInfo*>(p + b_base);
    int4* d_tbl = reinterpret_cast<int4*>(p + b_base + b_info);
    unsigned long long* d_acc = reinterpret_cast<unsigned long long*>(p + b_base + b_info + b_tbl);
    sc.h_base.assign((size_t)G + 1, 0ull);
    for (int g = 0; g < G; ++g)
        sc.h_base[g + 1] = sc.h_base[g] + factorial_u64(h_offsets[g + 1] - h_offsets[g]);
    // the pageable copy is staged before the call returns
    if (cudaMemcpyAsync(d_base, sc.h_base.data(), (size_t)(G + 1) * 8, cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
        return TM_ECUDA;
    ovl_prep_kernel<<<(G + 127) / 128, 128, 0, s>>>(d_tasks, d_offsets, G, d_devs, num, den, d_info,
                                                   d_tbl, d_acc, d_status);
    const unsigned long long total = sc.h_base[G];
    const unsigned long long threads = (total + kRanksPerThread - 1) / kRanksPerThread;
    if (threads > 0)
        ovl_enum_kernel<<<(unsigned)((threads + kOvlBlock - 1) / kOvlBlock), kOvlBlock, 0, s>>>(
            d_base, G, d_info, d_tbl, num, den, d_acc);
    ovl_finalize_kernel<<<(G + 127) / 128, 128, 0, s>>>(d_info, d_tbl, G, d_acc, d_stats, d_status);
    return cudaGetLastError() == cudaSuccess ? TM_OK : TM_ECUDA;
}

int overlap_rate_ok(int32_t num, int32_t den)
{
    return num >= 1 && den >= num && den <= kOvlMaxRate;
}

}  // namespace tmgpu

// tm_device.cuh -- device-side building blocks of the temporal execution
// model (Sec. 4.1 of the paper) in closed form.
//
// Appending task j to an order advances three engine-free times: the end of
// the last HtD (h), of the last kernel (k) and of the last DtH (d):
//     h' = h + htd_j
//     k' = max(k, h') + k_j          (K waits for its own HtD and the K queue)
//     d' = max(d, k') + dth_j        (DtH waits for its own K and the DtH queue)
// Starting from h = k = 0 and d = dinit, the makespan of an order is the
// final d.  With two DMA engines dinit = 0.  With one DMA engine the only
// transfer queue holds every HtD before any DtH (Sec. 3.2, Fig. 2), so the
// first DtH cannot start before sum(htd): dinit = sum(htd), and h stays the
// running HtD sum.  These recurrences are the event-driven simulation of
// Fig. 6 with every start time written as the max of the two ends it waits
// for; all values stay <= the group's duration sum, which the host checks
// fits in int32, so int32 add/max is exact.
#pragma once

#include <stdint.h>

#include "tm.h"
#include "tm_internal.h"

namespace tmgpu {

struct Eng {
    int32_t h, k, d;
};

__device__ __forceinline__ Eng step(Eng s, int32_t htd, int32_t k, int32_t dth)
{
    Eng r;
    r.h = s.h + htd;
    r.k = max(s.k, r.h) + k;
    r.d = max(s.d, r.k) + dth;
    return r;
}

// Per-group input check (the device twin of the host-side validation).
// Returns 0 or a tm_status code; on success writes the HtD sum and the
// initial DtH-free time.
__device__ __forceinline__ int check_group(const tm_task* tasks, int n,
                                           int dma, int nmax, int32_t* hs_out,
                                           int32_t* dinit_out)
{
    if (n < 1 || n > nmax) return TM_EINVAL;
    if (dma != 1 && dma != 2) return TM_EINVAL;
    int64_t total = 0, hs = 0;
    for (int i = 0; i < n; ++i) {
        tm_task t = tasks[i];
        if (t.htd < 0 || t.k < 0 || t.dth < 0) return TM_ENEG;
        total += (int64_t)t.htd + t.k + t.dth;
        hs += t.htd;
    }
    if (total > INT32_MAX) return TM_EOVERFLOW;
    *hs_out = (int32_t)hs;
    *dinit_out = dma == 1 ? (int32_t)hs : 0;
    return 0;
}

// Ascending list of up to 16 task indices packed as 4-bit nibbles.
__device__ __forceinline__ uint64_t nib_identity(int n)
{
    const uint64_t all = 0xFEDCBA9876543210ull;
    return n >= 16 ? all : (all & ((1ull << (4 * n)) - 1));
}

__device__ __forceinline__ int nib_get(uint64_t list, int c)
{
    return (int)((list >> (4 * c)) & 0xF);
}

// Removes entry c, shifting the later entries down.
__device__ __forceinline__ uint64_t nib_remove(uint64_t list, int c)
{
    uint64_t low = list & ((1ull << (4 * c)) - 1);
    uint64_t high = (list >> (4 * c + 4)) << (4 * c);
    return low | high;
}

// Division of a 32-bit numerator by k! (1 <= k <= 12) as one 64 x 64-bit
// multiply-high by ceil(2^64 / k!) (division by invariant integers using
// multiplication, Granlund and Montgomery, PLDI 1994): for r < 2^32 and a
// divisor d < 2^32 the error term stays below 2^-32 < 1/d, so the quotient
// is exact.
struct FactRecip {
    unsigned long long m[13];
};
constexpr FactRecip make_fact_recip()
{
    FactRecip r{};
    unsigned long long f = 1;
    for (int k = 0; k <= 12; ++k) {
        if (k > 1) f *= (unsigned long long)k;
        r.m[k] = f == 1 ? 0ull : (~0ull) / f + 1ull;   // k! = 1 handled apart
    }
    return r;
}
__constant__ FactRecip c_fact_recip = make_fact_recip();

__device__ __forceinline__ uint32_t div_fact(uint32_t r, int k)
{
    return k <= 1 ? r : (uint32_t)__umul64hi((unsigned long long)r, c_fact_recip.m[k]);
}

// Makespan of the order with lexicographic rank `rank` (n <= 12, rank < n!),
// generic and slow; writes the order to order_out if not NULL.  A rank out
// of range is clamped digit by digit, so table reads stay inside the group.
__device__ inline int32_t makespan_of_rank(const int4* tbl, int n, int32_t dinit,
                                           uint32_t rank, uint8_t* order_out)
{
    uint64_t list = nib_identity(n);
    Eng s{0, 0, dinit};
    for (int i = 0; i < n; ++i) {
        const int k = n - 1 - i;
        const uint32_t c = min(div_fact(rank, k), (uint32_t)k);
        rank -= c * (uint32_t)factorial_u64(k);
        int e = nib_get(list, (int)c);
        list = nib_remove(list, (int)c);
        if (order_out) order_out[i] = (uint8_t)e;
        int4 t = tbl[e];
        s = step(s, t.x, t.y, t.z);
    }
    return s.d;
}

// The same for a whole warp, each lane with its own rank, taking the task
// rows from the lanes instead of memory: lane j holds task j's row
// (j < n).  n must be the same on every lane and every lane must call.
__device__ inline int32_t makespan_of_rank_warp(int4 row, int n, int32_t dinit, uint32_t rank,
                                                uint8_t* order_out)
{
    uint64_t list = nib_identity(n);
    Eng s{0, 0, dinit};
    for (int i = 0; i < n; ++i) {
        const int k = n - 1 - i;
        const uint32_t c = min(div_fact(rank, k), (uint32_t)k);
        rank -= c * (uint32_t)factorial_u64(k);
        const int e = nib_get(list, (int)c);
        list = nib_remove(list, (int)c);
        if (order_out) order_out[i] = (uint8_t)e;
        const int32_t h = __shfl_sync(0xFFFFFFFFu, row.x, e);
        const int32_t kk = __shfl_sync(0xFFFFFFFFu, row.y, e);
        const int32_t dd = __shfl_sync(0xFFFFFFFFu, row.z, e);
        s = step(s, h, kk, dd);
    }
    return s.d;
}

}  // namespace tmgpu

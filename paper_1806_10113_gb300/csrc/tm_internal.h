// tm_internal.h -- data layout and launch helpers shared by the CUDA
// translation units of libtm.so.  Nothing here is visible through tm.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "tm.h"

namespace tmgpu {

// Per-group facts derived once per launch by the prep kernel.
struct GroupInfo {
    int32_t off;     // index of the group's first task
    int32_t n;       // number of tasks
    int32_t dinit;   // time the DtH stream becomes free before the first
                     // task: 0 with two DMA engines; with one engine the
                     // single transfer queue carries every HtD first, so it
                     // is the sum of HtD (Sec. 3.2, Fig. 2)
    int32_t hs;      // sum of HtD of the group
    int32_t status;  // 0 or a tm_status code
    int32_t pad0, pad1, pad2;
};

// Exhaustive-search plan (see tm_plan_create in tm.h).
struct Plan {
    int device = 0;
    int G = 0;
    int T = 0;                  // total tasks
    int levels = 5;             // orders enumerated per work item: levels!
    uint32_t total_items = 0;   // work items over all groups
    uint32_t items_per_thread = 1;
    uint32_t threads = 0;
    int launches = 0;
    int32_t* d_offsets = nullptr;         // [G + 1]
    uint32_t* d_item_base = nullptr;      // [G + 1] first work item of each group
    GroupInfo* d_info = nullptr;          // [G]
    int4* d_tbl = nullptr;                // [T] {htd, k, dth, 0}
    unsigned long long* d_acc = nullptr;  // [3 G] min key, max key, sum
    cudaEvent_t ev_before = nullptr;      // optional timing hook
    cudaEvent_t ev_after = nullptr;
};

// 0! .. 16!
__host__ __device__ inline uint64_t factorial_u64(int n)
{
    uint64_t f = 1;
    for (int i = 2; i <= n; ++i) f *= (uint64_t)i;
    return f;
}

// Launchers (return cudaError_t of the launch).
cudaError_t launch_exhaustive(const Plan& plan, const tm_task* d_tasks,
                              const tm_device* d_devs, tm_stats* d_stats,
                              int32_t* d_status, cudaStream_t stream);
int exhaustive_launch_count(const Plan& plan);
int exhaustive_resident_threads(int levels, int device);

cudaError_t launch_predict(const tm_task* d_tasks, const int32_t* d_offsets,
                           int G, const int32_t* d_orders,
                           const tm_device* d_devs, int32_t* d_makespans,
                           int32_t* d_status, cudaStream_t stream);

cudaError_t launch_heuristic(const tm_task* d_tasks, const int32_t* d_offsets,
                             int G, const tm_device* d_devs,
                             int32_t* d_orders, int32_t* d_makespans,
                             int32_t* d_status, cudaStream_t stream);

}  // namespace tmgpu

// heuristic.cu -- the Batch Reordering heuristic kernel (Sec. 5.1,
// Algorithm 1): half a warp per group (groups hold at most 16 tasks), so a
// warp runs two groups' dependent selection chains side by side; the
// per-group work is in heuristic.cuh.
#include "heuristic.cuh"

namespace tmgpu {
namespace {

__global__ void heuristic_kernel(const tm_task* __restrict__ tasks,
                                 const int32_t* __restrict__ offsets, int G,
                                 const tm_device* __restrict__ devs,
                                 int32_t* __restrict__ orders_out,
                                 int32_t* __restrict__ ms_out, int32_t* __restrict__ status)
{
    int g = (int)((blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 4);
    int lane = threadIdx.x & 15;
    if (g >= G) return;   // the whole half warp
    int off = offsets[g];
    heur::heuristic_group_seg<16>(tasks, off, offsets[g + 1] - off, devs[g].dma_engines, g, lane,
                                  orders_out, ms_out, status);
}

}  // namespace

cudaError_t launch_heuristic(const tm_task* d_tasks, const int32_t* d_offsets, int G,
                             const tm_device* d_devs, int32_t* d_orders, int32_t* d_makespans,
                             int32_t* d_status, cudaStream_t stream)
{
    if (G == 0) return cudaSuccess;
    uint64_t threads = (uint64_t)G * 16;
    heuristic_kernel<<<(unsigned)((threads + 127) / 128), 128, 0, stream>>>(
        d_tasks, d_offsets, G, d_devs, d_orders, d_makespans, d_status);
    return cudaGetLastError();
}

}  // namespace tmgpu

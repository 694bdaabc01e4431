// predict.cu -- makespan of one given order per group (Sec. 4.1 model).
// One thread per group runs the closed-form recurrence of tm_device.cuh.
#include "tm_device.cuh"

namespace tmgpu {
namespace {

__global__ void predict_kernel(const tm_task* __restrict__ tasks,
                               const int32_t* __restrict__ offsets, int G,
                               const int32_t* __restrict__ orders,
                               const tm_device* __restrict__ devs,
                               int32_t* __restrict__ out, int32_t* __restrict__ status)
{
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    int off = offsets[g];
    int n = offsets[g + 1] - off;
    int32_t hs = 0, dinit = 0;
    int st = check_group(tasks + off, n, devs[g].dma_engines, TM_MAX_TASKS, &hs, &dinit);
    uint32_t seen = 0;
    for (int i = 0; st == 0 && i < n; ++i) {
        int o = orders[off + i];
        if (o < 0 || o >= n || ((seen >> o) & 1u)) st = TM_EINVAL;
        else seen |= 1u << o;
    }
    if (st != 0) {
        if (status) status[g] = st;
        return;
    }
    Eng s{0, 0, dinit};
    for (int i = 0; i < n; ++i) {
        tm_task t = tasks[off + orders[off + i]];
        s = step(s, t.htd, t.k, t.dth);
    }
    out[g] = s.d;
    if (status) status[g] = 0;
}

}  // namespace

cudaError_t launch_predict(const tm_task* d_tasks, const int32_t* d_offsets, int G,
                           const int32_t* d_orders, const tm_device* d_devs,
                           int32_t* d_makespans, int32_t* d_status, cudaStream_t stream)
{
    if (G == 0) return cudaSuccess;
    predict_kernel<<<(G + 127) / 128, 128, 0, stream>>>(d_tasks, d_offsets, G, d_orders, d_devs,
                                                        d_makespans, d_status);
    return cudaGetLastError();
}

}  // namespace tmgpu

// refine.cu -- tm_refine_batch_dev: the exact-model descent of refine.cuh
// from the caller's orders, one warp per group.
#include "refine.cuh"

namespace tmgpu {
namespace {

constexpr int kRefineWarps = 4;

__global__ void __launch_bounds__(32 * kRefineWarps)
refine_kernel(const tm_task* __restrict__ tasks, const int32_t* __restrict__ offsets, int G,
              const tm_device* __restrict__ devs, int32_t* __restrict__ orders,
              int32_t* __restrict__ ms_out, int32_t* __restrict__ status)
{
    __shared__ int4 s_rows[kRefineWarps][16];
    __shared__ int4 s_pre[kRefineWarps][17];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = blockIdx.x * kRefineWarps + w;
    if (g >= G) return;   // the whole warp
    const int off = offsets[g], n = offsets[g + 1] - off;
    int32_t hs = 0, dinit = 0;
    int rc = check_group(tasks + off, n, devs[g].dma_engines, TM_MAX_TASKS, &hs, &dinit);
    // the given order must be a permutation of 0 .. n - 1
    uint64_t o = 0;
    if (rc == 0) {
        const int e = lane < n ? orders[off + lane] : 0;
        const bool bad = lane < n && (e < 0 || e >= n);
        const unsigned seen = __reduce_or_sync(0xFFFFFFFFu, lane < n && !bad ? 1u << e : 0u);
        if (__any_sync(0xFFFFFFFFu, bad) || seen != (n >= 32 ? 0xFFFFFFFFu : (1u << n) - 1u))
            rc = TM_EINVAL;
        for (int p = 0; p < n; ++p)
            o |= (uint64_t)(__shfl_sync(0xFFFFFFFFu, e, p) & 0xF) << (4 * p);
    }
    if (rc != 0) {
        if (lane == 0 && status) status[g] = rc;
        return;
    }
    if (lane < n) {
        const tm_task t = tasks[off + lane];
        s_rows[w][lane] = make_int4(t.htd, t.k, t.dth, 0);
    }
    __syncwarp();
    int32_t ms = refine::finish_order(o, n, 0, Eng{0, 0, dinit}, s_rows[w]);
    refine::descend(&o, &ms, n, dinit, s_rows[w], s_pre[w], lane);
    if (lane < n) orders[off + lane] = (int32_t)((o >> (4 * lane)) & 0xF);
    if (lane == 0) {
        if (ms_out) ms_out[g] = ms;
        if (status) status[g] = 0;
    }
}

}  // namespace
}  // namespace tmgpu

extern "C" int tm_refine_batch_dev(const tm_task* d_tasks, const int32_t* d_offsets, int G,
                                   const tm_device* d_devs, int32_t* d_orders,
                                   int32_t* d_makespans, int32_t* d_status, void* stream)
{
    using namespace tmgpu;
    if (G < 0) return TM_EINVAL;
    if (G == 0) return TM_OK;
    if (!d_tasks || !d_offsets || !d_devs || !d_orders) return TM_EINVAL;
    const unsigned blocks = (unsigned)((G + kRefineWarps - 1) / kRefineWarps);
    refine_kernel<<<blocks, 32 * kRefineWarps, 0, static_cast<cudaStream_t>(stream)>>>(
        d_tasks, d_offsets, G, d_devs, d_orders, d_makespans, d_status);
    return cudaGetLastError() == cudaSuccess ? TM_OK : TM_ECUDA;
}

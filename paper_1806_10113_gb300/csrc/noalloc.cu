// noalloc.cu -- tm_exhaustive_batch_noalloc: the exhaustive search for
// callers that cannot allocate device memory.
//
// Who needs it: a caller whose device memory is entirely reserved by
// another allocator (a framework's caching pool that owns the whole GPU),
// or one that cannot pay for cudaMalloc / cudaFree (cudaFree waits for the
// whole device) on its hot path, cannot create a tm_plan, because creating a
// plan allocates.  This entry point takes the caller's input and output
// buffers and keeps its own working memory in one fixed file-scope device
// array instead.
//
// The array is a static __device__ object of 1 MiB, so every GPU that
// loads the library holds it until the process exits.  Its size bounds the
// batch: at most TM_NOALLOC_MAX_GROUPS groups, TM_NOALLOC_MAX_TASKS tasks
// and TM_NOALLOC_MAX_SUBSETS 4-task subsets (sum of C(n, 4) over groups).
//
// Host code must not use the array's symbol as an address: on the host it
// names a stand-in object, not device memory.  The first call on each
// device, with that device current, does the set-up: it asks the runtime
// for the array's device address (cudaGetSymbolAddress) and loads every
// kernel the call can launch.  Under lazy module loading (the CUDA default)
// a module -- this file's, with the 1 MiB array, and the search's -- is only
// loaded, and its device memory only taken, when first used; doing it all
// in the set-up means no later call loads anything.  So make the first call
// before the caller's own allocator reserves the device's memory (or run
// with CUDA_MODULE_LOADING=EAGER, which loads every module at start-up), and
// before starting any stream capture.  The set-up is redone if the device's
// context changes (after cudaDeviceReset, for example); the same rules then
// apply to the first call after it.
//
// All calls share the one array, and it keeps whatever the previous call
// left there; each call re-initialises the parts that must start from a
// known value (offsets, work list, reduction words) on its stream before
// the search.  Two calls whose work overlaps on the GPU race on the array:
// serialise them (one stream, or events).
#include <cuda.h>

#include <mutex>

#include "tm_internal.h"

namespace tmgpu {
namespace {

constexpr int kMaxGroups = TM_NOALLOC_MAX_GROUPS;
constexpr int kPdmax = 4;
constexpr size_t kScratchBytes = (size_t)1 << 20;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct InitArgs {
    GroupPlan gp[kMaxGroups + 1];
    int G;
};

// Writes the batch's work layout into the scratch array and resets the
// reduction words, which the previous call may have left in any state.
__global__ void noalloc_init_kernel(InitArgs a, GroupPlan* gp, unsigned long long* acc)
{
    for (int i = threadIdx.x; i <= a.G; i += blockDim.x) gp[i] = a.gp[i];
    for (int i = threadIdx.x; i < kAccStride * a.G; i += blockDim.x)
        acc[i] = (i % kAccStride == 0) ? ~0ull : 0ull;
}

std::mutex g_mu;

// The context current on the calling thread, from the driver's
// cuCtxGetCurrent (found through the runtime, so the library does not link
// the driver library); nullptr if the driver does not offer it.
CUcontext current_context()
{
    using CtxGetCurrent = CUresult (*)(CUcontext*);
    static const CtxGetCurrent fn = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return static_cast<CtxGetCurrent>(nullptr);
        return reinterpret_cast<CtxGetCurrent>(f);
    }();
    CUcontext ctx = nullptr;
    if (fn && fn(&ctx) != CUDA_SUCCESS) ctx = nullptr;
    return ctx;
}

struct DeviceSetup {
    CUcontext ctx = nullptr;   // the context the set-up ran in
    void* addr = nullptr;      // device address of g_scratch in that context
};
DeviceSetup g_setup[64];       // per device ordinal

// Device address of g_scratch on `device` (current).  The first call, and
// the first after the device's context changed, also loads this file's
// kernel and the search's kernels.
int scratch_address(int device, unsigned char** out)
{
    if (device < 0 || device >= 64) return TM_EINVAL;
    std::lock_guard<std::mutex> lock(g_mu);
    DeviceSetup& su = g_setup[device];
    if (!su.addr || su.ctx != current_context()) {
        void* p = nullptr;
        cudaFuncAttributes fa;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return TM_ECUDA;
        if (cudaFuncGetAttributes(&fa, noalloc_init_kernel) != cudaSuccess) return TM_ECUDA;
        if (exhaustive_preload() != cudaSuccess) return TM_ECUDA;
        su.addr = p;
        su.ctx = current_context();   // read after the runtime has made its context current
    }
    *out = static_cast<unsigned char*>(su.addr);
    return TM_OK;
}

}  // namespace
}  // namespace tmgpu

extern "C" int tm_exhaustive_batch_noalloc(const tm_task* d_tasks, const int32_t* h_offsets,
                                           int G, const tm_device* d_devs, tm_stats* d_stats,
                                           int32_t* d_status, void* stream)
{
    using namespace tmgpu;
    if (!h_offsets || G < 0 || (G > 0 && (!d_tasks || !d_devs || !d_stats))) return TM_EINVAL;
    if (G > kMaxGroups) return TM_ECAPACITY;
    InitArgs a;
    a.G = G;
    Plan p;
    int rc = plan_decompose(h_offsets, G, kPdmax, 256u, a.gp, &p);
    if (rc != TM_OK) return rc;
    if (p.T > TM_NOALLOC_MAX_TASKS || p.total_subs > TM_NOALLOC_MAX_SUBSETS ||
        plan_carve(p, nullptr) > kScratchBytes)
        return TM_ECAPACITY;
    if (G == 0) return TM_OK;

    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) return TM_ECUDA;
    unsigned char* base = nullptr;
    if ((rc = scratch_address(device, &base)) != TM_OK) return rc;
    p.device = device;
    exhaustive_partition(p, device);
    plan_carve(p, base);

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    noalloc_init_kernel<<<1, 256, 0, s>>>(a, p.d_gp, p.d_acc);
    if (cudaGetLastError() != cudaSuccess) return TM_ECUDA;
    cudaError_t e = launch_exhaustive(p, d_tasks, d_devs, d_stats, d_status, s);
    return e == cudaSuccess ? TM_OK : TM_ECUDA;
}

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
// The array is a static __device__ object, so every GPU that loads the
// library holds it until the process exits.  Its size bounds the batch:
// at most TM_NOALLOC_MAX_GROUPS groups and TM_NOALLOC_MAX_TASKS tasks.
//
// Host code must not use the array's symbol as an address: on the host it
// names a stand-in object, not device memory.  The first call on each
// device, with that device current, asks the runtime for the array's device
// address (cudaGetSymbolAddress) and caches it; make that first call before
// starting any stream capture.
//
// All calls share the one array, and it keeps whatever the previous call
// left there; each call re-initialises the parts that must start from a
// known value (offsets, work list, reduction words) on its stream before
// the search.  Two calls whose work overlaps on the GPU race on the array:
// serialise them (one stream, or events).
#include <mutex>

#include "tm_internal.h"

namespace tmgpu {
namespace {

constexpr int kMaxGroups = TM_NOALLOC_MAX_GROUPS;
constexpr int kMaxTasks = TM_NOALLOC_MAX_TASKS;
constexpr int kLevels = 5;

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kOffOffsets = 0;
constexpr size_t kOffItemBase = kOffOffsets + align256((kMaxGroups + 1) * sizeof(int32_t));
constexpr size_t kOffInfo = kOffItemBase + align256((kMaxGroups + 1) * sizeof(uint32_t));
constexpr size_t kOffTbl = kOffInfo + align256(kMaxGroups * sizeof(GroupInfo));
constexpr size_t kOffAcc = kOffTbl + align256(kMaxTasks * sizeof(int4));
constexpr size_t kScratchBytes = kOffAcc + align256(3 * kMaxGroups * sizeof(unsigned long long));
static_assert(kScratchBytes <= 32768, "no-allocation scratch must stay modest");

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct InitArgs {
    int32_t offsets[kMaxGroups + 1];
    uint32_t item_base[kMaxGroups + 1];
    int G;
};

// Writes the batch layout into the scratch array and resets the reduction
// words, which the previous call may have left in any state.
__global__ void noalloc_init_kernel(InitArgs a, unsigned char* base)
{
    int32_t* offsets = reinterpret_cast<int32_t*>(base + kOffOffsets);
    uint32_t* item_base = reinterpret_cast<uint32_t*>(base + kOffItemBase);
    unsigned long long* acc = reinterpret_cast<unsigned long long*>(base + kOffAcc);
    for (int i = threadIdx.x; i <= a.G; i += blockDim.x) {
        offsets[i] = a.offsets[i];
        item_base[i] = a.item_base[i];
    }
    for (int i = threadIdx.x; i < 3 * a.G; i += blockDim.x)
        acc[i] = (i % 3 == 0) ? ~0ull : 0ull;
}

std::mutex g_mu;
void* g_addr[64] = {};  // device address of g_scratch, per device ordinal

int scratch_address(int device, unsigned char** out)
{
    if (device < 0 || device >= 64) return TM_EINVAL;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[device]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return TM_ECUDA;
        g_addr[device] = p;
    }
    *out = static_cast<unsigned char*>(g_addr[device]);
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
    if (h_offsets[0] != 0) return TM_EINVAL;
    InitArgs a;
    a.G = G;
    uint64_t total = 0;
    for (int g = 0; g <= G; ++g) a.offsets[g] = h_offsets[g];
    for (int g = 0; g < G; ++g) {
        int n = h_offsets[g + 1] - h_offsets[g];
        if (n < 1) return TM_EINVAL;
        if (n > TM_MAX_EXHAUSTIVE) return TM_ETOOBIG;
        a.item_base[g] = (uint32_t)total;
        if (n >= 5) total += factorial_u64(n) / factorial_u64(n < kLevels ? n : kLevels);
        if (total >= 0xFFFFFFFFull) return TM_ETOOBIG;
    }
    a.item_base[G] = (uint32_t)total;
    if (h_offsets[G] > kMaxTasks) return TM_ECAPACITY;
    if (G == 0) return TM_OK;

    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) return TM_ECUDA;
    unsigned char* base = nullptr;
    int rc = scratch_address(device, &base);
    if (rc != TM_OK) return rc;

    Plan p;
    p.device = device;
    p.G = G;
    p.T = h_offsets[G];
    p.levels = kLevels;
    p.total_items = (uint32_t)total;
    int resident = exhaustive_resident_threads(kLevels, device);
    if (resident <= 0) resident = 152 * 1024;
    uint64_t per = (total + resident - 1) / (uint64_t)resident;
    p.items_per_thread = (uint32_t)(per > 0 ? per : 1);
    p.threads = (uint32_t)((total + p.items_per_thread - 1) / p.items_per_thread);
    p.launches = exhaustive_launch_count(p) + 1;
    p.d_offsets = reinterpret_cast<int32_t*>(base + kOffOffsets);
    p.d_item_base = reinterpret_cast<uint32_t*>(base + kOffItemBase);
    p.d_info = reinterpret_cast<GroupInfo*>(base + kOffInfo);
    p.d_tbl = reinterpret_cast<int4*>(base + kOffTbl);
    p.d_acc = reinterpret_cast<unsigned long long*>(base + kOffAcc);

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    noalloc_init_kernel<<<1, 256, 0, s>>>(a, base);
    if (cudaGetLastError() != cudaSuccess) return TM_ECUDA;
    cudaError_t e = launch_exhaustive(p, d_tasks, d_devs, d_stats, d_status, s);
    return e == cudaSuccess ? TM_OK : TM_ECUDA;
}

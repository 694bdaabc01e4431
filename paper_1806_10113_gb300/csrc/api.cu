// api.cu -- the extern "C" entry points declared in include/tm.h: host-side
// input checks, the per-thread device buffers of the host-pointer calls,
// exhaustive-search plans, and the stream-ordered _dev launches.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <memory>
#include <mutex>
#include <vector>

#include "tm_internal.h"

using tmgpu::Plan;

struct tm_plan {
    Plan p;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t ev_node[2] = {nullptr, nullptr};   // timing records, if captured
};

namespace {

// ---- host-side validation (mirrors the per-group device checks) ----------

int check_tasks(const tm_task* t, int n)
{
    int64_t total = 0;
    for (int i = 0; i < n; ++i) {
        if (t[i].htd < 0 || t[i].k < 0 || t[i].dth < 0) return TM_ENEG;
        total += (int64_t)t[i].htd + t[i].k + t[i].dth;
    }
    return total > INT32_MAX ? TM_EOVERFLOW : TM_OK;
}

int check_batch(const tm_task* tasks, const int32_t* offsets, int G, const tm_device* devs,
                int nmax)
{
    if (G < 0 || !offsets || (G > 0 && (!tasks || !devs))) return TM_EINVAL;
    if (offsets[0] != 0) return TM_EINVAL;
    for (int g = 0; g < G; ++g) {
        int n = offsets[g + 1] - offsets[g];
        if (n < 1) return TM_EINVAL;
        if (n > nmax) return nmax == TM_MAX_EXHAUSTIVE ? TM_ETOOBIG : TM_EINVAL;
        if (devs[g].dma_engines != 1 && devs[g].dma_engines != 2) return TM_EINVAL;
        int rc = check_tasks(tasks + offsets[g], n);
        if (rc != TM_OK) return rc;
    }
    return TM_OK;
}

// Every time of the partial-overlap loop stays below the sum of kernels and
// of transfers stretched by den / num (rounded up).
int check_overlap(const tm_task* tasks, const int32_t* offsets, int G, int32_t num, int32_t den)
{
    if (!tmgpu::overlap_rate_ok(num, den)) return TM_EINVAL;
    for (int g = 0; g < G; ++g) {
        int64_t bound = 0;
        for (int i = offsets[g]; i < offsets[g + 1]; ++i)
            bound += tasks[i].k + ((int64_t)tasks[i].htd * den + num - 1) / num +
                     ((int64_t)tasks[i].dth * den + num - 1) / num;
        if (bound > INT32_MAX) return TM_EOVERFLOW;
    }
    return TM_OK;
}

int check_orders(const int32_t* orders, const int32_t* offsets, int G)
{
    if (G > 0 && !orders) return TM_EINVAL;
    for (int g = 0; g < G; ++g) {
        int n = offsets[g + 1] - offsets[g];
        uint32_t seen = 0;
        for (int i = 0; i < n; ++i) {
            int o = orders[offsets[g] + i];
            if (o < 0 || o >= n || ((seen >> o) & 1u)) return TM_EINVAL;
            seen |= 1u << o;
        }
    }
    return TM_OK;
}

// ---- device buffers owned by the library, one set per host thread --------

struct DevBuf {
    void* p = nullptr;
    size_t cap = 0;
    bool ensure(size_t bytes)
    {
        if (bytes <= cap) return true;
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
        size_t want = std::max<size_t>(bytes, 256);
        if (cudaMalloc(&p, want) != cudaSuccess) { p = nullptr; return false; }
        cap = want;
        return true;
    }
    template <class T> T* as() const { return static_cast<T*>(p); }
    void release() { if (p) cudaFree(p); p = nullptr; cap = 0; }
};

// Page-locked host staging, grown on demand (contents not kept).
// Page-locked host memory mapped into the device's address space: kernels
// read and write it in place through `d` (over NVLink-C2C on GB300).
struct PinBuf {
    void* p = nullptr;
    void* d = nullptr;
    size_t cap = 0;
    bool ensure(size_t bytes)
    {
        if (bytes <= cap) return true;
        release();
        const size_t want = std::max<size_t>(bytes, 4096);
        if (cudaHostAlloc(&p, want, cudaHostAllocMapped) != cudaSuccess) { p = nullptr; return false; }
        if (cudaHostGetDevicePointer(&d, p, 0) != cudaSuccess) { release(); return false; }
        cap = want;
        return true;
    }
    void release() { if (p) cudaFreeHost(p); p = nullptr; d = nullptr; cap = 0; }
};

struct Context {
    int device = -1;
    cudaStream_t stream = nullptr;
    DevBuf tasks, offsets, devs, orders, out, stats, status;
    PinBuf pin_in, pin_out;          // mapped inputs / outputs of the exhaustive host call
    tm_plan* plan = nullptr;
    std::vector<int32_t> plan_offsets;
    unsigned plan_epoch = 0;
    // the mapped blocks the plan's captured graph reads and writes
    const void* graph_in = nullptr;
    const void* graph_out = nullptr;
    void release()
    {
        if (plan) tm_plan_destroy(plan);
        plan = nullptr;
        plan_offsets.clear();
        for (DevBuf* b : {&tasks, &offsets, &devs, &orders, &out, &stats, &status})
            b->release();
        pin_in.release();
        pin_out.release();
        if (stream) cudaStreamDestroy(stream);
        stream = nullptr;
    }
    ~Context()
    {
        // At process exit the CUDA runtime may already be gone; only free
        // while it still answers.
        if (cudaGetDevice(&device) == cudaSuccess) release();
    }
};

thread_local std::unique_ptr<Context> t_ctx;

std::mutex g_tune_mu;
tm_tuning g_default_tuning{0, 0, 0, 0, 0, 0};
unsigned g_tuning_epoch = 0;   // bumped on every change; cached plans compare it

int context(Context** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TM_ECUDA;
    if (!t_ctx || t_ctx->device != dev) {
        if (t_ctx) t_ctx->release();
        t_ctx.reset(new Context());
        t_ctx->device = dev;
        if (cudaStreamCreateWithFlags(&t_ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
            t_ctx.reset();
            return TM_ECUDA;
        }
    }
    *out = t_ctx.get();
    return TM_OK;
}

#define TM_CUDA(call)                                \
    do {                                             \
        if ((call) != cudaSuccess) return TM_ECUDA;  \
    } while (0)

int copy_in(DevBuf& b, const void* src, size_t bytes, cudaStream_t s)
{
    if (!b.ensure(bytes)) return TM_ENOMEM;
    if (bytes) TM_CUDA(cudaMemcpyAsync(b.p, src, bytes, cudaMemcpyHostToDevice, s));
    return TM_OK;
}

int first_error(const int32_t* status, int G)
{
    for (int g = 0; g < G; ++g)
        if (status[g] != 0) return status[g];
    return TM_OK;
}

// ---- plans -----------------------------------------------------------------

bool tuning_invalid(const tm_tuning& t)
{
    return (t.pdmax != 0 && (t.pdmax < 3 || t.pdmax > 5)) || t.fuse_finalize < 0 ||
           t.fuse_finalize > 2 || t.blocks_per_sm < 0 || t.item_cost < 0 ||
           t.item_cost > (1 << 20) || t.chunks_per_thread < 0 || t.chunks_per_thread > 64 ||
           (t.fuse_finalize == 1 && t.chunks_per_thread > 1) || t.unroll < 0 || t.unroll > 8;
}

void free_plan(Plan& p)
{
    if (p.d_gp) cudaFree(p.d_gp);   // the start of the plan's single block
    p.d_gp = nullptr;
    p.d_info = nullptr;
    p.d_tbl = nullptr;
    p.d_sub = nullptr;
    p.d_acc = nullptr;
    p.d_target = nullptr;
    p.d_done = nullptr;
}

// Host-side table of the fused finalize: per group the number of
// enumeration threads whose item range touches it (thread t covers the items
// whose cost range starts in its static_range).
void fused_tables(const Plan& p, const std::vector<tmgpu::GroupPlan>& gp,
                  std::vector<uint32_t>& target)
{
    target.assign(std::max(p.G, 1), 0);
    const uint64_t total = gp[p.G].cost_base;
    int g = 0;
    for (uint64_t t = 0; t < p.threads; ++t) {
        uint64_t x0, x1;
        tmgpu::static_range(t, p.leaves_per_thread, p.split_c, p.split_warps, p.split_hi,
                            p.split_klo, &x0, &x1);
        if (x0 >= total) break;
        const uint32_t i0 = tmgpu::plan_first_item(gp.data(), p.G, p.pdmax, p.item_cost, x0);
        const uint32_t i1 = tmgpu::plan_first_item(gp.data(), p.G, p.pdmax, p.item_cost,
                                                   std::min(x1, total));
        if (i0 >= i1) continue;
        while (gp[g + 1].item_base <= i0) ++g;        // the group holding item i0
        for (int h = g; h < p.G && gp[h].item_base < i1; ++h)
            if (gp[h + 1].item_base > gp[h].item_base) ++target[h];
    }
}

int build_plan(const int32_t* h_offsets, int G, const tm_tuning& tune, Plan& p)
{
    const int pdmax = tune.pdmax == 0 ? 4 : tune.pdmax;
    const bool fused = tune.fuse_finalize == 1;
    const uint32_t item_cost = tune.item_cost == 0 ? 4096u : (uint32_t)tune.item_cost;
    if (tuning_invalid(tune)) return TM_EINVAL;
    if (!h_offsets || G < 0) return TM_EINVAL;
    std::vector<tmgpu::GroupPlan> gp((size_t)G + 1);
    int rc = tmgpu::plan_decompose(h_offsets, G, pdmax, item_cost, gp.data(), &p);
    if (rc != TM_OK) return rc;
    TM_CUDA(cudaGetDevice(&p.device));
    p.chunks_per_thread = tune.chunks_per_thread == 0 ? 1 : tune.chunks_per_thread;
    p.unroll = tune.unroll == 0 ? 2 : tune.unroll;
    tmgpu::exhaustive_partition(p, p.device, tune.blocks_per_sm);
    std::vector<uint32_t> target;
    fused_tables(p, gp, target);
    const size_t main_bytes = tmgpu::plan_carve(p, nullptr);
    const size_t fused_bytes = tmgpu::plan_carve_fused(p, nullptr);
    void* base = nullptr;
    if (cudaMalloc(&base, main_bytes + fused_bytes) != cudaSuccess) return TM_ENOMEM;
    tmgpu::plan_carve(p, static_cast<unsigned char*>(base));
    tmgpu::plan_carve_fused(p, static_cast<unsigned char*>(base) + main_bytes);
    if (!fused) p.d_target = p.d_done = nullptr;   // separate finalize kernel
    p.launches = tmgpu::exhaustive_launch_count(p);
    std::vector<unsigned long long> acc(tmgpu::kAccStride * (size_t)std::max(G, 1), 0ull);
    for (size_t g = 0; g * tmgpu::kAccStride < acc.size(); ++g) acc[g * tmgpu::kAccStride] = ~0ull;
    bool ok = cudaMemcpy(p.d_gp, gp.data(), gp.size() * sizeof(tmgpu::GroupPlan),
                         cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemcpy(p.d_acc, acc.data(), acc.size() * sizeof(unsigned long long),
                         cudaMemcpyHostToDevice) == cudaSuccess &&
              (!fused ||
               (cudaMemcpy(p.d_target, target.data(), target.size() * sizeof(uint32_t),
                           cudaMemcpyHostToDevice) == cudaSuccess &&
                cudaMemset(p.d_done, 0, tmgpu::kDoneStride * target.size() * sizeof(uint32_t)) ==
                    cudaSuccess));
    ok = ok && cudaMemset(p.d_next, 0, sizeof(uint32_t)) == cudaSuccess;
    if (!ok) { free_plan(p); return TM_ECUDA; }
    return TM_OK;
}

}  // namespace

extern "C" {

const char* tm_strerror(int code)
{
    switch (code) {
    case TM_OK: return "ok";
    case TM_EINVAL: return "invalid argument";
    case TM_ENEG: return "negative duration";
    case TM_EOVERFLOW: return "group durations sum above INT32_MAX";
    case TM_ETOOBIG: return "too many tasks for exhaustive search (n > 12)";
    case TM_ECUDA: return "CUDA runtime error";
    case TM_ETIMEOUT: return "device-side wait timed out";
    case TM_ENOMEM: return "out of memory";
    case TM_ECAPACITY: return "batch exceeds the no-allocation entry point's fixed capacity";
    default: return "unknown tm status";
    }
}

const char* tm_version(void) { return "tm 0.1 sm_103a"; }

int tm_plan_create_tuned(const int32_t* h_offsets, int G, const tm_tuning* tuning,
                         tm_plan** plan_out)
{
    if (!plan_out) return TM_EINVAL;
    tm_tuning tune{0, 0, 0, 0, 0, 0};
    if (tuning) tune = *tuning;
    std::unique_ptr<tm_plan> plan(new (std::nothrow) tm_plan());
    if (!plan) return TM_ENOMEM;
    int rc = build_plan(h_offsets, G, tune, plan->p);
    if (rc != TM_OK) return rc;
    *plan_out = plan.release();
    return TM_OK;
}

int tm_plan_create(const int32_t* h_offsets, int G, tm_plan** plan_out)
{
    tm_tuning tune;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        tune = g_default_tuning;
    }
    return tm_plan_create_tuned(h_offsets, G, &tune, plan_out);
}

int tm_set_default_tuning(const tm_tuning* tuning)
{
    tm_tuning t{0, 0, 0, 0, 0, 0};
    if (tuning) t = *tuning;
    if (tuning_invalid(t)) return TM_EINVAL;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_default_tuning = t;
    ++g_tuning_epoch;
    return TM_OK;
}

void tm_plan_destroy(tm_plan* plan)
{
    if (!plan) return;
    if (plan->exec) cudaGraphExecDestroy(plan->exec);
    if (plan->graph) cudaGraphDestroy(plan->graph);
    free_plan(plan->p);
    delete plan;
}

int tm_plan_capture(tm_plan* plan, const tm_task* d_tasks, const tm_device* d_devs,
                    tm_stats* d_stats, int32_t* d_orders_out, int32_t* d_makespans_out,
                    int32_t* d_status)
{
    if (!plan) return TM_EINVAL;
    if (plan->p.G > 0 && (!d_tasks || !d_devs || !d_stats || !d_orders_out)) return TM_EINVAL;
    cudaStream_t s = nullptr;
    TM_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t le = tmgpu::launch_exhaustive(plan->p, d_tasks, d_devs, d_stats, d_status, s,
                                                  d_orders_out, d_makespans_out);
        e = cudaStreamEndCapture(s, &graph);
        if (e == cudaSuccess) e = le;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    cudaStreamDestroy(s);
    if (e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return TM_ECUDA;
    }
    if (plan->exec) cudaGraphExecDestroy(plan->exec);
    if (plan->graph) cudaGraphDestroy(plan->graph);
    plan->graph = graph;
    plan->exec = exec;
    plan->ev_node[0] = plan->ev_node[1] = nullptr;
    size_t count = 0;
    if (plan->p.ev_before && cudaGraphGetNodes(graph, nullptr, &count) == cudaSuccess) {
        std::vector<cudaGraphNode_t> nodes(count);
        if (cudaGraphGetNodes(graph, nodes.data(), &count) == cudaSuccess) {
            for (cudaGraphNode_t nd : nodes) {
                cudaGraphNodeType type;
                cudaEvent_t ev = nullptr;
                if (cudaGraphNodeGetType(nd, &type) != cudaSuccess ||
                    type != cudaGraphNodeTypeEventRecord ||
                    cudaGraphEventRecordNodeGetEvent(nd, &ev) != cudaSuccess)
                    continue;
                if (ev == plan->p.ev_before) plan->ev_node[0] = nd;
                if (ev == plan->p.ev_after) plan->ev_node[1] = nd;
            }
        }
    }
    return TM_OK;
}

int tm_plan_graph_set_timing(tm_plan* plan, void* event_before, void* event_after)
{
    if (!plan || !plan->exec || !plan->ev_node[0] || !plan->ev_node[1] || !event_before ||
        !event_after)
        return TM_EINVAL;
    if (cudaGraphExecEventRecordNodeSetEvent(plan->exec, plan->ev_node[0],
                                             (cudaEvent_t)event_before) != cudaSuccess ||
        cudaGraphExecEventRecordNodeSetEvent(plan->exec, plan->ev_node[1],
                                             (cudaEvent_t)event_after) != cudaSuccess)
        return TM_ECUDA;
    return TM_OK;
}

int tm_plan_graph_launch(const tm_plan* plan, void* stream)
{
    if (!plan || !plan->exec) return TM_EINVAL;
    return cudaGraphLaunch(plan->exec, (cudaStream_t)stream) == cudaSuccess ? TM_OK : TM_ECUDA;
}

int tm_plan_launches(const tm_plan* plan) { return plan ? plan->p.launches : 0; }

int tm_plan_set_timing(tm_plan* plan, void* event_before, void* event_after)
{
    if (!plan || (!event_before) != (!event_after)) return TM_EINVAL;
    plan->p.ev_before = (cudaEvent_t)event_before;
    plan->p.ev_after = (cudaEvent_t)event_after;
    return TM_OK;
}

int tm_plan_walk_counts(const tm_plan* plan, unsigned long long* prefixes,
                        unsigned long long* full)
{
    if (!plan || !prefixes || !full) return TM_EINVAL;
    *prefixes = plan->p.total_prefixes;
    *full = plan->p.total_prefixes;
    if (plan->p.unroll < 5 || !plan->p.d_full || plan->p.total_items == 0) return TM_OK;
    unsigned long long v = 0;
    if (cudaMemcpy(&v, plan->p.d_full, sizeof v, cudaMemcpyDeviceToHost) != cudaSuccess)
        return TM_ECUDA;
    *full = v;
    return TM_OK;
}

int tm_exhaustive_batch_dev(const tm_plan* plan, const tm_task* d_tasks, const tm_device* d_devs,
                            tm_stats* d_stats, int32_t* d_status, void* stream)
{
    if (!plan) return TM_EINVAL;
    if (plan->p.G > 0 && (!d_tasks || !d_devs || !d_stats)) return TM_EINVAL;
    cudaError_t e = tmgpu::launch_exhaustive(plan->p, d_tasks, d_devs, d_stats, d_status,
                                          (cudaStream_t)stream);
    return e == cudaSuccess ? TM_OK : TM_ECUDA;
}

int tm_schedule_batch_dev(const tm_plan* plan, const tm_task* d_tasks, const tm_device* d_devs,
                          tm_stats* d_stats, int32_t* d_orders_out, int32_t* d_makespans_out,
                          int32_t* d_status, void* stream)
{
    if (!plan) return TM_EINVAL;
    if (plan->p.G > 0 && (!d_tasks || !d_devs || !d_stats || !d_orders_out)) return TM_EINVAL;
    cudaError_t e = tmgpu::launch_exhaustive(plan->p, d_tasks, d_devs, d_stats, d_status,
                                             (cudaStream_t)stream, d_orders_out, d_makespans_out);
    return e == cudaSuccess ? TM_OK : TM_ECUDA;
}

int tm_predict_batch_dev(const tm_task* d_tasks, const int32_t* d_offsets, int G,
                         const int32_t* d_orders, const tm_device* d_devs, int32_t* d_makespans,
                         int32_t* d_status, void* stream)
{
    if (G < 0) return TM_EINVAL;
    if (G > 0 && (!d_tasks || !d_offsets || !d_orders || !d_devs || !d_makespans))
        return TM_EINVAL;
    cudaError_t e = tmgpu::launch_predict(d_tasks, d_offsets, G, d_orders, d_devs, d_makespans,
                                       d_status, (cudaStream_t)stream);
    return e == cudaSuccess ? TM_OK : TM_ECUDA;
}

int tm_heuristic_batch_dev(const tm_task* d_tasks, const int32_t* d_offsets, int G,
                           const tm_device* d_devs, int32_t* d_orders_out,
                           int32_t* d_makespans_out, int32_t* d_status, void* stream)
{
    if (G < 0) return TM_EINVAL;
    if (G > 0 && (!d_tasks || !d_offsets || !d_devs || !d_orders_out)) return TM_EINVAL;
    cudaError_t e = tmgpu::launch_heuristic(d_tasks, d_offsets, G, d_devs, d_orders_out,
                                         d_makespans_out, d_status, (cudaStream_t)stream);
    return e == cudaSuccess ? TM_OK : TM_ECUDA;
}

int tm_predict_batch(const tm_task* tasks, const int32_t* offsets, int G, const int32_t* orders,
                     const tm_device* devs, int32_t* makespans)
{
    int rc = check_batch(tasks, offsets, G, devs, TM_MAX_TASKS);
    if (rc == TM_OK) rc = check_orders(orders, offsets, G);
    if (rc != TM_OK) return rc;
    if (G == 0) return TM_OK;
    if (!makespans) return TM_EINVAL;
    Context* c = nullptr;
    if ((rc = context(&c)) != TM_OK) return rc;
    int T = offsets[G];
    cudaStream_t s = c->stream;
    if ((rc = copy_in(c->tasks, tasks, T * sizeof(tm_task), s)) != TM_OK) return rc;
    if ((rc = copy_in(c->offsets, offsets, (G + 1) * sizeof(int32_t), s)) != TM_OK) return rc;
    if ((rc = copy_in(c->orders, orders, T * sizeof(int32_t), s)) != TM_OK) return rc;
    if ((rc = copy_in(c->devs, devs, G * sizeof(tm_device), s)) != TM_OK) return rc;
    if (!c->out.ensure(G * sizeof(int32_t)) || !c->status.ensure(G * sizeof(int32_t)))
        return TM_ENOMEM;
    TM_CUDA(tmgpu::launch_predict(c->tasks.as<tm_task>(), c->offsets.as<int32_t>(), G,
                               c->orders.as<int32_t>(), c->devs.as<tm_device>(),
                               c->out.as<int32_t>(), c->status.as<int32_t>(), s));
    std::vector<int32_t> out(G), status(G);
    TM_CUDA(cudaMemcpyAsync(out.data(), c->out.p, G * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    TM_CUDA(cudaMemcpyAsync(status.data(), c->status.p, G * sizeof(int32_t),
                            cudaMemcpyDeviceToHost, s));
    TM_CUDA(cudaStreamSynchronize(s));
    if ((rc = first_error(status.data(), G)) != TM_OK) return rc;
    std::memcpy(makespans, out.data(), G * sizeof(int32_t));
    return TM_OK;
}

int tm_predict(const tm_task* tasks, int n, const int32_t* order, const tm_device* dev,
               int32_t* makespan)
{
    if (n < 1 || n > TM_MAX_TASKS) return TM_EINVAL;
    int32_t offsets[2] = {0, n};
    return tm_predict_batch(tasks, offsets, 1, order, dev, makespan);
}

}  // extern "C"

namespace {

// Host-pointer exhaustive search, with the heuristic too when orders_out is
// given.  The plan is cached per thread for repeated group sizes.
int exhaustive_host(const tm_task* tasks, const int32_t* offsets, int G, const tm_device* devs,
                    tm_stats* stats, int32_t* orders_out, int32_t* makespans_out)
{
    int rc = check_batch(tasks, offsets, G, devs, TM_MAX_EXHAUSTIVE);
    if (rc != TM_OK) return rc;
    if (G == 0) return TM_OK;
    if (!stats) return TM_EINVAL;
    Context* c = nullptr;
    if ((rc = context(&c)) != TM_OK) return rc;
    std::vector<int32_t> offs(offsets, offsets + G + 1);
    unsigned epoch;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        epoch = g_tuning_epoch;
    }
    if (!c->plan || c->plan_offsets != offs || c->plan_epoch != epoch) {
        if (c->plan) tm_plan_destroy(c->plan);
        c->plan = nullptr;
        c->plan_offsets.clear();
        if ((rc = tm_plan_create(offsets, G, &c->plan)) != TM_OK) return rc;
        c->plan_offsets = offs;
        c->plan_epoch = epoch;
        c->graph_in = c->graph_out = nullptr;
    }
    const int T = offsets[G];
    cudaStream_t s = c->stream;
    // Inputs (tasks, device models) and outputs (stats, status, makespans,
    // orders) live in one mapped page-locked block each: the prep kernel
    // reads the inputs in place and the finalize kernel writes the results
    // in place, so the call issues no copy at all.
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t i_devs = al((size_t)T * sizeof(tm_task)), in_bytes = i_devs + (size_t)G * 4;
    const size_t o_status = al((size_t)G * sizeof(tm_stats)), o_ms = o_status + al((size_t)G * 4),
                 o_orders = o_ms + al((size_t)G * 4), out_bytes = o_orders + (size_t)T * 4;
    if (!c->pin_in.ensure(in_bytes) || !c->pin_out.ensure(out_bytes)) return TM_ENOMEM;
    unsigned char* hin = static_cast<unsigned char*>(c->pin_in.p);
    std::memcpy(hin, tasks, (size_t)T * sizeof(tm_task));
    std::memcpy(hin + i_devs, devs, (size_t)G * 4);
    unsigned char* din = static_cast<unsigned char*>(c->pin_in.d);
    unsigned char* dout = static_cast<unsigned char*>(c->pin_out.d);
    const tm_task* d_tasks = reinterpret_cast<const tm_task*>(din);
    const tm_device* d_devs = reinterpret_cast<const tm_device*>(din + i_devs);
    tm_stats* d_stats = reinterpret_cast<tm_stats*>(dout);
    int32_t* d_status = reinterpret_cast<int32_t*>(dout + o_status);
    int32_t* d_ms = reinterpret_cast<int32_t*>(dout + o_ms);
    int32_t* d_orders = reinterpret_cast<int32_t*>(dout + o_orders);
    if (orders_out) {
        // the whole pass as one CUDA graph, captured once per plan and blocks
        if (c->graph_in != din || c->graph_out != dout) {
            if ((rc = tm_plan_capture(c->plan, d_tasks, d_devs, d_stats, d_orders, d_ms,
                                      d_status)) != TM_OK)
                return rc;
            c->graph_in = din;
            c->graph_out = dout;
        }
        rc = tm_plan_graph_launch(c->plan, s);
    } else {
        rc = tm_exhaustive_batch_dev(c->plan, d_tasks, d_devs, d_stats, d_status, s);
    }
    if (rc != TM_OK) return rc;
    TM_CUDA(cudaStreamSynchronize(s));
    const unsigned char* hout = static_cast<const unsigned char*>(c->pin_out.p);
    if ((rc = first_error(reinterpret_cast<const int32_t*>(hout + o_status), G)) != TM_OK) return rc;
    std::memcpy(stats, hout, (size_t)G * sizeof(tm_stats));
    if (orders_out) {
        std::memcpy(orders_out, hout + o_orders, (size_t)T * sizeof(int32_t));
        if (makespans_out) std::memcpy(makespans_out, hout + o_ms, (size_t)G * sizeof(int32_t));
    }
    return TM_OK;
}

}  // namespace

extern "C" {

int tm_exhaustive_batch(const tm_task* tasks, const int32_t* offsets, int G,
                        const tm_device* devs, tm_stats* stats)
{
    return exhaustive_host(tasks, offsets, G, devs, stats, nullptr, nullptr);
}

int tm_schedule_batch(const tm_task* tasks, const int32_t* offsets, int G, const tm_device* devs,
                      tm_stats* stats, int32_t* orders_out, int32_t* makespans_out)
{
    if (G > 0 && !orders_out) return TM_EINVAL;
    return exhaustive_host(tasks, offsets, G, devs, stats, orders_out, makespans_out);
}

int tm_exhaustive(const tm_task* tasks, int n, const tm_device* dev, tm_stats* stats,
                  double* mean)
{
    if (n < 1) return TM_EINVAL;
    if (n > TM_MAX_EXHAUSTIVE) return TM_ETOOBIG;
    int32_t offsets[2] = {0, n};
    int rc = tm_exhaustive_batch(tasks, offsets, 1, dev, stats);
    if (rc == TM_OK && mean) *mean = stats->mean;
    return rc;
}

int tm_heuristic_batch(const tm_task* tasks, const int32_t* offsets, int G,
                       const tm_device* devs, int32_t* orders_out, int32_t* makespans_out)
{
    int rc = check_batch(tasks, offsets, G, devs, TM_MAX_TASKS);
    if (rc != TM_OK) return rc;
    if (G == 0) return TM_OK;
    if (!orders_out) return TM_EINVAL;
    Context* c = nullptr;
    if ((rc = context(&c)) != TM_OK) return rc;
    int T = offsets[G];
    cudaStream_t s = c->stream;
    if ((rc = copy_in(c->tasks, tasks, T * sizeof(tm_task), s)) != TM_OK) return rc;
    if ((rc = copy_in(c->offsets, offsets, (G + 1) * sizeof(int32_t), s)) != TM_OK) return rc;
    if ((rc = copy_in(c->devs, devs, G * sizeof(tm_device), s)) != TM_OK) return rc;
    if (!c->orders.ensure(T * sizeof(int32_t)) || !c->out.ensure(G * sizeof(int32_t)) ||
        !c->status.ensure(G * sizeof(int32_t)))
        return TM_ENOMEM;
    TM_CUDA(tmgpu::launch_heuristic(c->tasks.as<tm_task>(), c->offsets.as<int32_t>(), G,
                                 c->devs.as<tm_device>(), c->orders.as<int32_t>(),
                                 c->out.as<int32_t>(), c->status.as<int32_t>(), s));
    std::vector<int32_t> orders(T), out(G), status(G);
    TM_CUDA(cudaMemcpyAsync(orders.data(), c->orders.p, T * sizeof(int32_t),
                            cudaMemcpyDeviceToHost, s));
    TM_CUDA(cudaMemcpyAsync(out.data(), c->out.p, G * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    TM_CUDA(cudaMemcpyAsync(status.data(), c->status.p, G * sizeof(int32_t),
                            cudaMemcpyDeviceToHost, s));
    TM_CUDA(cudaStreamSynchronize(s));
    if ((rc = first_error(status.data(), G)) != TM_OK) return rc;
    std::memcpy(orders_out, orders.data(), T * sizeof(int32_t));
    if (makespans_out) std::memcpy(makespans_out, out.data(), G * sizeof(int32_t));
    return TM_OK;
}

int tm_heuristic(const tm_task* tasks, int n, const tm_device* dev, int32_t* order_out,
                 int32_t* makespan_out)
{
    if (n < 1 || n > TM_MAX_TASKS) return TM_EINVAL;
    int32_t offsets[2] = {0, n};
    return tm_heuristic_batch(tasks, offsets, 1, dev, order_out, makespan_out);
}

// ---- partial-overlap variant ---------------------------------------------------

int tm_predict_overlap_batch(const tm_task* tasks, const int32_t* offsets, int G,
                             const int32_t* orders, const tm_device* devs, int32_t rate_num,
                             int32_t rate_den, int32_t* makespans)
{
    int rc = check_batch(tasks, offsets, G, devs, TM_MAX_TASKS);
    if (rc == TM_OK) rc = check_orders(orders, offsets, G);
    if (rc == TM_OK) rc = check_overlap(tasks, offsets, G, rate_num, rate_den);
    if (rc != TM_OK) return rc;
    if (G == 0) return TM_OK;
    if (!makespans) return TM_EINVAL;
    Context* c = nullptr;
    if ((rc = context(&c)) != TM_OK) return rc;
    const int T = offsets[G];
    cudaStream_t s = c->stream;
    if ((rc = copy_in(c->tasks, tasks, T * sizeof(tm_task), s)) != TM_OK) return rc;
    if ((rc = copy_in(c->offsets, offsets, (G + 1) * sizeof(int32_t), s)) != TM_OK) return rc;
    if ((rc = copy_in(c->orders, orders, T * sizeof(int32_t), s)) != TM_OK) return rc;
    if ((rc = copy_in(c->devs, devs, G * sizeof(tm_device), s)) != TM_OK) return rc;
    if (!c->out.ensure(G * sizeof(int32_t)) || !c->status.ensure(G * sizeof(int32_t)))
        return TM_ENOMEM;
    TM_CUDA(tmgpu::launch_overlap_predict(c->tasks.as<tm_task>(), c->offsets.as<int32_t>(), G,
                                          c->orders.as<int32_t>(), c->devs.as<tm_device>(),
                                          rate_num, rate_den, c->out.as<int32_t>(),
                                          c->status.as<int32_t>(), s));
    std::vector<int32_t> out(G), status(G);
    TM_CUDA(cudaMemcpyAsync(out.data(), c->out.p, G * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    TM_CUDA(cudaMemcpyAsync(status.data(), c->status.p, G * sizeof(int32_t),
                            cudaMemcpyDeviceToHost, s));
    TM_CUDA(cudaStreamSynchronize(s));
    if ((rc = first_error(status.data(), G)) != TM_OK) return rc;
    std::memcpy(makespans, out.data(), G * sizeof(int32_t));
    return TM_OK;
}

int tm_predict_overlap(const tm_task* tasks, int n, const int32_t* order, const tm_device* dev,
                       int32_t rate_num, int32_t rate_den, int32_t* makespan)
{
    if (n < 1 || n > TM_MAX_TASKS) return TM_EINVAL;
    int32_t offsets[2] = {0, n};
    return tm_predict_overlap_batch(tasks, offsets, 1, order, dev, rate_num, rate_den, makespan);
}

int tm_predict_overlap_batch_dev(const tm_task* d_tasks, const int32_t* d_offsets, int G,
                                 const int32_t* d_orders, const tm_device* d_devs,
                                 int32_t rate_num, int32_t rate_den, int32_t* d_makespans,
                                 int32_t* d_status, void* stream)
{
    if (G < 0 || !tmgpu::overlap_rate_ok(rate_num, rate_den)) return TM_EINVAL;
    if (G > 0 && (!d_tasks || !d_offsets || !d_orders || !d_devs || !d_makespans)) return TM_EINVAL;
    cudaError_t e = tmgpu::launch_overlap_predict(d_tasks, d_offsets, G, d_orders, d_devs, rate_num,
                                                  rate_den, d_makespans, d_status,
                                                  (cudaStream_t)stream);
    return e == cudaSuccess ? TM_OK : TM_ECUDA;
}

int tm_exhaustive_overlap_batch_dev(const tm_task* d_tasks, const int32_t* d_offsets,
                                    const int32_t* h_offsets, int G, const tm_device* d_devs,
                                    int32_t rate_num, int32_t rate_den, tm_stats* d_stats,
                                    int32_t* d_status, void* stream)
{
    if (G < 0 || !tmgpu::overlap_rate_ok(rate_num, rate_den)) return TM_EINVAL;
    if (G == 0) return TM_OK;
    if (!d_tasks || !d_offsets || !h_offsets || !d_devs || !d_stats) return TM_EINVAL;
    if (h_offsets[0] != 0) return TM_EINVAL;
    for (int g = 0; g < G; ++g) {
        const int n = h_offsets[g + 1] - h_offsets[g];
        if (n < 1) return TM_EINVAL;
        if (n > TM_MAX_EXHAUSTIVE) return TM_ETOOBIG;
    }
    return tmgpu::overlap_exhaustive(d_tasks, d_offsets, h_offsets, G, d_devs, rate_num, rate_den,
                                     d_stats, d_status, (cudaStream_t)stream);
}

int tm_exhaustive_overlap_batch(const tm_task* tasks, const int32_t* offsets, int G,
                                const tm_device* devs, int32_t rate_num, int32_t rate_den,
                                tm_stats* stats)
{
    int rc = check_batch(tasks, offsets, G, devs, TM_MAX_EXHAUSTIVE);
    if (rc == TM_OK) rc = check_overlap(tasks, offsets, G, rate_num, rate_den);
    if (rc != TM_OK) return rc;
    if (G == 0) return TM_OK;
    if (!stats) return TM_EINVAL;
    Context* c = nullptr;
    if ((rc = context(&c)) != TM_OK) return rc;
    const int T = offsets[G];
    cudaStream_t s = c->stream;
    if ((rc = copy_in(c->tasks, tasks, T * sizeof(tm_task), s)) != TM_OK) return rc;
    if ((rc = copy_in(c->offsets, offsets, (G + 1) * sizeof(int32_t), s)) != TM_OK) return rc;
    if ((rc = copy_in(c->devs, devs, G * sizeof(tm_device), s)) != TM_OK) return rc;
    if (!c->stats.ensure(G * sizeof(tm_stats)) || !c->status.ensure(G * sizeof(int32_t)))
        return TM_ENOMEM;
    rc = tmgpu::overlap_exhaustive(c->tasks.as<tm_task>(), c->offsets.as<int32_t>(), offsets, G,
                                   c->devs.as<tm_device>(), rate_num, rate_den,
                                   c->stats.as<tm_stats>(), c->status.as<int32_t>(), s);
    if (rc != TM_OK) return rc;
    std::vector<tm_stats> out(G);
    std::vector<int32_t> status(G);
    TM_CUDA(cudaMemcpyAsync(out.data(), c->stats.p, G * sizeof(tm_stats), cudaMemcpyDeviceToHost, s));
    TM_CUDA(cudaMemcpyAsync(status.data(), c->status.p, G * sizeof(int32_t),
                            cudaMemcpyDeviceToHost, s));
    TM_CUDA(cudaStreamSynchronize(s));
    if ((rc = first_error(status.data(), G)) != TM_OK) return rc;
    std::memcpy(stats, out.data(), G * sizeof(tm_stats));
    return TM_OK;
}

}  // extern "C"

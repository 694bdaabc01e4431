// api.cu -- the extern "C" entry points declared in include/tm.h: host-side
// input checks, the per-thread device buffers of the host-pointer calls,
// exhaustive-search plans, and the stream-ordered _dev launches.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <memory>
#include <vector>

#include "tm_internal.h"

using tmgpu::Plan;

struct tm_plan {
    Plan p;
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

struct Context {
    int device = -1;
    cudaStream_t stream = nullptr;
    DevBuf tasks, offsets, devs, orders, out, stats, status;
    tm_plan* plan = nullptr;
    std::vector<int32_t> plan_offsets;
    void release()
    {
        if (plan) tm_plan_destroy(plan);
        plan = nullptr;
        plan_offsets.clear();
        for (DevBuf* b : {&tasks, &offsets, &devs, &orders, &out, &stats, &status}) b->release();
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

void free_plan(Plan& p)
{
    if (p.d_gp) cudaFree(p.d_gp);   // the start of the plan's single block
    p.d_gp = nullptr;
    p.d_info = nullptr;
    p.d_tbl = nullptr;
    p.d_sub = nullptr;
    p.d_acc = nullptr;
}

int build_plan(const int32_t* h_offsets, int G, int pdmax, Plan& p)
{
    if (!h_offsets || G < 0) return TM_EINVAL;
    std::vector<tmgpu::GroupPlan> gp((size_t)G + 1);
    int rc = tmgpu::plan_decompose(h_offsets, G, pdmax, gp.data(), &p);
    if (rc != TM_OK) return rc;
    TM_CUDA(cudaGetDevice(&p.device));
    tmgpu::exhaustive_partition(p, p.device);
    size_t bytes = tmgpu::plan_carve(p, nullptr);
    void* base = nullptr;
    if (cudaMalloc(&base, bytes) != cudaSuccess) return TM_ENOMEM;
    tmgpu::plan_carve(p, static_cast<unsigned char*>(base));
    std::vector<unsigned long long> acc(3 * (size_t)std::max(G, 1));
    for (size_t g = 0; 3 * g < acc.size(); ++g) acc[3 * g] = ~0ull;
    bool ok = cudaMemcpy(p.d_gp, gp.data(), gp.size() * sizeof(tmgpu::GroupPlan),
                         cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemcpy(p.d_acc, acc.data(), acc.size() * sizeof(unsigned long long),
                         cudaMemcpyHostToDevice) == cudaSuccess;
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

int tm_plan_create(const int32_t* h_offsets, int G, tm_plan** plan_out)
{
    if (!plan_out) return TM_EINVAL;
    std::unique_ptr<tm_plan> plan(new (std::nothrow) tm_plan());
    if (!plan) return TM_ENOMEM;
    int rc = build_plan(h_offsets, G, 4, plan->p);
    if (rc != TM_OK) return rc;
    *plan_out = plan.release();
    return TM_OK;
}

void tm_plan_destroy(tm_plan* plan)
{
    if (!plan) return;
    free_plan(plan->p);
    delete plan;
}

int tm_plan_launches(const tm_plan* plan) { return plan ? plan->p.launches : 0; }

int tm_plan_set_timing(tm_plan* plan, void* event_before, void* event_after)
{
    if (!plan || (!event_before) != (!event_after)) return TM_EINVAL;
    plan->p.ev_before = (cudaEvent_t)event_before;
    plan->p.ev_after = (cudaEvent_t)event_after;
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

int tm_exhaustive_batch(const tm_task* tasks, const int32_t* offsets, int G,
                        const tm_device* devs, tm_stats* stats)
{
    int rc = check_batch(tasks, offsets, G, devs, TM_MAX_EXHAUSTIVE);
    if (rc != TM_OK) return rc;
    if (G == 0) return TM_OK;
    if (!stats) return TM_EINVAL;
    Context* c = nullptr;
    if ((rc = context(&c)) != TM_OK) return rc;
    std::vector<int32_t> offs(offsets, offsets + G + 1);
    if (!c->plan || c->plan_offsets != offs) {
        if (c->plan) tm_plan_destroy(c->plan);
        c->plan = nullptr;
        c->plan_offsets.clear();
        if ((rc = tm_plan_create(offsets, G, &c->plan)) != TM_OK) return rc;
        c->plan_offsets = offs;
    }
    int T = offsets[G];
    cudaStream_t s = c->stream;
    if ((rc = copy_in(c->tasks, tasks, T * sizeof(tm_task), s)) != TM_OK) return rc;
    if ((rc = copy_in(c->devs, devs, G * sizeof(tm_device), s)) != TM_OK) return rc;
    if (!c->stats.ensure(G * sizeof(tm_stats)) || !c->status.ensure(G * sizeof(int32_t)))
        return TM_ENOMEM;
    rc = tm_exhaustive_batch_dev(c->plan, c->tasks.as<tm_task>(), c->devs.as<tm_device>(),
                                 c->stats.as<tm_stats>(), c->status.as<int32_t>(), s);
    if (rc != TM_OK) return rc;
    std::vector<tm_stats> out(G);
    std::vector<int32_t> status(G);
    TM_CUDA(cudaMemcpyAsync(out.data(), c->stats.p, G * sizeof(tm_stats), cudaMemcpyDeviceToHost,
                            s));
    TM_CUDA(cudaMemcpyAsync(status.data(), c->status.p, G * sizeof(int32_t),
                            cudaMemcpyDeviceToHost, s));
    TM_CUDA(cudaStreamSynchronize(s));
    if ((rc = first_error(status.data(), G)) != TM_OK) return rc;
    std::memcpy(stats, out.data(), G * sizeof(tm_stats));
    return TM_OK;
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

}  // extern "C"

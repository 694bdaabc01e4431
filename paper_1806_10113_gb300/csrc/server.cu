// server.cu -- the serving loop (declared in include/tm.h, "serving"): task
// groups arrive one by one; a host worker thread gathers whatever is waiting
// into a batch whenever one of the server's lanes is free (continuous
// batching) and runs it on that lane's CUDA stream.  Exact lanes run the
// exhaustive search for groups small enough to solve exactly; search lanes
// run the beam search (or the paper's heuristic, Sec. 5.1) for the rest, so
// that a small group never waits behind a long search.  Each lane owns fixed
// device and pinned host memory sized at creation; a request waits on the
// host until a lane of its kind has room for it (memory-admitted slots), so
// serving allocates nothing.
//
// Per batch, on the lane's stream: one H2D copy of the packed batch, the
// kernels, one D2H copy of the packed results, an event.  Results of one
// group do not depend on the other groups of its batch.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "learn_internal.h"

namespace {

using Clock = std::chrono::steady_clock;
using tmgpu::GroupPlan;
using tmgpu::Plan;

struct Request {
    uint64_t ticket;
    int32_t n, dma;
    tm_task tasks[TM_MAX_TASKS];
    Clock::time_point t0;
};

inline size_t al16(size_t x) { return (x + 15) & ~size_t(15); }

// Byte layout of one batch's packed input (H2D) block.
struct InLayout {
    size_t off, dev, gp, tasks, bytes;
    InLayout(int G, int T)
    {
        off = 0;
        dev = al16(off + (size_t)(G + 1) * 4);
        gp = al16(dev + (size_t)G * 4);
        tasks = al16(gp + (size_t)(G + 1) * sizeof(GroupPlan));
        bytes = al16(tasks + (size_t)T * sizeof(tm_task));
    }
};

// ... and of its output (D2H) block: exact lanes fill stats and status,
// search lanes status, ms, won and orders.
struct OutLayout {
    size_t stats, status, ms, won, orders, bytes;
    OutLayout(bool exact, int G, int T)
    {
        stats = 0;
        status = al16(exact ? (size_t)G * sizeof(tm_stats) : 0);
        ms = al16(status + (size_t)G * 4);
        won = al16(ms + (exact ? 0 : (size_t)G * 4));
        orders = al16(won + (exact ? 0 : (size_t)G * 4));
        bytes = al16(orders + (exact ? 0 : (size_t)T * 4));
    }
};

struct Lane {
    bool exact = true;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev_done = nullptr;
    unsigned char *h_in = nullptr, *d_in = nullptr, *h_out = nullptr, *d_out = nullptr;
    void* plan_block = nullptr;
    Plan plan;                       // exact lanes
    tmgpu::BeamScratch beam;         // search lanes
    std::vector<Request> reqs;
    int T = 0;
    bool busy = false;
    int launch_rc = TM_OK;
};

}  // namespace

struct tm_server {
    tm_server_config cfg{};
    int device = 0;
    int pdmax = 4;
    uint32_t item_cost = 4096;
    const tm_ranker* ranker = nullptr;
    std::vector<std::unique_ptr<Lane>> lanes;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request> pending[2];          // [0] exact, [1] search
    std::deque<tm_server_result> done;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;
    std::atomic<int64_t> batches{0}, completed{0}, max_batch{0};

    void enqueue(const Request& r) { pending[r.n <= cfg.exact_max_n ? 0 : 1].push_back(r); }
    bool idle() const { return pending[0].empty() && pending[1].empty(); }
    void run();
    bool try_launch(Lane& L);
    void complete(Lane& L);
    void release();
};

namespace {

int check_request(const tm_task* tasks, int n, const tm_device* dev)
{
    if (!tasks || !dev || n < 1 || n > TM_MAX_TASKS) return TM_EINVAL;
    if (dev->dma_engines != 1 && dev->dma_engines != 2) return TM_EINVAL;
    int64_t total = 0;
    for (int i = 0; i < n; ++i) {
        if (tasks[i].htd < 0 || tasks[i].k < 0 || tasks[i].dth < 0) return TM_ENEG;
        total += (int64_t)tasks[i].htd + tasks[i].k + tasks[i].dth;
    }
    return total > INT32_MAX ? TM_EOVERFLOW : TM_OK;
}

}  // namespace

// Gathers waiting requests of the lane's kind into lane L (first come, first
// served, while the lane has room) and enqueues the batch.  Called with `mu`
// held.
bool tm_server::try_launch(Lane& L)
{
    std::deque<Request>& q = pending[L.exact ? 0 : 1];
    if (q.empty()) return false;
    const int Gcap = cfg.lane_groups, Tcap = cfg.lane_tasks;
    const uint32_t Scap = (uint32_t)cfg.lane_subsets;
    int tasks = 0;
    uint32_t subs = 0;
    L.reqs.clear();
    while (!q.empty() && (int)L.reqs.size() < Gcap) {
        const Request& r = q.front();
        const uint32_t c4 = L.exact ? tmgpu::choose4(r.n) : 0u;
        if (tasks + r.n > Tcap || subs + c4 > Scap) break;   // waits for the next free lane
        tasks += r.n;
        subs += c4;
        L.reqs.push_back(r);
        q.pop_front();
    }
    if (L.reqs.empty()) return false;
    L.T = tasks;
    L.busy = true;
    const int G = (int)L.reqs.size(), T = tasks;
    batches.fetch_add(1);
    int64_t mb = max_batch.load();
    while (G > mb && !max_batch.compare_exchange_weak(mb, G)) {}

    // pack the batch into the lane's pinned input block
    const InLayout in(G, T);
    int32_t* h_off = reinterpret_cast<int32_t*>(L.h_in + in.off);
    tm_device* h_dev = reinterpret_cast<tm_device*>(L.h_in + in.dev);
    GroupPlan* h_gp = reinterpret_cast<GroupPlan*>(L.h_in + in.gp);
    tm_task* h_tasks = reinterpret_cast<tm_task*>(L.h_in + in.tasks);
    int off = 0;
    for (int g = 0; g < G; ++g) {
        const Request& r = L.reqs[g];
        h_off[g] = off;
        h_dev[g].dma_engines = r.dma;
        std::memcpy(h_tasks + off, r.tasks, (size_t)r.n * sizeof(tm_task));
        off += r.n;
    }
    h_off[G] = off;
    int rc = TM_OK;
    if (L.exact) {
        rc = tmgpu::plan_decompose(h_off, G, pdmax, item_cost, h_gp, &L.plan);
        if (rc == TM_OK) tmgpu::exhaustive_partition(L.plan, device, cfg.tuning.blocks_per_sm);
        L.plan.d_gp = reinterpret_cast<GroupPlan*>(L.d_in + in.gp);
    }
    const OutLayout out(L.exact, G, T);
    const int32_t* d_off = reinterpret_cast<const int32_t*>(L.d_in + in.off);
    const tm_device* d_dev = reinterpret_cast<const tm_device*>(L.d_in + in.dev);
    const tm_task* d_tasks = reinterpret_cast<const tm_task*>(L.d_in + in.tasks);
    int32_t* d_status = reinterpret_cast<int32_t*>(L.d_out + out.status);
    auto ok = [&](cudaError_t e) { if (e != cudaSuccess && rc == TM_OK) rc = TM_ECUDA; };
    if (rc == TM_OK) ok(cudaMemcpyAsync(L.d_in, L.h_in, in.bytes, cudaMemcpyHostToDevice, L.stream));
    if (rc == TM_OK && L.exact) {
        ok(tmgpu::launch_exhaustive(L.plan, d_tasks, d_dev,
                                    reinterpret_cast<tm_stats*>(L.d_out + out.stats), d_status,
                                    L.stream));
    } else if (rc == TM_OK) {
        int32_t* d_ms = reinterpret_cast<int32_t*>(L.d_out + out.ms);
        int32_t* d_won = reinterpret_cast<int32_t*>(L.d_out + out.won);
        int32_t* d_orders = reinterpret_cast<int32_t*>(L.d_out + out.orders);
        if (cfg.beam_width > 0 && ranker) {
            const int brc = tmgpu::beam_batch(ranker, L.beam, d_tasks, d_off, h_off, G, d_dev,
                                              cfg.beam_width, cfg.refine_starts, d_orders, d_ms,
                                              d_status, d_won, L.stream);
            if (brc != TM_OK) rc = brc;
        } else {
            ok(tmgpu::launch_heuristic(d_tasks, d_off, G, d_dev, d_orders, d_ms, d_status,
                                       L.stream));
            ok(cudaMemsetAsync(d_won, 0, (size_t)G * 4, L.stream));
        }
    }
    if (rc == TM_OK) ok(cudaMemcpyAsync(L.h_out, L.d_out, out.bytes, cudaMemcpyDeviceToHost, L.stream));
    ok(cudaEventRecord(L.ev_done, L.stream));
    L.launch_rc = rc;
    return true;
}

// Turns a finished lane's output block into results.  Called with `mu` held.
void tm_server::complete(Lane& L)
{
    const auto now = Clock::now();
    const int G = (int)L.reqs.size();
    const OutLayout out(L.exact, G, L.T);
    const tm_stats* stats = reinterpret_cast<const tm_stats*>(L.h_out + out.stats);
    const int32_t* status = reinterpret_cast<const int32_t*>(L.h_out + out.status);
    const int32_t* ms = reinterpret_cast<const int32_t*>(L.h_out + out.ms);
    const int32_t* won = reinterpret_cast<const int32_t*>(L.h_out + out.won);
    const int32_t* orders = reinterpret_cast<const int32_t*>(L.h_out + out.orders);
    int off = 0;
    for (int g = 0; g < G; ++g) {
        const Request& r = L.reqs[g];
        tm_server_result res;
        std::memset(&res, 0, sizeof(res));
        res.ticket = r.ticket;
        res.n = r.n;
        res.latency_ns = std::chrono::duration_cast<std::chrono::nanoseconds>(now - r.t0).count();
        res.status = L.launch_rc != TM_OK ? L.launch_rc : status[g];
        for (int i = r.n; i < TM_MAX_TASKS; ++i) res.order[i] = -1;
        if (res.status == TM_OK) {
            if (L.exact) {
                res.method = TM_METHOD_EXHAUSTIVE;
                res.makespan = stats[g].best;
                for (int i = 0; i < r.n; ++i) res.order[i] = stats[g].best_order[i];
            } else {
                res.method = won[g] ? TM_METHOD_BEAM : TM_METHOD_HEURISTIC;
                res.makespan = ms[g];
                for (int i = 0; i < r.n; ++i) res.order[i] = orders[off + i];
            }
        }
        off += r.n;
        done.push_back(res);
    }
    completed.fetch_add(G);
    L.reqs.clear();
    L.busy = false;
}

void tm_server::run()
{
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lock(mu);
    for (;;) {
        bool any_busy = false, progressed = false;
        for (auto& lp : lanes) {
            Lane& L = *lp;
            if (L.busy) {
                const cudaError_t q = cudaEventQuery(L.ev_done);
                if (q == cudaSuccess || q != cudaErrorNotReady) {
                    if (q != cudaSuccess && L.launch_rc == TM_OK) L.launch_rc = TM_ECUDA;
                    complete(L);
                    progressed = true;
                    cv_done.notify_all();
                } else {
                    any_busy = true;
                }
            }
            if (!L.busy && try_launch(L)) {
                any_busy = true;
                progressed = true;
            }
        }
        if (stop && idle() && !any_busy) break;
        if (progressed) continue;
        if (any_busy) {
            // poll the lanes' events; new requests are picked up on the next pass
            lock.unlock();
            std::this_thread::yield();
            lock.lock();
        } else {
            cv_work.wait(lock, [&] { return stop || !idle(); });
        }
    }
}

void tm_server::release()
{
    for (auto& lp : lanes) {
        Lane& L = *lp;
        if (L.stream) cudaStreamSynchronize(L.stream);
        if (L.ev_done) cudaEventDestroy(L.ev_done);
        if (L.stream) cudaStreamDestroy(L.stream);
        if (L.h_in) cudaFreeHost(L.h_in);
        if (L.h_out) cudaFreeHost(L.h_out);
        if (L.d_in) cudaFree(L.d_in);
        if (L.d_out) cudaFree(L.d_out);
        if (L.plan_block) cudaFree(L.plan_block);
        L.beam.release();
    }
    lanes.clear();
}

extern "C" {

int tm_server_create(const tm_server_config* config, const tm_ranker* ranker,
                     tm_server** server_out)
{
    if (!config || !server_out) return TM_EINVAL;
    *server_out = nullptr;
    tm_server_config c = *config;
    if (c.lanes == 0) c.lanes = 2;
    if (c.lane_groups == 0) c.lane_groups = 1024;
    if (c.lane_tasks == 0) c.lane_tasks = TM_MAX_TASKS * c.lane_groups;
    if (c.lane_subsets == 0) c.lane_subsets = 210 * c.lane_groups;
    if (c.lanes < 1 || c.lanes > 8 || c.lane_groups < 1 || c.lane_groups > (1 << 16) ||
        c.lane_tasks < TM_MAX_TASKS || c.lane_tasks > (1 << 22) || c.lane_subsets < 495 ||
        c.lane_subsets > (1 << 26) || c.exact_max_n < 0 || c.exact_max_n > TM_MAX_EXHAUSTIVE ||
        c.beam_width < 0 || c.beam_width > TM_BEAM_MAX_WIDTH || c.refine_starts < 0 ||
        c.refine_starts > TM_BEAM_MAX_REFINE_STARTS)
        return TM_EINVAL;
    if (c.beam_width > 0 && !ranker) return TM_EINVAL;
    const tm_tuning& t = c.tuning;
    if ((t.pdmax != 0 && (t.pdmax < 3 || t.pdmax > 5)) || t.fuse_finalize == 1 ||
        t.fuse_finalize < 0 || t.fuse_finalize > 2 || t.blocks_per_sm < 0 || t.item_cost < 0 ||
        t.item_cost > (1 << 20) || t.chunks_per_thread < 0 || t.chunks_per_thread > 64)
        return TM_EINVAL;
    std::unique_ptr<tm_server> s(new (std::nothrow) tm_server());
    if (!s) return TM_ENOMEM;
    s->cfg = c;
    s->ranker = ranker;
    s->pdmax = t.pdmax ? t.pdmax : 4;
    s->item_cost = t.item_cost ? (uint32_t)t.item_cost : 4096u;
    if (cudaGetDevice(&s->device) != cudaSuccess) return TM_ECUDA;
    if (ranker && ranker->device != s->device) return TM_EINVAL;
    const int Gc = c.lane_groups, Tc = c.lane_tasks;
    const InLayout in(Gc, Tc);
    int rc = TM_OK;
    // c.lanes exact lanes (if any group size is solved exactly), then c.lanes
    // search lanes
    for (int l = 0; l < 2 * c.lanes && rc == TM_OK; ++l) {
        const bool exact = l < c.lanes;
        if (exact && c.exact_max_n == 0) continue;
        if (!exact && c.exact_max_n == TM_MAX_TASKS) continue;
        s->lanes.emplace_back(new Lane());
        Lane& L = *s->lanes.back();
        L.exact = exact;
        const OutLayout out(exact, Gc, Tc);
        auto ok = [&](cudaError_t e) { if (e != cudaSuccess && rc == TM_OK) rc = TM_ENOMEM; };
        ok(cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking));
        ok(cudaEventCreateWithFlags(&L.ev_done, cudaEventDisableTiming));
        ok(cudaHostAlloc(reinterpret_cast<void**>(&L.h_in), in.bytes, cudaHostAllocDefault));
        ok(cudaHostAlloc(reinterpret_cast<void**>(&L.h_out), out.bytes, cudaHostAllocDefault));
        ok(cudaMalloc(reinterpret_cast<void**>(&L.d_in), in.bytes));
        ok(cudaMalloc(reinterpret_cast<void**>(&L.d_out), out.bytes));
        if (rc != TM_OK) break;
        if (exact) {
            // exhaustive-search working memory at the lane's capacity
            Plan& p = L.plan;
            p.G = Gc;
            p.T = Tc;
            p.total_subs = (uint32_t)c.lane_subsets;
            const size_t bytes = tmgpu::plan_carve(p, nullptr);
            ok(cudaMalloc(&L.plan_block, bytes));
            if (rc != TM_OK) break;
            tmgpu::plan_carve(p, static_cast<unsigned char*>(L.plan_block));
            p.d_target = p.d_done = nullptr;   // separate finalize kernel
            p.device = s->device;
            p.chunks_per_thread = t.chunks_per_thread == 0 ? 1 : t.chunks_per_thread;
            // every group's reduction words start (and are left by each
            // finalize) at min = ~0, max = 0, sum = 0
            std::vector<unsigned long long> acc((size_t)tmgpu::kAccStride * Gc, 0ull);
            for (int g = 0; g < Gc; ++g) acc[(size_t)g * tmgpu::kAccStride] = ~0ull;
            ok(cudaMemcpy(p.d_acc, acc.data(), acc.size() * sizeof(unsigned long long),
                          cudaMemcpyHostToDevice));
        } else if (c.beam_width > 0) {
            for (int nm = c.exact_max_n + 1; nm <= TM_MAX_TASKS && rc == TM_OK; ++nm)
                if (!L.beam.reserve(Gc, nm, c.beam_width)) rc = TM_ENOMEM;
        }
    }
    if (rc != TM_OK) {
        s->release();
        return rc;
    }
    tm_server* raw = s.get();
    s->worker = std::thread([raw] { raw->run(); });
    *server_out = s.release();
    return TM_OK;
}

int tm_server_submit(tm_server* s, const tm_task* tasks, int n, const tm_device* dev,
                     uint64_t* ticket_out)
{
    if (!s) return TM_EINVAL;
    if (int rc = check_request(tasks, n, dev)) return rc;
    Request r;
    r.n = n;
    r.dma = dev->dma_engines;
    std::memcpy(r.tasks, tasks, (size_t)n * sizeof(tm_task));
    r.t0 = Clock::now();
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (s->stop) return TM_EINVAL;
        r.ticket = s->next_ticket++;
        s->enqueue(r);
    }
    s->cv_work.notify_one();
    if (ticket_out) *ticket_out = r.ticket;
    return TM_OK;
}

int tm_server_poll(tm_server* s, tm_server_result* out, int max, int wait_us, int* count)
{
    if (!s || !count || max < 0 || (max > 0 && !out)) return TM_EINVAL;
    std::unique_lock<std::mutex> lock(s->mu);
    if (s->done.empty() && wait_us > 0)
        s->cv_done.wait_for(lock, std::chrono::microseconds(wait_us),
                            [&] { return !s->done.empty(); });
    int k = 0;
    while (k < max && !s->done.empty()) {
        out[k++] = s->done.front();
        s->done.pop_front();
    }
    *count = k;
    return TM_OK;
}

int tm_server_replay(tm_server* s, const tm_task* tasks, const int32_t* offsets, int G,
                     const tm_device* devs, const int64_t* arrival_ns, tm_server_result* out)
{
    if (!s || G < 0 || (G > 0 && (!tasks || !offsets || !devs || !arrival_ns || !out)))
        return TM_EINVAL;
    if (G > 0 && offsets[0] != 0) return TM_EINVAL;
    for (int g = 0; g < G; ++g) {
        if (int rc = check_request(tasks + offsets[g], offsets[g + 1] - offsets[g], devs + g))
            return rc;
        if (g > 0 && arrival_ns[g] < arrival_ns[g - 1]) return TM_EINVAL;
    }
    uint64_t first = 0;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (s->stop) return TM_EINVAL;
        first = s->next_ticket;
        s->next_ticket += (uint64_t)G;
    }
    const auto start = Clock::now();
    std::vector<tm_server_result> buf(256);
    int got = 0, g = 0;
    auto collect = [&](int wait_us) {
        int k = 0;
        tm_server_poll(s, buf.data(), (int)buf.size(), wait_us, &k);
        for (int i = 0; i < k; ++i) {
            const uint64_t t = buf[i].ticket;
            if (t >= first && t < first + (uint64_t)G) {
                out[t - first] = buf[i];
                ++got;
            } else {
                // a result of another caller's request: hand it back
                std::lock_guard<std::mutex> lock(s->mu);
                s->done.push_back(buf[i]);
            }
        }
    };
    while (g < G) {
        const auto due = start + std::chrono::nanoseconds(arrival_ns[g]);
        const auto now = Clock::now();
        if (now < due) {
            // far from the next arrival: collect results meanwhile; close to
            // it: spin without touching the server's lock
            const int64_t us =
                std::chrono::duration_cast<std::chrono::microseconds>(due - now).count();
            if (us > 200) collect((int)std::min<int64_t>(us - 100, 1000));
            else std::this_thread::yield();
            continue;
        }
        // every request already due joins the queue in one lock
        {
            std::lock_guard<std::mutex> lock(s->mu);
            for (; g < G && Clock::now() >= start + std::chrono::nanoseconds(arrival_ns[g]); ++g) {
                Request r;
                r.ticket = first + (uint64_t)g;
                r.n = offsets[g + 1] - offsets[g];
                r.dma = devs[g].dma_engines;
                std::memcpy(r.tasks, tasks + offsets[g], (size_t)r.n * sizeof(tm_task));
                r.t0 = start + std::chrono::nanoseconds(arrival_ns[g]);   // the scheduled arrival
                s->enqueue(r);
            }
        }
        s->cv_work.notify_one();
    }
    while (got < G) collect(1000);
    return TM_OK;
}

int tm_server_counters(const tm_server* s, int64_t* batches, int64_t* completed,
                       int64_t* max_batch_groups)
{
    if (!s) return TM_EINVAL;
    if (batches) *batches = s->batches.load();
    if (completed) *completed = s->completed.load();
    if (max_batch_groups) *max_batch_groups = s->max_batch.load();
    return TM_OK;
}

void tm_server_destroy(tm_server* s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    s->release();
    delete s;
}

}  // extern "C"

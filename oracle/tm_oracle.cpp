/*
 * tm_oracle.cpp -- plain, slow CPU oracle (TEST INFRASTRUCTURE ONLY).
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load this code.  It shares nothing with the CUDA library.
 *
 * Model (Sec. 4.1, Figs. 4 and 6).  A task is HtD -> K -> DtH.  Commands are
 * placed in FIFO software queues, one per command type, in the order of the
 * tasks.  The simulation keeps a clock T_sim; at each step the commands at
 * the head of their queue whose predecessor inside the same task has
 * finished start at T_sim; the clock then moves to the earliest end among
 * the running commands, those commands leave their queues, and the step
 * repeats.  The total time of the group is the last end time.
 *   - Two DMA engines (Sec. 3.2, Fig. 3; Fig. 4b): three FIFOs HtD, K, DtH.
 *     HtD and DtH transfers proceed concurrently.
 *   - One DMA engine (Sec. 3.2, Fig. 2; Fig. 4a): all transfers share one
 *     FIFO, filled with every HtD (in task order) and then every DtH (in
 *     task order); so no DtH can start before the last HtD has finished.
 *   - One kernel FIFO: no concurrent kernel execution (end of Sec. 4.1).
 *
 * Readings where the paper is silent or ambiguous (each is listed in the
 * design notes of the repository):
 *   R1  Ideal overlap: concurrent HtD and DtH run at full speed.  The paper's
 *       partially-overlapped transfer model (Sec. 4.2.1, Fig. 5) gives no
 *       formula, and the end-time changes quoted for Fig. 6 fit no single
 *       slowdown factor.
 *   R3  A null stage has duration 0; several commands of one stage are given
 *       as their summed duration (Sec. 4.1).
 *   R4  Commands that end at the same instant are all retired before any new
 *       command starts.  Under R1 this does not change any start time.
 *
 * Exhaustive search (Sec. 1: the brute-force search over N! orders): every
 * order, in lexicographic order starting from the identity, is simulated.
 * Ties for best / worst go to the first order met, i.e. the lowest
 * lexicographic rank.  mean = (double)sum / (double)n!.
 *
 * Heuristic (Sec. 5.1, Algorithm 1).  The paper describes the selection
 * criteria in words only and prints no chosen order, so the readings below
 * are this oracle's; the code is pinned to them by runs of Algorithm 1
 * derived by hand on groups of Table 2 tasks (every update, every candidate's
 * cost, both completions of the last two tasks), and by properties (a valid
 * permutation, the exact optimum for n = 2, never better than the exhaustive
 * best).  Whether a reading is the authors' own is PARITY UNPINNED: nothing
 * in the paper can decide it.
 *   H1  select_first_task: largest K - HtD; ties -> longer DtH; ties -> lower
 *       task index.
 *   H2  update(OT): simulate OT as if it were the whole group; t_HTD, t_K and
 *       t_DTH are the end times of its last HtD, K and DtH command.
 *   H3  select_next_task: a candidate's HtD should fill the kernel time left
 *       after the last HtD (t_K - t_HTD), and its kernel, which starts at
 *       s = max(t_K, t_HTD + HtD_j), should fill the DtH time left after s
 *       (t_DTH - s).  cost_j = |(t_K - t_HTD) - HtD_j| + |(t_DTH - s) - K_j|;
 *       smallest cost wins; ties -> longer K; ties -> lower index.
 *   H4  select_last_tasks: with two tasks {a, b} left, simulate both complete
 *       orders; the shorter total wins; ties -> the order whose last task has
 *       the shorter DtH; ties -> lower index first.
 *   H5  Tasks are T_0..T_{n-1}.  n = 1: [0].  n = 2: select_last_tasks on
 *       both tasks from an empty OT.  n >= 3: Algorithm 1 as written.
 */
#include "tm_oracle.h"

#include <algorithm>
#include <atomic>
#include <climits>
#include <cstdlib>
#include <numeric>
#include <thread>
#include <vector>

namespace {

enum CmdType { HTD = 0, KER = 1, DTH = 2 };

struct Cmd {
    int pos;       /* position of the task in the order */
    int type;      /* HTD, KER or DTH */
    int64_t dur;
};

/* A FIFO software queue with the command that currently runs at its head. */
struct Fifo {
    std::vector<Cmd> items;
    size_t head = 0;
    bool busy = false;
    int64_t end = 0;
    bool empty() const { return head == items.size(); }
    const Cmd& front() const { return items[head]; }
};

int64_t stage(const orc_task& t, int type)
{
    return type == HTD ? t.htd : (type == KER ? t.k : t.dth);
}

/* One simulation run.  Returns the total time, or -1 if the queues could not
 * drain (which the model never allows; kept as a self-check). */
int64_t simulate(const orc_task* tasks, int n, const int32_t* order,
                 int dma_engines, int64_t* timeline)
{
    std::vector<Fifo> fifo(dma_engines == 2 ? 3 : 2);
    if (dma_engines == 2) {
        for (int i = 0; i < n; ++i) {
            const orc_task& t = tasks[order[i]];
            fifo[0].items.push_back({i, HTD, stage(t, HTD)});
            fifo[1].items.push_back({i, KER, stage(t, KER)});
            fifo[2].items.push_back({i, DTH, stage(t, DTH)});
        }
    } else {
        /* One DMA queue: every HtD first, then every DtH (Fig. 2). */
        for (int i = 0; i < n; ++i)
            fifo[0].items.push_back({i, HTD, stage(tasks[order[i]], HTD)});
        for (int i = 0; i < n; ++i)
            fifo[0].items.push_back({i, DTH, stage(tasks[order[i]], DTH)});
        for (int i = 0; i < n; ++i)
            fifo[1].items.push_back({i, KER, stage(tasks[order[i]], KER)});
    }

    std::vector<char> done(3 * n, 0);
    std::vector<int64_t> t_start(3 * n, 0), t_end(3 * n, 0);
    int64_t T_sim = 0;

    for (;;) {
        /* Start every ready head: its queue is free and, for K and DtH, the
         * previous command of the same task has completed. */
        for (Fifo& f : fifo) {
            if (f.busy || f.empty()) continue;
            const Cmd& c = f.front();
            bool ready = (c.type == HTD) || done[3 * c.pos + (c.type - 1)];
            if (!ready) continue;
            f.busy = true;
            f.end = T_sim + c.dur;
            t_start[3 * c.pos + c.type] = T_sim;
        }
        /* Advance the clock to the earliest end among running commands. */
        bool any = false;
        int64_t next = INT64_MAX;
        for (const Fifo& f : fifo)
            if (f.busy) { any = true; next = std::min(next, f.end); }
        if (!any) break;
        T_sim = next;
        /* Retire every command that ends now. */
        for (Fifo& f : fifo) {
            if (!f.busy || f.end != T_sim) continue;
            const Cmd& c = f.front();
            done[3 * c.pos + c.type] = 1;
            t_end[3 * c.pos + c.type] = T_sim;
            f.head++;
            f.busy = false;
        }
    }
    for (const Fifo& f : fifo)
        if (!f.empty()) return -1;

    if (timeline) {
        for (int i = 0; i < n; ++i)
            for (int ty = 0; ty < 3; ++ty) {
                timeline[6 * i + 2 * ty + 0] = t_start[3 * i + ty];
                timeline[6 * i + 2 * ty + 1] = t_end[3 * i + ty];
            }
    }
    return T_sim;
}

/* The partial-overlap variant (Sec. 4.2.1; reading R1' of the build's design
 * notes): while an HtD and a DtH transfer run at the same time, each
 * progresses at the fraction rate_num / rate_den of its full speed, and the
 * end times of the running transfers are re-estimated whenever that changes
 * (Sec. 4.1, Fig. 6: "the overlapping degree is calculated and new end times
 * for both commands are re-calculated").  Time stays on whole nanoseconds: a
 * transfer of d ns holds d * rate_den units of work, progresses rate_den
 * units per ns alone and rate_num units per ns overlapped, and ends at the
 * first whole nanosecond by which its work is done.  Kernels are unaffected.
 * With one DMA engine no two transfers ever run together.  The queue and
 * dependency rules are those of simulate() above. */
int64_t simulate_overlap(const orc_task* tasks, int n, const int32_t* order, int dma_engines,
                         int64_t rate_num, int64_t rate_den, int64_t* timeline)
{
    std::vector<Fifo> fifo(dma_engines == 2 ? 3 : 2);
    for (int i = 0; i < n; ++i) {
        const orc_task& t = tasks[order[i]];
        fifo[0].items.push_back({i, HTD, stage(t, HTD)});
        if (dma_engines == 2) {
            fifo[1].items.push_back({i, KER, stage(t, KER)});
            fifo[2].items.push_back({i, DTH, stage(t, DTH)});
        }
    }
    if (dma_engines == 1) {
        for (int i = 0; i < n; ++i) fifo[0].items.push_back({i, DTH, stage(tasks[order[i]], DTH)});
        for (int i = 0; i < n; ++i) fifo[1].items.push_back({i, KER, stage(tasks[order[i]], KER)});
    }
    std::vector<char> done(3 * n, 0);
    std::vector<int64_t> t_start(3 * n, 0), t_end(3 * n, 0);
    std::vector<int64_t> left(fifo.size(), 0);   /* work left of each running head */
    int64_t T_sim = 0;
    for (;;) {
        for (size_t q = 0; q < fifo.size(); ++q) {
            Fifo& f = fifo[q];
            if (f.busy || f.empty()) continue;
            const Cmd& c = f.front();
            bool ready = (c.type == HTD) || done[3 * c.pos + (c.type - 1)];
            if (!ready) continue;
            f.busy = true;
            left[q] = c.type == KER ? c.dur : c.dur * rate_den;
            t_start[3 * c.pos + c.type] = T_sim;
        }
        /* how many transfers run now decides their speed */
        int transfers = 0;
        for (const Fifo& f : fifo)
            if (f.busy && f.front().type != KER) ++transfers;
        auto speed = [&](const Fifo& f) -> int64_t {
            if (f.front().type == KER) return 1;
            return transfers >= 2 ? rate_num : rate_den;
        };
        /* re-estimate every running command's end from its work left */
        bool any = false;
        int64_t next = INT64_MAX;
        for (size_t q = 0; q < fifo.size(); ++q) {
            Fifo& f = fifo[q];
            if (!f.busy) continue;
            const int64_t v = speed(f);
            f.end = T_sim + (left[q] + v - 1) / v;
            any = true;
            next = std::min(next, f.end);
        }
        if (!any) break;
        for (size_t q = 0; q < fifo.size(); ++q)
            if (fifo[q].busy) left[q] -= speed(fifo[q]) * (next - T_sim);
        T_sim = next;
        for (size_t q = 0; q < fifo.size(); ++q) {
            Fifo& f = fifo[q];
            if (!f.busy || f.end != T_sim) continue;
            const Cmd& c = f.front();
            done[3 * c.pos + c.type] = 1;
            t_end[3 * c.pos + c.type] = T_sim;
            f.head++;
            f.busy = false;
        }
    }
    for (const Fifo& f : fifo)
        if (!f.empty()) return -1;
    if (timeline) {
        for (int i = 0; i < n; ++i)
            for (int ty = 0; ty < 3; ++ty) {
                timeline[6 * i + 2 * ty + 0] = t_start[3 * i + ty];
                timeline[6 * i + 2 * ty + 1] = t_end[3 * i + ty];
            }
    }
    return T_sim;
}

/* Chained tasks (Sec. 6.1, experiment setup): `workers` workers each submit
 * a chain of `rounds` dependent tasks; a worker's next task is released only
 * once its previous task has completely finished.  The paper enumerates
 * (T!)^N orders for T workers and chains of N tasks, i.e. the group runs as
 * N rounds in sequence, round r holding the r-th task of every worker in
 * some order.  Task index r * workers + w is worker w's task of round r; an
 * order `seq` lists the n = workers * rounds task indices, round 0's block
 * first.  The queues are those of simulate(), filled in sequence order, with
 * one extra dependency: the HtD of worker w's round-r task (r >= 1) starts
 * only after the DtH of its round-(r - 1) task has ended.  With one DMA
 * engine each round is submitted as a group of its own: the transfer FIFO
 * holds round 0's HtDs, then round 0's DtHs, then round 1's HtDs, and so on
 * (one FIFO holding every HtD before any DtH could never drain under the
 * chain dependency).  Returns the total time, or -1 if the queues cannot
 * drain (a self-check). */
int64_t simulate_chain(const orc_task* tasks, int workers, int rounds, const int32_t* seq,
                       int dma_engines, int64_t* timeline)
{
    const int n = workers * rounds;
    std::vector<int> pos_of(n, 0);
    for (int p = 0; p < n; ++p) pos_of[seq[p]] = p;
    std::vector<Fifo> fifo(dma_engines == 2 ? 3 : 2);
    if (dma_engines == 2) {
        for (int p = 0; p < n; ++p) {
            const orc_task& t = tasks[seq[p]];
            fifo[0].items.push_back({p, HTD, stage(t, HTD)});
            fifo[1].items.push_back({p, KER, stage(t, KER)});
            fifo[2].items.push_back({p, DTH, stage(t, DTH)});
        }
    } else {
        for (int r = 0; r < rounds; ++r) {
            for (int i = 0; i < workers; ++i) {
                const int p = r * workers + i;
                fifo[0].items.push_back({p, HTD, stage(tasks[seq[p]], HTD)});
            }
            for (int i = 0; i < workers; ++i) {
                const int p = r * workers + i;
                fifo[0].items.push_back({p, DTH, stage(tasks[seq[p]], DTH)});
            }
        }
        for (int p = 0; p < n; ++p) fifo[1].items.push_back({p, KER, stage(tasks[seq[p]], KER)});
    }
    std::vector<char> done(3 * n, 0);
    std::vector<int64_t> t_start(3 * n, 0), t_end(3 * n, 0);
    int64_t T_sim = 0;
    for (;;) {
        for (Fifo& f : fifo) {
            if (f.busy || f.empty()) continue;
            const Cmd& c = f.front();
            bool ready;
            if (c.type == HTD) {
                /* the previous task of the same worker must have finished */
                const int t = seq[c.pos];
                ready = t < workers || done[3 * pos_of[t - workers] + DTH];
            } else {
                ready = done[3 * c.pos + (c.type - 1)];
            }
            if (!ready) continue;
            f.busy = true;
            f.end = T_sim + c.dur;
            t_start[3 * c.pos + c.type] = T_sim;
        }
        bool any = false;
        int64_t next = INT64_MAX;
        for (const Fifo& f : fifo)
            if (f.busy) { any = true; next = std::min(next, f.end); }
        if (!any) break;
        T_sim = next;
        for (Fifo& f : fifo) {
            if (!f.busy || f.end != T_sim) continue;
            const Cmd& c = f.front();
            done[3 * c.pos + c.type] = 1;
            t_end[3 * c.pos + c.type] = T_sim;
            f.head++;
            f.busy = false;
        }
    }
    for (const Fifo& f : fifo)
        if (!f.empty()) return -1;
    if (timeline) {
        for (int i = 0; i < n; ++i)
            for (int ty = 0; ty < 3; ++ty) {
                timeline[6 * i + 2 * ty + 0] = t_start[3 * i + ty];
                timeline[6 * i + 2 * ty + 1] = t_end[3 * i + ty];
            }
    }
    return T_sim;
}

/* Chained orders are enumerated like a counter whose digits are the rounds'
 * permutations, round 0 most significant: the next order advances the last
 * round to its next permutation, and a round that wraps around to its first
 * permutation carries into the round before it.  Each round's block holds
 * fixed task indices, so this is the lexicographic order of the sequences.
 * Returns false after the last order (the sequence is then the first one). */
bool next_chain_order(std::vector<int32_t>& seq, int workers, int rounds, int first_round)
{
    for (int r = rounds - 1; r >= first_round; --r)
        if (std::next_permutation(seq.begin() + r * workers, seq.begin() + (r + 1) * workers))
            return true;
    return false;
}

uint64_t factorial(int n)
{
    uint64_t f = 1;
    for (int i = 2; i <= n; ++i) f *= (uint64_t)i;
    return f;
}

bool valid_tasks(const orc_task* tasks, int n)
{
    for (int i = 0; i < n; ++i)
        if (tasks[i].htd < 0 || tasks[i].k < 0 || tasks[i].dth < 0)
            return false;
    return true;
}

/* Exhaustive search over the orders whose first element is `first`
 * (first < 0: all orders).  Ranks are global lexicographic ranks. */
struct Partial {
    int64_t best = INT64_MAX, worst = INT64_MIN, sum = 0;
    uint64_t best_rank = 0, worst_rank = 0;
    std::vector<int32_t> best_order, worst_order;
};

/* Lexicographic rank of the first order that starts with prefix[0..plen). */
uint64_t prefix_rank(const int32_t* prefix, int plen, int n)
{
    std::vector<char> used(n, 0);
    uint64_t rank = 0;
    for (int i = 0; i < plen; ++i) {
        int smaller = 0;
        for (int e = 0; e < prefix[i]; ++e) smaller += !used[e];
        rank += (uint64_t)smaller * factorial(n - 1 - i);
        used[prefix[i]] = 1;
    }
    return rank;
}

/* Every order that starts with prefix[0..plen), in lexicographic order. */
Partial search_prefix(const orc_task* tasks, int n, int dma, const int32_t* prefix,
                      int plen)
{
    Partial r;
    std::vector<int32_t> p(prefix, prefix + plen);
    std::vector<char> used(n, 0);
    for (int i = 0; i < plen; ++i) used[prefix[i]] = 1;
    for (int e = 0; e < n; ++e)
        if (!used[e]) p.push_back(e);
    uint64_t rank = prefix_rank(prefix, plen, n);
    do {
        int64_t ms = simulate(tasks, n, p.data(), dma, nullptr);
        r.sum += ms;
        if (ms < r.best) { r.best = ms; r.best_rank = rank; r.best_order = p; }
        if (ms > r.worst) { r.worst = ms; r.worst_rank = rank; r.worst_order = p; }
        ++rank;
    } while (std::next_permutation(p.begin() + plen, p.end()));
    return r;
}

Partial search(const orc_task* tasks, int n, int dma, int first)
{
    Partial r;
    std::vector<int32_t> p(n);
    std::iota(p.begin(), p.end(), 0);
    uint64_t rank = 0;
    auto begin = p.begin();
    if (first >= 0) {
        /* [first, remaining ascending]: the first order of that subtree. */
        std::rotate(p.begin(), p.begin() + first, p.begin() + first + 1);
        rank = (uint64_t)first * factorial(n - 1);
        begin = p.begin() + 1;
    }
    do {
        int64_t ms = simulate(tasks, n, p.data(), dma, nullptr);
        r.sum += ms;
        if (ms < r.best) { r.best = ms; r.best_rank = rank; r.best_order = p; }
        if (ms > r.worst) { r.worst = ms; r.worst_rank = rank; r.worst_order = p; }
        ++rank;
    } while (std::next_permutation(begin, p.end()));
    return r;
}

void fill_stats(const Partial& r, int n, orc_stats* out)
{
    out->best = r.best;
    out->worst = r.worst;
    out->sum = r.sum;
    out->mean = (double)r.sum / (double)factorial(n);
    out->best_rank = r.best_rank;
    out->worst_rank = r.worst_rank;
    for (int i = 0; i < 16; ++i) {
        out->best_order[i] = i < n ? r.best_order[i] : -1;
        out->worst_order[i] = i < n ? r.worst_order[i] : -1;
    }
}

int resolve_threads(int nthreads)
{
    if (nthreads > 0) return nthreads;
    unsigned h = std::thread::hardware_concurrency();
    return h ? (int)h : 1;
}

/* Run body(i) for i in [0, count) on a pool of threads. */
template <class F>
void parallel_for(int count, int nthreads, F body)
{
    nthreads = std::max(1, std::min(resolve_threads(nthreads), count));
    std::atomic<int> next{0};
    auto worker = [&]() {
        for (int i = next++; i < count; i = next++) body(i);
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < nthreads; ++t) pool.emplace_back(worker);
    worker();
    for (auto& th : pool) th.join();
}

/* ---- heuristic (Algorithm 1) --------------------------------------------- */

struct EngineTimes { int64_t t_htd, t_k, t_dth; };

/* H2: simulate OT as the whole group, report the ends of its last commands. */
EngineTimes update(const orc_task* tasks, const std::vector<int32_t>& ot,
                   int dma)
{
    int m = (int)ot.size();
    std::vector<int64_t> tl(6 * m);
    simulate(tasks, m, ot.data(), dma, tl.data());
    /* ot holds task indices into `tasks`; simulate() indexes tasks[order[i]]. */
    return {tl[6 * (m - 1) + 1], tl[6 * (m - 1) + 3], tl[6 * (m - 1) + 5]};
}

int64_t total_time(const orc_task* tasks, const std::vector<int32_t>& order,
                   int dma)
{
    return simulate(tasks, (int)order.size(), order.data(), dma, nullptr);
}

int select_first_task(const orc_task* tasks, const std::vector<int32_t>& rt)
{
    int best = -1;
    for (int j : rt) {
        if (best < 0) { best = j; continue; }
        int64_t gj = (int64_t)tasks[j].k - tasks[j].htd;
        int64_t gb = (int64_t)tasks[best].k - tasks[best].htd;
        if (gj > gb || (gj == gb && tasks[j].dth > tasks[best].dth))
            best = j;   /* rt is ascending, so equal keys keep the lower index */
    }
    return best;
}

int select_next_task(const orc_task* tasks, const std::vector<int32_t>& rt,
                     const EngineTimes& e)
{
    int best = -1;
    int64_t best_cost = 0;
    for (int j : rt) {
        int64_t h = tasks[j].htd, k = tasks[j].k;
        int64_t s = std::max(e.t_k, e.t_htd + h);
        int64_t cost = std::llabs((e.t_k - e.t_htd) - h) +
                       std::llabs((e.t_dth - s) - k);
        if (best < 0 || cost < best_cost ||
            (cost == best_cost && tasks[j].k > tasks[best].k)) {
            best = j;
            best_cost = cost;
        }
    }
    return best;
}

void select_last_tasks(const orc_task* tasks, std::vector<int32_t>& ot,
                       int a, int b, int dma)
{
    /* a < b */
    std::vector<int32_t> ab = ot, ba = ot;
    ab.push_back(a); ab.push_back(b);
    ba.push_back(b); ba.push_back(a);
    int64_t m_ab = total_time(tasks, ab, dma);
    int64_t m_ba = total_time(tasks, ba, dma);
    bool take_ba;
    if (m_ab != m_ba) take_ba = m_ba < m_ab;
    else take_ba = tasks[a].dth < tasks[b].dth;  /* last task = a in ba */
    ot = take_ba ? ba : ab;
}

void heuristic(const orc_task* tasks, int n, int dma, int32_t* order_out,
               int64_t* makespan_out)
{
    std::vector<int32_t> rt(n), ot;
    std::iota(rt.begin(), rt.end(), 0);
    auto remove = [&](int j) { rt.erase(std::find(rt.begin(), rt.end(), j)); };

    if (n == 1) {
        ot = {0};
    } else if (n == 2) {
        select_last_tasks(tasks, ot, 0, 1, dma);
    } else {
        int t_ini = select_first_task(tasks, rt);
        ot.push_back(t_ini);
        remove(t_ini);
        EngineTimes e = update(tasks, ot, dma);
        while (rt.size() > 2) {
            int t_next = select_next_task(tasks, rt, e);
            ot.push_back(t_next);
            remove(t_next);
            e = update(tasks, ot, dma);
        }
        select_last_tasks(tasks, ot, rt[0], rt[1], dma);
    }
    for (int i = 0; i < n; ++i) order_out[i] = ot[i];
    if (makespan_out) *makespan_out = total_time(tasks, ot, dma);
}

}  // namespace

extern "C" {

int orc_predict(const orc_task* tasks, int n, const int32_t* order,
                int dma_engines, int64_t* makespan, int64_t* timeline)
{
    if (!tasks || !order || !makespan || n < 1 || n > 64) return -1;
    if (dma_engines != 1 && dma_engines != 2) return -1;
    if (!valid_tasks(tasks, n)) return -1;
    std::vector<char> seen(n, 0);
    for (int i = 0; i < n; ++i) {
        if (order[i] < 0 || order[i] >= n || seen[order[i]]) return -1;
        seen[order[i]] = 1;
    }
    int64_t ms = simulate(tasks, n, order, dma_engines, timeline);
    if (ms < 0) return -1;
    *makespan = ms;
    return 0;
}

int orc_exhaustive(const orc_task* tasks, int n, int dma_engines,
                   orc_stats* out)
{
    if (!tasks || !out || n < 1 || n > 12) return -1;
    if (dma_engines != 1 && dma_engines != 2) return -1;
    if (!valid_tasks(tasks, n)) return -1;
    fill_stats(search(tasks, n, dma_engines, -1), n, out);
    return 0;
}

int orc_exhaustive_batch(const orc_task* tasks, const int32_t* offsets, int G,
                         const int32_t* dma_engines, int nthreads,
                         orc_stats* out)
{
    if (!tasks || !offsets || !dma_engines || !out || G < 0) return -1;
    for (int g = 0; g < G; ++g) {
        int n = offsets[g + 1] - offsets[g];
        if (n < 1 || n > 12) return -1;
        if (dma_engines[g] != 1 && dma_engines[g] != 2) return -1;
        if (!valid_tasks(tasks + offsets[g], n)) return -1;
    }
    /* One work item per (group, first element): subtree ranks are ordered
     * by first element, so merging subtrees in that order keeps the first
     * best / worst. */
    std::vector<int> item_group, item_first;
    for (int g = 0; g < G; ++g) {
        int n = offsets[g + 1] - offsets[g];
        for (int f = 0; f < n; ++f) {
            item_group.push_back(g);
            item_first.push_back(n == 1 ? -1 : f);
            if (n == 1) break;
        }
    }
    std::vector<Partial> parts(item_group.size());
    parallel_for((int)parts.size(), nthreads, [&](int i) {
        int g = item_group[i];
        int n = offsets[g + 1] - offsets[g];
        parts[i] = search(tasks + offsets[g], n, dma_engines[g], item_first[i]);
    });
    size_t i = 0;
    for (int g = 0; g < G; ++g) {
        int n = offsets[g + 1] - offsets[g];
        Partial acc;
        int subtrees = n == 1 ? 1 : n;
        for (int s = 0; s < subtrees; ++s, ++i) {
            const Partial& p = parts[i];
            acc.sum += p.sum;
            if (p.best < acc.best) {
                acc.best = p.best; acc.best_rank = p.best_rank;
                acc.best_order = p.best_order;
            }
            if (p.worst > acc.worst) {
                acc.worst = p.worst; acc.worst_rank = p.worst_rank;
                acc.worst_order = p.worst_order;
            }
        }
        fill_stats(acc, n, out + g);
    }
    return 0;
}

int orc_exhaustive_prefixes(const orc_task* tasks, const int32_t* offsets,
                            const int32_t* dma_engines, const int32_t* item_group,
                            const int32_t* item_prefix, int plen, int nitems,
                            int nthreads, orc_stats* out)
{
    if (!tasks || !offsets || !dma_engines || !item_group || !out || nitems < 0 ||
        plen < 0 || (plen > 0 && !item_prefix))
        return -1;
    for (int i = 0; i < nitems; ++i) {
        int g = item_group[i];
        int n = offsets[g + 1] - offsets[g];
        if (n < 1 || n > 12 || plen > n) return -1;
        if (dma_engines[g] != 1 && dma_engines[g] != 2) return -1;
        std::vector<char> seen(n, 0);
        for (int j = 0; j < plen; ++j) {
            int e = item_prefix[plen * i + j];
            if (e < 0 || e >= n || seen[e]) return -1;
            seen[e] = 1;
        }
    }
    parallel_for(nitems, nthreads, [&](int i) {
        int g = item_group[i];
        int n = offsets[g + 1] - offsets[g];
        Partial r = search_prefix(tasks + offsets[g], n, dma_engines[g],
                                  item_prefix + plen * i, plen);
        fill_stats(r, n, out + i);
        out[i].mean = (double)r.sum / (double)factorial(n - plen);
    });
    return 0;
}

int orc_heuristic(const orc_task* tasks, int n, int dma_engines,
                  int32_t* order_out, int64_t* makespan_out)
{
    if (!tasks || !order_out || n < 1 || n > 16) return -1;
    if (dma_engines != 1 && dma_engines != 2) return -1;
    if (!valid_tasks(tasks, n)) return -1;
    heuristic(tasks, n, dma_engines, order_out, makespan_out);
    return 0;
}

int orc_heuristic_batch(const orc_task* tasks, const int32_t* offsets, int G,
                        const int32_t* dma_engines, int nthreads,
                        int32_t* orders_out, int64_t* makespans_out)
{
    if (!tasks || !offsets || !dma_engines || !orders_out || G < 0) return -1;
    for (int g = 0; g < G; ++g) {
        int n = offsets[g + 1] - offsets[g];
        if (n < 1 || n > 16) return -1;
        if (dma_engines[g] != 1 && dma_engines[g] != 2) return -1;
        if (!valid_tasks(tasks + offsets[g], n)) return -1;
    }
    parallel_for(G, nthreads, [&](int g) {
        int n = offsets[g + 1] - offsets[g];
        heuristic(tasks + offsets[g], n, dma_engines[g],
                  orders_out + offsets[g],
                  makespans_out ? makespans_out + g : nullptr);
    });
    return 0;
}

int orc_predict_overlap(const orc_task* tasks, int n, const int32_t* order, int dma_engines,
                        int32_t rate_num, int32_t rate_den, int64_t* makespan,
                        int64_t* timeline)
{
    if (!tasks || !order || !makespan || n < 1 || n > 64) return -1;
    if (dma_engines != 1 && dma_engines != 2) return -1;
    if (rate_num < 1 || rate_den < rate_num) return -1;
    if (!valid_tasks(tasks, n)) return -1;
    std::vector<char> seen(n, 0);
    for (int i = 0; i < n; ++i) {
        if (order[i] < 0 || order[i] >= n || seen[order[i]]) return -1;
        seen[order[i]] = 1;
    }
    int64_t ms = simulate_overlap(tasks, n, order, dma_engines, rate_num, rate_den, timeline);
    if (ms < 0) return -1;
    *makespan = ms;
    return 0;
}

int orc_exhaustive_overlap(const orc_task* tasks, int n, int dma_engines, int32_t rate_num,
                           int32_t rate_den, orc_stats* out)
{
    if (!tasks || !out || n < 1 || n > 12) return -1;
    if (dma_engines != 1 && dma_engines != 2) return -1;
    if (rate_num < 1 || rate_den < rate_num) return -1;
    if (!valid_tasks(tasks, n)) return -1;
    std::vector<int32_t> p(n);
    std::iota(p.begin(), p.end(), 0);
    int64_t best = INT64_MAX, worst = INT64_MIN, sum = 0;
    uint64_t rank = 0, best_rank = 0, worst_rank = 0;
    std::vector<int32_t> best_order, worst_order;
    do {
        const int64_t ms = simulate_overlap(tasks, n, p.data(), dma_engines, rate_num, rate_den,
                                            nullptr);
        if (ms < 0) return -1;
        sum += ms;
        if (ms < best) { best = ms; best_rank = rank; best_order = p; }
        if (ms > worst) { worst = ms; worst_rank = rank; worst_order = p; }
        ++rank;
    } while (std::next_permutation(p.begin(), p.end()));
    out->best = best;
    out->worst = worst;
    out->sum = sum;
    out->mean = (double)sum / (double)factorial(n);
    out->best_rank = best_rank;
    out->worst_rank = worst_rank;
    for (int i = 0; i < 16; ++i) {
        out->best_order[i] = i < n ? best_order[i] : -1;
        out->worst_order[i] = i < n ? worst_order[i] : -1;
    }
    return 0;
}

static bool valid_chain_seq(const int32_t* seq, int workers, int rounds)
{
    const int n = workers * rounds;
    std::vector<char> seen(n, 0);
    for (int p = 0; p < n; ++p) {
        const int t = seq[p];
        if (t < 0 || t >= n || seen[t] || t / workers != p / workers) return false;
        seen[t] = 1;
    }
    return true;
}

static bool valid_chain_shape(int workers, int rounds)
{
    return workers >= 1 && workers <= 8 && rounds >= 1 && workers * rounds <= 16;
}

int orc_predict_chain(const orc_task* tasks, int workers, int rounds, const int32_t* seq,
                      int dma_engines, int64_t* makespan, int64_t* timeline)
{
    if (!tasks || !seq || !makespan || !valid_chain_shape(workers, rounds)) return -1;
    if (dma_engines != 1 && dma_engines != 2) return -1;
    if (!valid_tasks(tasks, workers * rounds) || !valid_chain_seq(seq, workers, rounds))
        return -1;
    const int64_t ms = simulate_chain(tasks, workers, rounds, seq, dma_engines, timeline);
    if (ms < 0) return -1;
    *makespan = ms;
    return 0;
}

int orc_exhaustive_chain_batch(const orc_task* tasks, const int32_t* offsets,
                               const int32_t* workers, int G, const int32_t* dma_engines,
                               int nthreads, orc_stats* out)
{
    if (!tasks || !offsets || !workers || !dma_engines || !out || G < 0) return -1;
    for (int g = 0; g < G; ++g) {
        const int n = offsets[g + 1] - offsets[g], w = workers[g];
        if (w < 1 || n % w != 0 || !valid_chain_shape(w, n / w)) return -1;
        if (dma_engines[g] != 1 && dma_engines[g] != 2) return -1;
        if (!valid_tasks(tasks + offsets[g], n)) return -1;
    }
    /* One work item per (group, permutation of the first round); item q of a
     * group covers ranks [q * (T!)^(N-1), (q + 1) * (T!)^(N-1)). */
    std::vector<int> item_group, item_q;
    for (int g = 0; g < G; ++g)
        for (uint64_t q = 0; q < factorial(workers[g]); ++q) {
            item_group.push_back(g);
            item_q.push_back((int)q);
        }
    std::vector<Partial> parts(item_group.size());
    parallel_for((int)parts.size(), nthreads, [&](int i) {
        const int g = item_group[i], T = workers[g];
        const int n = offsets[g + 1] - offsets[g], R = n / T;
        const orc_task* t = tasks + offsets[g];
        std::vector<int32_t> seq(n);
        std::iota(seq.begin(), seq.end(), 0);
        /* round 0's permutation of lexicographic rank q: its digits in the
         * factorial number system pick, position by position, among the
         * task indices not yet used */
        std::vector<int32_t> rest(seq.begin(), seq.begin() + T);
        uint64_t q = (uint64_t)item_q[i];
        for (int j = 0; j < T; ++j) {
            const uint64_t f = factorial(T - 1 - j);
            seq[j] = rest[q / f];
            rest.erase(rest.begin() + (long)(q / f));
            q %= f;
        }
        uint64_t per_first = 1;
        for (int r = 1; r < R; ++r) per_first *= factorial(T);
        uint64_t rank = (uint64_t)item_q[i] * per_first;
        Partial& pr = parts[i];
        do {
            const int64_t ms = simulate_chain(t, T, R, seq.data(), dma_engines[g], nullptr);
            pr.sum += ms;
            if (ms < pr.best) { pr.best = ms; pr.best_rank = rank; pr.best_order = seq; }
            if (ms > pr.worst) { pr.worst = ms; pr.worst_rank = rank; pr.worst_order = seq; }
            ++rank;
        } while (next_chain_order(seq, T, R, 1));
    });
    size_t i = 0;
    for (int g = 0; g < G; ++g) {
        const int T = workers[g], n = offsets[g + 1] - offsets[g], R = n / T;
        Partial acc;
        for (uint64_t q = 0; q < factorial(T); ++q, ++i) {
            const Partial& p = parts[i];
            acc.sum += p.sum;
            if (p.best < acc.best) {
                acc.best = p.best; acc.best_rank = p.best_rank; acc.best_order = p.best_order;
            }
            if (p.worst > acc.worst) {
                acc.worst = p.worst; acc.worst_rank = p.worst_rank;
                acc.worst_order = p.worst_order;
            }
        }
        fill_stats(acc, n, out + g);
        uint64_t count = 1;
        for (int r = 0; r < R; ++r) count *= factorial(T);
        out[g].mean = (double)acc.sum / (double)count;
    }
    return 0;
}

int orc_exhaustive_chain(const orc_task* tasks, int workers, int rounds, int dma_engines,
                         orc_stats* out)
{
    if (!valid_chain_shape(workers, rounds)) return -1;
    const int32_t offsets[2] = {0, workers * rounds};
    const int32_t w = workers, d = dma_engines;
    return orc_exhaustive_chain_batch(tasks, offsets, &w, 1, &d, 0, out);
}

int orc_hardware_threads(void) { return resolve_threads(0); }

}  // extern "C"

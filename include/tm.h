/*
 * tm.h -- C ABI of libtm.so: the temporal execution model, exhaustive order
 * search and task reordering heuristic of Lazaro-Munoz et al., "Improving
 * tasks throughput on accelerators using OpenCL command concurrency"
 * (arXiv 1806.10113), evaluated by hand-written CUDA kernels for sm_103a.
 *
 * THE MODEL (Sec. 4.1, Figs. 4 and 6).  A task group TG is n independent
 * tasks; task j is an HtD transfer, a kernel K and a DtH transfer, run in
 * that order, with durations htd_j, k_j, dth_j (int32 nanoseconds).  For an
 * order (a permutation tau of 0..n-1), commands enter FIFO queues in that
 * order and each starts once its queue is free and the previous stage of
 * its own task has finished.  There is one kernel queue (no concurrent
 * kernel execution).  With two DMA engines (Sec. 3.2, Fig. 3) HtD and DtH
 * have their own queues and overlap at full speed; with one DMA engine
 * (Sec. 3.2, Fig. 2) one transfer queue carries every HtD and then every
 * DtH.  The result ("makespan") is the end of the last command.  Concurrent
 * HtD/DtH transfers are modelled at full speed: the paper's partial-overlap
 * slowdown (Sec. 4.2.1) gives no formula.
 *
 * CONVENTIONS.
 *  - Every function returns TM_OK (0) or a negative tm_status code; on error
 *    no output is written.  tm_strerror() names a code.
 *  - Functions without the _dev suffix take HOST pointers, run on the
 *    calling thread's current CUDA device and return when the results are
 *    in the caller's buffers.  They keep no caller pointer after returning.
 *    Their device buffers are owned by the library, one set per host thread,
 *    reused across calls and grown when needed.
 *  - _dev functions take DEVICE pointers and a CUDA stream (passed as
 *    void*, NULL = legacy default stream) and are stream-ordered: they
 *    return after enqueuing work.  Their per-group input checks run on the
 *    device and are reported in an optional int32 status[G] array (0 or a
 *    tm_status code); a group that fails its check gets no output.
 *  - Ragged batches: group g owns tasks[offsets[g] .. offsets[g+1]),
 *    offsets[0] = 0, offsets nondecreasing, 1 <= offsets[g+1]-offsets[g].
 *    Orders are given and returned with the same layout, holding task
 *    indices local to their group (0 .. n_g - 1).
 *  - Input limits: durations >= 0 (else TM_ENEG); the sum of all durations
 *    of a group <= INT32_MAX (else TM_EOVERFLOW), which bounds every time
 *    the model produces; n <= TM_MAX_TASKS (16); exhaustive search needs
 *    n <= TM_MAX_EXHAUSTIVE (12, so that n! < 2^32) (else TM_ETOOBIG).
 *  - The library is thread-safe across host threads.  A tm_plan must not be
 *    used by two launches that can run at the same time.
 */
#ifndef TM_H
#define TM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TM_MAX_TASKS 16
#define TM_MAX_EXHAUSTIVE 12

typedef enum tm_status {
    TM_OK = 0,
    TM_EINVAL = -1,     /* NULL pointer, n or G out of range, bad offsets,
                           dma_engines not 1 or 2, order not a permutation */
    TM_ENEG = -2,       /* a negative duration */
    TM_EOVERFLOW = -3,  /* a group's durations sum above INT32_MAX */
    TM_ETOOBIG = -4,    /* exhaustive search asked for n > 12 */
    TM_ECUDA = -5,      /* a CUDA runtime call failed */
    TM_ETIMEOUT = -6,   /* a bounded device-side wait expired */
    TM_ENOMEM = -7,     /* device or host allocation failed */
    TM_ECAPACITY = -8   /* batch larger than tm_exhaustive_batch_noalloc's
                           fixed working memory */
} tm_status;

/* One task (Sec. 4.1): durations of its three stages in ns.  A null stage is
 * 0; a stage made of several commands is given as their sum.  12 bytes. */
typedef struct tm_task {
    int32_t htd, k, dth;
} tm_task;

/* Device model (Sec. 3.2): the number of DMA engines, 1 or 2. */
typedef struct tm_device {
    int32_t dma_engines;
} tm_device;

/* Result of an exhaustive search over all n! orders of one group.
 * Ranks are lexicographic ranks of the order (rank 0 = 0,1,...,n-1); ties
 * for best / worst go to the lowest rank.  Entries of best_order /
 * worst_order past n are 0xFF.  72 bytes, 8-byte aligned. */
typedef struct tm_stats {
    int32_t best;           /* minimum makespan (ns) */
    int32_t worst;          /* maximum makespan (ns) */
    int64_t sum;            /* exact sum of all n! makespans */
    double mean;            /* (double)sum / (double)n!, IEEE round-to-nearest */
    uint64_t best_rank;
    uint64_t worst_rank;
    uint8_t best_order[16];
    uint8_t worst_order[16];
} tm_stats;

/* ---- single group, host pointers --------------------------------------- */

/* Makespan of one order (Sec. 4.1).  tasks[n], order[n] (a permutation of
 * 0..n-1); writes *makespan.  1 <= n <= 16. */
int tm_predict(const tm_task* tasks, int n, const int32_t* order,
               const tm_device* dev, int32_t* makespan);

/* Evaluates all n! orders (the brute-force search of Sec. 1 that the paper
 * calls infeasible at run time) and reduces them to best / worst / sum /
 * mean with the first best and worst order.  1 <= n <= 12.  `mean` may be
 * NULL; otherwise it receives stats->mean. */
int tm_exhaustive(const tm_task* tasks, int n, const tm_device* dev,
                  tm_stats* stats, double* mean);

/* Batch Reordering heuristic (Sec. 5.1, Algorithm 1) with these readings:
 *  select_first_task: largest k - htd; ties -> larger dth -> lower index.
 *  update(OT): the model run on the ordered set OT alone; t_HTD, t_K, t_DTH
 *    are the ends of its last HtD, K and DtH.
 *  select_next_task: minimise |(t_K - t_HTD) - htd_j| + |(t_DTH - s_j) - k_j|
 *    with s_j = max(t_K, t_HTD + htd_j); ties -> larger k -> lower index.
 *  select_last_tasks: with two tasks left, the completion with the smaller
 *    makespan; ties -> the one whose last task has the smaller dth -> lower
 *    index first.  n = 1 gives [0]; n = 2 applies select_last_tasks to both.
 * Writes order_out[n] and, if not NULL, *makespan_out.  1 <= n <= 16. */
int tm_heuristic(const tm_task* tasks, int n, const tm_device* dev,
                 int32_t* order_out, int32_t* makespan_out);

/* ---- ragged batches, host pointers -------------------------------------- */

/* devs[G]: one device model per group.  orders / makespans as above. */
int tm_predict_batch(const tm_task* tasks, const int32_t* offsets, int G,
                     const int32_t* orders, const tm_device* devs,
                     int32_t* makespans);

int tm_exhaustive_batch(const tm_task* tasks, const int32_t* offsets, int G,
                        const tm_device* devs, tm_stats* stats);

int tm_heuristic_batch(const tm_task* tasks, const int32_t* offsets, int G,
                       const tm_device* devs, int32_t* orders_out,
                       int32_t* makespans_out /* may be NULL */);

/* ---- ragged batches, device pointers, stream-ordered --------------------- */

int tm_predict_batch_dev(const tm_task* d_tasks, const int32_t* d_offsets,
                         int G, const int32_t* d_orders,
                         const tm_device* d_devs, int32_t* d_makespans,
                         int32_t* d_status /* may be NULL */, void* stream);

int tm_heuristic_batch_dev(const tm_task* d_tasks, const int32_t* d_offsets,
                           int G, const tm_device* d_devs,
                           int32_t* d_orders_out,
                           int32_t* d_makespans_out /* may be NULL */,
                           int32_t* d_status /* may be NULL */, void* stream);

/* An exhaustive-search plan fixes the group sizes of a batch and the work
 * decomposition over them; it owns the device work list and the per-group
 * reduction words.  Creating it checks sizes (TM_EINVAL, TM_ETOOBIG) and
 * allocates device memory on the current device; executing it allocates
 * nothing.  h_offsets: host array of G + 1 offsets. */
typedef struct tm_plan tm_plan;

int tm_plan_create(const int32_t* h_offsets, int G, tm_plan** plan_out);

/* Tuning knobs of an exhaustive-search plan (an autotuner picks them; 0
 * means "the library's default").  None changes any result.
 *   pdmax          prefix positions each work item walks depth-first, 3..5
 *                  (a work item holds pdmax! x 24 orders; default 4)
 *   fuse_finalize  1: each group is finalized by the last enumeration
 *                  thread to finish it (one launch fewer); 2: a separate
 *                  finalize kernel; 0: default (2)
 *   blocks_per_sm  resident enumeration blocks per SM used to size the
 *                  work split, 1..occupancy limit; 0: the occupancy limit
 *   item_cost      the work split gives each thread the same estimated cost,
 *                  a work item costing its orders plus item_cost (fixed
 *                  per-item work, in orders); 0: default 4096
 *   chunks_per_thread  1: each enumeration thread takes one fixed share of
 *                  the cost; 2..64: the cost is cut into that many chunks per
 *                  thread, which warps take from a counter as they finish
 *                  (dynamic balance, for batches whose orders cost unevenly;
 *                  needs fuse_finalize != 1); 0: default 1
 *   unroll         1: the depth-first walk's level with three prefix tasks
 *                  left runs as straight-line code, and the orders' sum
 *                  shares the FMA pipe (faster on batches of one group
 *                  size); 2: as a loop (less code: faster on batches that
 *                  mix group sizes); 3: as 1, with each order's addition
 *                  on the FMA pipe too; 4: as 3, compiled for four
 *                  resident blocks per SM (at most 128 registers); 5: as
 *                  3, and a prefix whose 24 completions all end on one
 *                  engine's path (the DtH engine's, the kernel engine's or
 *                  the HtD engine's, on every lane of the warp) takes the
 *                  closed form of their minimum, maximum and sum; 6: as
 *                  5, with the suffix tables' beta and gamma held in
 *                  shared memory (24 KB per block) instead of registers,
 *                  compiled for four resident blocks per SM; 7: as 6, with
 *                  the dominance vote and the closed forms of a level's
 *                  six prefixes in one pass and less unrolled code (faster
 *                  on batches of 10-task groups, slower on 12-task ones);
 *                  8: as 6 with 7's less unrolled code (faster on batches
 *                  that mix group sizes); 0: default 2 */
typedef struct tm_tuning {
    int32_t pdmax;
    int32_t fuse_finalize;
    int32_t blocks_per_sm;
    int32_t item_cost;
    int32_t chunks_per_thread;
    int32_t unroll;
} tm_tuning;

int tm_plan_create_tuned(const int32_t* h_offsets, int G, const tm_tuning* tuning,
                         tm_plan** plan_out);

/* Process-wide tuning used by tm_plan_create and by the plans that the
 * host-pointer exhaustive calls build internally (NULL restores the
 * library's defaults).  Plans created earlier keep their tuning.  Returns
 * TM_EINVAL for out-of-range knobs. */
int tm_set_default_tuning(const tm_tuning* tuning);
void tm_plan_destroy(tm_plan* plan);

/* Runs the exhaustive search of every group of the plan.  d_tasks must use
 * the plan's offsets; d_stats[G].  Stream-ordered; launches of one plan must
 * not overlap. */
int tm_exhaustive_batch_dev(const tm_plan* plan, const tm_task* d_tasks,
                            const tm_device* d_devs, tm_stats* d_stats,
                            int32_t* d_status /* may be NULL */, void* stream);

/* The whole scheduling pass of the paper's method for every group of the
 * plan: the exhaustive search (d_stats) and the reordering heuristic
 * (d_orders_out in the task layout; d_makespans_out may be NULL), in the
 * plan's launches (tm_plan_launches: prep, enumeration, finalize; the
 * heuristic's warps run beside the finalize warps).  Same results as
 * tm_exhaustive_batch_dev followed by tm_heuristic_batch_dev.  d_status
 * reports the per-group input checks. */
int tm_schedule_batch_dev(const tm_plan* plan, const tm_task* d_tasks,
                          const tm_device* d_devs, tm_stats* d_stats,
                          int32_t* d_orders_out, int32_t* d_makespans_out,
                          int32_t* d_status /* may be NULL */, void* stream);

/* Host-pointer form of tm_schedule_batch_dev (synchronous).  n <= 12.  The
 * calling thread's plan for the last batch shape is kept, and its launches
 * are captured once as a CUDA graph that later calls with the same shape
 * replay; inputs and results pass through mapped page-locked memory. */
int tm_schedule_batch(const tm_task* tasks, const int32_t* offsets, int G,
                      const tm_device* devs, tm_stats* stats,
                      int32_t* orders_out, int32_t* makespans_out /* may be NULL */);

/* CUDA graph of one scheduling pass.  tm_plan_capture records one
 * tm_schedule_batch_dev pass over these fixed device buffers (d_makespans
 * and d_status may be NULL) into a graph owned by the plan (replacing any
 * earlier one; timing events set with tm_plan_set_timing are recorded too);
 * tm_plan_graph_launch replays it on a stream: same results, one launch call
 * per pass.  The buffers must stay valid while the graph is used.  Capture
 * uses a private stream of the library; it allocates the graph. */
int tm_plan_capture(tm_plan* plan, const tm_task* d_tasks, const tm_device* d_devs,
                    tm_stats* d_stats, int32_t* d_orders_out, int32_t* d_makespans_out,
                    int32_t* d_status);
int tm_plan_graph_launch(const tm_plan* plan, void* stream);

/* If the graph was captured with timing events set (tm_plan_set_timing),
 * makes later replays record these events instead, around the enumeration
 * kernel (no new capture).  TM_EINVAL if the graph has no timing nodes. */
int tm_plan_graph_set_timing(tm_plan* plan, void* event_before, void* event_after);

/* Number of kernel launches one tm_exhaustive_batch_dev call enqueues
 * (tm_schedule_batch_dev enqueues the same number). */
int tm_plan_launches(const tm_plan* plan);

/* Optional timing hook: cudaEvent_t handles (passed as void*, created by the
 * caller with timing enabled) that every later tm_exhaustive_batch_dev call
 * on this plan records on its stream immediately before and after its
 * enumeration kernel.  NULL, NULL turns it off.  The plan does not own the
 * events; the caller keeps them alive while the hook is set.  Without the
 * hook the finalize launch is a programmatic dependent launch (it may start
 * while the enumeration finishes, and waits for its results); with it the
 * pass runs in plain stream order. */
int tm_plan_set_timing(tm_plan* plan, void* event_before, void* event_after);

/* Work counts of the plan's last run, for measuring it (the exhaustive
 * search's decomposition: each order is a prefix of n - 4 tasks and one of
 * the 24 orders of the other four; Sec. 1's brute force over every order).
 * *prefixes: the prefixes one run walks, n! / 24 per group of n >= 4 tasks.
 * *full: how many of them had their 24 completions evaluated one by one;
 * under walk modes 5 to 8 (tm_tuning.unroll) the others took the closed
 * form of their minimum, maximum and sum; every other mode evaluates all of
 * them, and *full = *prefixes without a device read.  Modes 5 to 8 read a counter in
 * the plan's device memory (a synchronous copy): call it once the run has
 * finished (its stream synchronized).  Returns TM_OK, TM_EINVAL (a NULL
 * argument) or TM_ECUDA. */
int tm_plan_walk_counts(const tm_plan* plan, unsigned long long* prefixes,
                        unsigned long long* full);

/* ---- exhaustive search without any allocation ---------------------------- */

/* The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory: a caller whose GPU memory is all
 * reserved by another allocator (for example a framework's caching pool),
 * or one that cannot afford cudaMalloc / cudaFree (cudaFree waits for the
 * whole device) where it runs.  tm_plan_create allocates; this call does
 * not.  It computes the same results as tm_exhaustive_batch_dev, bit for
 * bit, with its working memory in one fixed 1 MiB device array inside
 * libtm.so (held by every GPU that loads the library until the process
 * exits) instead of a plan.
 *   d_tasks, d_devs, d_stats, d_status: device pointers as in
 *     tm_exhaustive_batch_dev (d_status may be NULL); h_offsets: HOST array
 *     of G + 1 offsets.
 *   Limits: G <= TM_NOALLOC_MAX_GROUPS, offsets[G] <= TM_NOALLOC_MAX_TASKS
 *     and sum over groups of C(n, 4) <= TM_NOALLOC_MAX_SUBSETS, else
 *     TM_ECAPACITY (e.g. 64 groups of 8 tasks, or 9 groups of 12 fit);
 *     n <= 12 per group, else TM_ETOOBIG.
 *   It calls no cudaMalloc, cudaFree or other allocating routine.  The first
 *     call on a device (with that device current) does a one-time set-up:
 *     it looks up the array's device address and loads every kernel the
 *     call can launch.  Under lazy module loading (the CUDA default) that
 *     loading is what places the array in device memory, so make the first
 *     call before your own allocator reserves the device's memory (or set
 *     CUDA_MODULE_LOADING=EAGER), and before starting any stream capture.
 *     After the device's context changes (cudaDeviceReset) the next call
 *     repeats the set-up, under the same rules.
 *   Every call uses the same array, which keeps the previous call's
 *     contents; each call resets what must start from a known value.  Calls
 *     whose work can overlap on the GPU race on the array: serialise them.
 * Stream-ordered: returns after enqueuing its kernels. */
#define TM_NOALLOC_MAX_GROUPS 64
#define TM_NOALLOC_MAX_TASKS 768
#define TM_NOALLOC_MAX_SUBSETS 4800

int tm_exhaustive_batch_noalloc(const tm_task* d_tasks, const int32_t* h_offsets,
                                int G, const tm_device* d_devs, tm_stats* d_stats,
                                int32_t* d_status /* may be NULL */, void* stream);

/* ---- chained tasks ------------------------------------------------------------ */

/* The paper's experiment setup (Sec. 6.1): T workers each submit a chain of
 * N dependent tasks, a worker's next task released only when its previous
 * task has completely finished; the paper counts (T!)^N orders, i.e. the
 * group runs as N rounds in sequence, round r holding the r-th task of every
 * worker in some order.
 *   Layout: a chained group of n = T * N tasks (1 <= T <=
 *     TM_CHAIN_MAX_WORKERS, n <= TM_MAX_TASKS); tasks[r * T + w] is worker
 *     w's round-r task.  An order lists the n task indices round by round:
 *     positions r T .. r T + T - 1 hold a permutation of round r's indices.
 *   Model: the queues of Sec. 4.1 filled in that order, plus one dependency:
 *     the HtD of worker w's round-r task starts after the DtH of its
 *     round-(r - 1) task has ended.  With one DMA engine each round is
 *     submitted as a group of its own (its HtDs, then its DtHs, in the one
 *     transfer queue, round after round).
 *   Search: all (T!)^N orders, ranked lexicographically (the rounds as the
 *     digits of a counter, round 0 most significant), reduced as
 *     tm_exhaustive does (first best / worst rank, exact sum, mean = sum /
 *     (T!)^N); best_order / worst_order hold task indices (0xFF past n).
 *   Errors: TM_EINVAL for a bad shape (T, n % T, n) or an order that breaks
 *     the round layout; the input errors of tm_predict otherwise.  Host
 *     calls are synchronous and leave outputs untouched on error; _dev calls
 *     are stream-ordered and report per group in d_status (may be NULL),
 *     with h_offsets / h_workers the HOST copies of the device arrays. */
#define TM_CHAIN_MAX_WORKERS 8

int tm_predict_chain(const tm_task* tasks, int workers, int rounds, const int32_t* order,
                     const tm_device* dev, int32_t* makespan);
int tm_exhaustive_chain(const tm_task* tasks, int workers, int rounds, const tm_device* dev,
                        tm_stats* out);
/* Ragged batch: group g owns tasks[offsets[g] .. offsets[g + 1]) and has
 * workers[g] workers. */
int tm_exhaustive_chain_batch(const tm_task* tasks, const int32_t* offsets,
                              const int32_t* workers, int G, const tm_device* devs,
                              tm_stats* out);
int tm_exhaustive_chain_batch_dev(const tm_task* d_tasks, const int32_t* d_offsets,
                                  const int32_t* h_offsets, const int32_t* d_workers,
                                  const int32_t* h_workers, int G, const tm_device* d_devs,
                                  tm_stats* d_stats, int32_t* d_status, void* stream);
int tm_predict_chain_batch_dev(const tm_task* d_tasks, const int32_t* d_offsets,
                               const int32_t* d_workers, int G, const int32_t* d_orders,
                               const tm_device* d_devs, int32_t* d_makespans, int32_t* d_status,
                               void* stream);
/* Work counts of the calling host thread's last exhaustive chained search
 * (any of the three forms above), for measuring it.  Groups of four workers
 * and at least two rounds end every order with the last round's 24 orders of
 * the four workers (a "tail" block); *tails counts those blocks, *closed
 * those that took the closed form of the case where the HtD engine's path
 * ends all 24 (decided by one vote over a warp's blocks; the others are
 * evaluated order by order).  Reads a device counter synchronously: call it
 * once the search has finished.  TM_OK, TM_EINVAL (a NULL argument) or
 * TM_ECUDA; both 0 before any search. */
int tm_chain_tail_counts(unsigned long long* tails, unsigned long long* closed);

/* ---- partial-overlap variant of the model --------------------------------- */

/* The paper's simulator also slows down an HtD and a DtH transfer that run
 * at the same time on two DMA engines, re-estimating both end times whenever
 * such an overlap starts or ends (Sec. 4.1, Fig. 6; Sec. 4.2.1); it gives no
 * formula.  Here the slowdown is a fixed rate: while both transfers run,
 * each progresses at rate_num / rate_den of its full speed
 * (1 <= rate_num <= rate_den <= 1024; rate_num == rate_den is the plain
 * model).  Time stays on whole nanoseconds: a transfer of d ns is
 * d * rate_den units of work, moving rate_den units per ns alone and
 * rate_num overlapped, and ends at the first whole ns by which its work is
 * done.  Kernels never slow down; with one DMA engine transfers never
 * overlap, so such groups get the plain model.  Every time the model can
 * reach stays below the sum of the kernels and of the transfers stretched by
 * rate_den / rate_num (rounded up); a group where that sum passes INT32_MAX
 * is rejected with TM_EOVERFLOW.  Arguments otherwise as the plain forms. */
int tm_predict_overlap(const tm_task* tasks, int n, const int32_t* order,
                       const tm_device* dev, int32_t rate_num, int32_t rate_den,
                       int32_t* makespan);
int tm_predict_overlap_batch(const tm_task* tasks, const int32_t* offsets, int G,
                             const int32_t* orders, const tm_device* devs,
                             int32_t rate_num, int32_t rate_den, int32_t* makespans);
int tm_predict_overlap_batch_dev(const tm_task* d_tasks, const int32_t* d_offsets,
                                 int G, const int32_t* d_orders,
                                 const tm_device* d_devs, int32_t rate_num,
                                 int32_t rate_den, int32_t* d_makespans,
                                 int32_t* d_status /* may be NULL */, void* stream);

/* Exhaustive search under the partial-overlap rule (n <= 12): every order is
 * simulated (the max-plus shortcut of the plain search does not apply), a
 * thread walking consecutive ranks.  Same tm_stats as tm_exhaustive_batch.
 * The _dev form takes the HOST copy of the offsets too, and uses working
 * memory owned by the library per host thread: calls from one host thread
 * must not overlap on the GPU (use one stream). */
int tm_exhaustive_overlap_batch(const tm_task* tasks, const int32_t* offsets, int G,
                                const tm_device* devs, int32_t rate_num,
                                int32_t rate_den, tm_stats* stats);
int tm_exhaustive_overlap_batch_dev(const tm_task* d_tasks, const int32_t* d_offsets,
                                    const int32_t* h_offsets, int G,
                                    const tm_device* d_devs, int32_t rate_num,
                                    int32_t rate_den, tm_stats* d_stats,
                                    int32_t* d_status /* may be NULL */, void* stream);

/* ---- learned order ranker and beam search --------------------------------- */

/* The paper has no learned component and no search beyond its O(n^2)
 * heuristic (Sec. 5.1); exhaustive search (above) stops at n = 12.  For
 * groups up to TM_MAX_TASKS (16) the library also offers a beam search whose
 * proposals come from a small learned ranker, the exact model (Sec. 4.1)
 * judging every order it returns.
 *
 * THE RANKER.  A 4-layer perceptron, 32 -> 128 -> 128 -> 128 -> 1 with ReLU,
 * scores "append task j next" from 32 features of task j, of the engine
 * times (end of the last HtD, K and DtH, Sec. 4.1) after the placed prefix
 * and of the tasks still unplaced, times scaled by n / (sum of the group's
 * durations).  Weights and activations are bfloat16 with float32
 * accumulation; the master parameters are float32, trained with Adam on the
 * softmax cross-entropy of each state's candidates against the task that a
 * reference order (normally the exhaustive best order) places there.
 * Parameters: one float32 vector of TM_RANKER_PARAMS values, laid out
 *   W1 [32 x 128] (row-major, input x output), b1 [128], W2 [128 x 128],
 *   b2 [128], W3 [128 x 128], b3 [128], w4 [128], b4 [1].
 * Feature rows are bfloat16 bit patterns (uint16_t), TM_RANKER_FEATURES per
 * row.  A ranker lives on the device that was current at creation; calls
 * with another device current return TM_EINVAL.  One ranker must not be
 * used by two calls that can run at the same time (it owns the scratch of
 * its training and beam calls, grown on demand with cudaMalloc). */
#define TM_RANKER_FEATURES 32
#define TM_RANKER_PARAMS 37377
#define TM_BEAM_MAX_WIDTH 64
#define TM_BEAM_MAX_REFINE_STARTS 8

typedef struct tm_ranker tm_ranker;

/* Allocates a ranker with He-uniform weights drawn by SplitMix64 from
 * `seed` (zero biases, zero Adam moments).  Synchronous. */
int tm_ranker_create(uint64_t seed, tm_ranker** ranker_out);
void tm_ranker_destroy(tm_ranker* ranker);

/* Copies the TM_RANKER_PARAMS float32 parameters out / in (host arrays;
 * synchronous: waits for the device).  set_params also resets the Adam
 * moments and step count. */
int tm_ranker_get_params(const tm_ranker* ranker, float* h_params);
int tm_ranker_set_params(tm_ranker* ranker, const float* h_params);

/* Scoring (tm_ranker_forward_dev, the beam search) runs on the tcgen05
 * tensor cores; every wait inside that kernel is bounded.  *count receives 1
 * if such a wait has ever expired for this ranker (the affected scores are
 * NaN), else 0.  Synchronous. */
int tm_ranker_errors(const tm_ranker* ranker, int32_t* count);

/* Training rows of a batch (host offsets): a group of n >= 2 tasks has
 * n - 1 states (positions p = 0 .. n - 2) with n - p candidate rows each,
 * n (n + 1) / 2 - 1 rows in all; n = 1 has none.  TM_EINVAL for bad
 * offsets, TM_ECAPACITY when rows would pass INT32_MAX - 16. */
int tm_ranker_rows_count(const int32_t* h_offsets, int G, int64_t* rows,
                         int32_t* states);

/* Builds the training rows of every group along its reference order:
 * d_orders (task layout, as tm_predict_batch_dev) or, if d_orders is NULL,
 * the best_order of d_stats[G] (from tm_exhaustive_batch_dev).  rows and
 * states must be tm_ranker_rows_count's values for these offsets.
 * Outputs: d_X [ceil16(rows) x 32] (rows past `rows` are zeroed),
 * d_state_off [states + 1] (state s owns rows d_state_off[s] ..
 * d_state_off[s + 1]), d_target [states] (the row of the placed task).
 * Candidates of a state come in ascending task index.  A group that fails
 * its input check, or whose order is not a permutation, gets zero rows and
 * its code in d_status (may be NULL).  Stream-ordered. */
int tm_ranker_rows_dev(tm_ranker* ranker, const tm_task* d_tasks,
                       const int32_t* d_offsets, int G, const tm_device* d_devs,
                       const int32_t* d_orders, const tm_stats* d_stats,
                       int64_t rows, int32_t states, uint16_t* d_X,
                       int32_t* d_state_off, int32_t* d_target,
                       int32_t* d_status, void* stream);

/* Scores rows: d_logits[rows] from d_X [rows x 32] (d_X 16-byte aligned,
 * else TM_EINVAL).  Stream-ordered. */
int tm_ranker_forward_dev(tm_ranker* ranker, const uint16_t* d_X, int64_t rows,
                          float* d_logits, void* stream);

/* Loss (mean over states of the softmax cross-entropy) and its gradient with
 * respect to the parameters, kept in the ranker for tm_ranker_adam_dev and
 * copied to d_grad [TM_RANKER_PARAMS] / d_loss [1] when those are not NULL.
 * d_X must be 16-byte aligned and hold ceil16(rows) rows whose tail past
 * `rows` is zero (as tm_ranker_rows_dev leaves it).  Stream-ordered. */
int tm_ranker_grad_dev(tm_ranker* ranker, const uint16_t* d_X, int64_t rows,
                       const int32_t* d_state_off, const int32_t* d_target,
                       int32_t states, float* d_grad, float* d_loss, void* stream);

/* The forward pass with its hidden layers kept, for tests and inspection:
 * the logits of `rows` feature rows as tm_ranker_forward_dev, and the
 * bfloat16 activations a1, a2, a3 (bit patterns) in d_acts [3 x rows x 128],
 * layer-major, row-major within a layer.  path 0: the tensor-core scoring
 * kernel of tm_ranker_forward_dev; path 1: the forward kernel of training
 * (tm_ranker_grad_dev).  d_X and d_acts 16-byte aligned.  Stream-ordered. */
int tm_ranker_forward_keep_dev(tm_ranker* ranker, const uint16_t* d_X, int64_t rows,
                               float* d_logits, uint16_t* d_acts, int path, void* stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) with learning rate lr
 * on the gradient of the last tm_ranker_grad_dev.  Stream-ordered. */
int tm_ranker_adam_dev(tm_ranker* ranker, float lr, void* stream);

/* Beam search over orders for every group (1 <= n <= 16; h_offsets is the
 * HOST copy of d_offsets).  Position by position, every live beam proposes
 * each unplaced task, the ranker scores the proposals, and the beam_width
 * (1 .. TM_BEAM_MAX_WIDTH) best by summed log-softmax score survive (ties:
 * lower beam, then lower task index); each beam carries the exact int32
 * engine times of its prefix.
 * refine_starts = 0: the result is the finished beam with the smallest
 * makespan if it beats the heuristic's order (tm_heuristic_batch_dev, run
 * first), else the heuristic's order.
 * refine_starts = K in 1 .. TM_BEAM_MAX_REFINE_STARTS: the K finished beams
 * of smallest makespan (ties: lower beam) and the heuristic's order each
 * start the exact-model descent of tm_refine_batch_dev, and the smallest
 * result wins (ties: the better-ranked start, the heuristic's last).
 * Either way the result is never worse than the heuristic and its makespan
 * is the model's exact value.  Writes d_orders_out (task layout),
 * d_makespans_out [G] (may be NULL), d_status [G] (may be NULL) and
 * d_beam_won [G] (may be NULL; 1 where the result came from a beam).
 * Stream-ordered. */
int tm_beam_batch_dev(tm_ranker* ranker, const tm_task* d_tasks,
                      const int32_t* d_offsets, const int32_t* h_offsets, int G,
                      const tm_device* d_devs, int beam_width, int refine_starts,
                      int32_t* d_orders_out, int32_t* d_makespans_out,
                      int32_t* d_status, int32_t* d_beam_won, void* stream);

/* Exact-model descent from the caller's orders (no counterpart in the paper;
 * it polishes the orders of the heuristic, Sec. 5.1, or of the beam
 * search).  For every group (1 <= n <= TM_MAX_TASKS) it repeatedly applies
 * the single move that lowers the makespan of the model (Sec. 4.1) the most
 * -- a swap of two positions, or one task moved to another position at
 * least two away -- until no move lowers it, or after 64 moves.  Ties go to
 * the first move in this order: swaps (i, j), i < j, by j then i; then
 * moves of the task at i to position j, by max(i, j), then i, then j.
 * d_orders (task layout, a permutation of 0 .. n - 1 per group) is read and
 * overwritten with the result; d_makespans [G] (may be NULL) receives its
 * makespan; d_status [G] (may be NULL) receives 0 or the group's error
 * (TM_EINVAL for an order that is not a permutation, and the input errors
 * of tm_predict; the group's order is then left as it was).
 * Stream-ordered. */
int tm_refine_batch_dev(const tm_task* d_tasks, const int32_t* d_offsets, int G,
                        const tm_device* d_devs, int32_t* d_orders,
                        int32_t* d_makespans, int32_t* d_status, void* stream);

/* ---- serving ---------------------------------------------------------------- */

/* A scheduling server for task groups that arrive one at a time (the paper
 * schedules each group as it is submitted to the device, Sec. 5.1; it has no
 * serving system).  A host worker thread gathers every waiting group into a
 * batch as soon as a lane of the right kind is free (continuous batching)
 * and runs it on that lane's CUDA stream.  Exact lanes give groups of
 * n <= exact_max_n the exhaustive optimum (first best order, as
 * tm_exhaustive_batch_dev); search lanes give larger groups the beam search
 * with `ranker` (tm_beam_batch_dev, with refine_starts) if beam_width > 0, else the heuristic
 * (tm_heuristic_batch_dev).  The two kinds run side by side, so a small
 * group never waits behind a long search.  A group's result does not depend
 * on the other groups of its batch.
 *
 * Memory: each lane owns fixed device and pinned host memory sized by the
 * config at creation; a batch takes at most lane_groups groups, lane_tasks
 * tasks and (exact lanes) lane_subsets 4-task subsets (C(n, 4) per group),
 * and a group waits on the host until a lane of its kind has room (first
 * come, first served within a kind).  Serving itself allocates nothing.
 *
 * Threads: submit / poll / replay may be called from any host thread; the
 * server runs on the device current at creation.  Results are delivered
 * once, to whichever poll (or the replay that submitted them) takes them. */
typedef struct tm_server tm_server;

typedef struct tm_server_config {
    int32_t lanes;          /* lanes of each kind (batches in flight), 1..8 (0: 2) */
    int32_t lane_groups;    /* groups per batch (0: 1024) */
    int32_t lane_tasks;     /* tasks per batch, >= 16 (0: 16 x lane_groups) */
    int32_t lane_subsets;   /* 4-task subsets per batch, >= 495 (0: 210 x lane_groups) */
    int32_t exact_max_n;    /* 0..12: groups up to this size are solved exactly */
    int32_t beam_width;     /* 0..64; 0: heuristic for the larger groups */
    tm_tuning tuning;       /* exhaustive-search knobs (fuse_finalize must not be 1) */
    int32_t refine_starts;  /* 0..TM_BEAM_MAX_REFINE_STARTS: as tm_beam_batch_dev */
} tm_server_config;

#define TM_METHOD_EXHAUSTIVE 0
#define TM_METHOD_BEAM 1
#define TM_METHOD_HEURISTIC 2

/* One scheduled group.  96 bytes. */
typedef struct tm_server_result {
    uint64_t ticket;        /* as returned by tm_server_submit */
    int32_t status;         /* TM_OK or the group's error code */
    int32_t n;
    int32_t makespan;       /* of `order`, by the model of Sec. 4.1 */
    int32_t method;         /* TM_METHOD_*: which search produced `order` */
    int64_t latency_ns;     /* submission (replay: scheduled arrival) to the
                               result being on the host */
    int32_t order[16];      /* task indices; entries past n are -1 */
} tm_server_result;

/* Creates a server and starts its worker thread.  ranker may be NULL when
 * beam_width is 0; it must outlive the server and must not be trained while
 * the server runs. */
int tm_server_create(const tm_server_config* config, const tm_ranker* ranker,
                     tm_server** server_out);

/* Queues one group (host pointers, copied before returning).  Input errors
 * (n outside 1..16, dma_engines, negative durations, sum above INT32_MAX)
 * are returned at once and the group is not queued. */
int tm_server_submit(tm_server* server, const tm_task* tasks, int n,
                     const tm_device* dev, uint64_t* ticket_out);

/* Takes up to max finished results, waiting up to wait_us microseconds for
 * the first one; *count receives how many were written. */
int tm_server_poll(tm_server* server, tm_server_result* out, int max, int wait_us,
                   int* count);

/* Open-loop load: submits group g of the batch (host arrays as in
 * tm_heuristic_batch) at arrival_ns[g] (nondecreasing) after the call
 * starts, from the calling thread, and returns when all G results are in
 * out[g].  Latencies are counted from the scheduled arrival times. */
int tm_server_replay(tm_server* server, const tm_task* tasks,
                     const int32_t* offsets, int G, const tm_device* devs,
                     const int64_t* arrival_ns, tm_server_result* out);

/* Batches launched, groups completed, and the largest batch so far (any
 * pointer may be NULL). */
int tm_server_counters(const tm_server* server, int64_t* batches,
                       int64_t* completed, int64_t* max_batch_groups);

/* Finishes every queued group, stops the worker and frees the server.
 * Results not yet polled are dropped. */
void tm_server_destroy(tm_server* server);

/* ---- misc ---------------------------------------------------------------- */

/* Measured int32 issue rates of this device, in operations per second:
 * independent chains of int32 maxima (max_per_s), additions (add_per_s) and
 * max-then-add recurrence steps k = max(k, h) + K counted as two operations
 * (max_add_per_s), every SM busy.  These are the operations the exhaustive
 * search's inner loop is made of (the FIFO recurrence of the model,
 * Sec. 4.1), so they bound it from above.  Runs 12 short kernels (about
 * 10 ms in all) on the legacy default stream and synchronises.  TM_EINVAL
 * for a NULL pointer, TM_ECUDA / TM_ENOMEM on CUDA failures. */
int tm_measure_int32_rates(double* max_per_s, double* add_per_s, double* max_add_per_s);


const char* tm_strerror(int code);

/* Library version, e.g. "tm 0.1 sm_103a". */
const char* tm_version(void);

#ifdef __cplusplus
}
#endif
#endif /* TM_H */

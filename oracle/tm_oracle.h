/*
 * tm_oracle.h -- plain, slow CPU oracle for the temporal execution model of
 * Lazaro-Munoz et al., "Improving tasks throughput on accelerators using
 * OpenCL command concurrency" (arXiv 1806.10113).
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists to check the CUDA path.
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load it.  It shares no code, header, table or helper with the CUDA
 * library; the two agree only because both follow the paper.
 *
 * Everything here is int64 so that the oracle itself cannot overflow; the
 * CUDA path is int32 and must reproduce these values exactly.
 */
#ifndef TM_ORACLE_H
#define TM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* One task: durations of its HtD transfer, kernel and DtH transfer (Sec. 4.1:
 * a task is the three stages HtD-K-DtH executed in order).  A stage that is
 * null, or made of several commands, is given as one summed duration. */
typedef struct orc_task {
    int32_t htd, k, dth;
} orc_task;

typedef struct orc_stats {
    int64_t best, worst;        /* min / max makespan over all n! orders      */
    int64_t sum;                /* exact sum of the n! makespans              */
    double mean;                /* (double)sum / (double)n!                   */
    uint64_t best_rank;         /* lexicographic rank of the FIRST best order */
    uint64_t worst_rank;        /* lexicographic rank of the FIRST worst      */
    int32_t best_order[16];
    int32_t worst_order[16];
} orc_stats;

/* Event-driven simulation of one order (Sec. 4.1, Figs. 4 and 6).
 * dma_engines = 2: three FIFOs (HtD, K, DtH).  dma_engines = 1: one DMA FIFO
 * holding every HtD in order and then every DtH in order, plus the K FIFO
 * (Sec. 3.2, Fig. 2).  `timeline`, if not NULL, receives 6*n int64 values:
 * for position i of the order, {start,end} of HtD, K, DtH at
 * timeline[6*i + 0..5].  Returns 0, or -1 on bad arguments. */
int orc_predict(const orc_task* tasks, int n, const int32_t* order,
                int dma_engines, int64_t* makespan, int64_t* timeline);

/* All n! orders, enumerated lexicographically from the identity (Sec. 1: the
 * brute-force search over N! orders).  n in [1, 12]. */
int orc_exhaustive(const orc_task* tasks, int n, int dma_engines,
                   orc_stats* out);

/* Ragged batch of groups: group g owns tasks[offsets[g] .. offsets[g+1]).
 * Work (groups x first-position subtrees) is spread over `nthreads` host
 * threads (<= 0: all hardware threads).  Results are identical to calling
 * orc_exhaustive per group. */
int orc_exhaustive_batch(const orc_task* tasks, const int32_t* offsets, int G,
                         const int32_t* dma_engines, int nthreads,
                         orc_stats* out);

/* Bounded samples for timing: item i enumerates, lexicographically, every
 * order of group item_group[i] that starts with the `plen` tasks
 * item_prefix[plen*i .. plen*i+plen) (distinct, in range).  out[i] holds
 * that subtree's best / worst / sum (ranks are global lexicographic ranks;
 * mean is sum / (n - plen)!).  Items run on `nthreads` host threads. */
int orc_exhaustive_prefixes(const orc_task* tasks, const int32_t* offsets,
                            const int32_t* dma_engines, const int32_t* item_group,
                            const int32_t* item_prefix, int plen, int nitems,
                            int nthreads, orc_stats* out);

/* Batch Reordering heuristic (Sec. 5.1, Algorithm 1) under the readings
 * H1-H5 documented in tm_oracle.cpp.  n in [1, 16].  Writes the order and
 * its simulated makespan. */
int orc_heuristic(const orc_task* tasks, int n, int dma_engines,
                  int32_t* order_out, int64_t* makespan_out);

int orc_heuristic_batch(const orc_task* tasks, const int32_t* offsets, int G,
                        const int32_t* dma_engines, int nthreads,
                        int32_t* orders_out, int64_t* makespans_out);

/* The partial-overlap variant of the model (Sec. 4.2.1; no formula in the
 * paper, so PARITY UNPINNED beyond the properties its tests check): an HtD
 * and a DtH transfer running together each progress at rate_num / rate_den
 * of full speed (1 <= rate_num <= rate_den); running transfers' end times
 * are re-estimated whenever that changes; ends are rounded up to whole ns.
 * rate_num == rate_den is the ideal model.  Same arguments otherwise as
 * orc_predict / orc_exhaustive (n <= 12). */
int orc_predict_overlap(const orc_task* tasks, int n, const int32_t* order,
                        int dma_engines, int32_t rate_num, int32_t rate_den,
                        int64_t* makespan, int64_t* timeline);
int orc_exhaustive_overlap(const orc_task* tasks, int n, int dma_engines,
                           int32_t rate_num, int32_t rate_den, orc_stats* out);

/* Chained tasks (Sec. 6.1, experiment setup): T = `workers` workers each
 * submit a chain of N = `rounds` dependent tasks, run as N rounds in
 * sequence (round r: the r-th task of every worker, in some order), so a
 * group has (T!)^N orders.  tasks[r * T + w] is worker w's task of round r;
 * seq lists the n = T * N task indices in run order, round 0's block first
 * (each block a permutation of its round's indices).  The HtD of a worker's
 * round-r task waits for the end of the DtH of its round-(r - 1) task.  One
 * DMA engine: the transfer FIFO holds each round's HtDs then its DtHs, round
 * after round.  1 <= T <= 8, T * N <= 16.  The exhaustive search enumerates
 * the (T!)^N orders lexicographically (the rounds as the digits of a
 * counter, round 0 most significant); ties go to the lowest rank;
 * mean = (double)sum / (double)(T!)^N; best_order / worst_order hold the
 * sequence.  Returns 0, or -1 on bad arguments. */
int orc_predict_chain(const orc_task* tasks, int workers, int rounds, const int32_t* seq,
                      int dma_engines, int64_t* makespan, int64_t* timeline);
int orc_exhaustive_chain(const orc_task* tasks, int workers, int rounds, int dma_engines,
                         orc_stats* out);
int orc_exhaustive_chain_batch(const orc_task* tasks, const int32_t* offsets,
                               const int32_t* workers, int G, const int32_t* dma_engines,
                               int nthreads, orc_stats* out);

/* Number of hardware threads the batch calls use when nthreads <= 0. */
int orc_hardware_threads(void);

#ifdef __cplusplus
}
#endif
#endif

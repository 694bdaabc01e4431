"""Chained tasks (Sec. 6.1 experiment setup) on the GPU against the oracle,
through the C ABI.  Makespans, sums, ranks and orders are integers and must
match exactly; the mean is the same IEEE expression on both sides."""
import math
import os
import random

import numpy as np
import pytest

import oracle
from paper_1806_10113_gb300 import build as tmbuild
from paper_1806_10113_gb300 import inputs
from tests.bruteforce import all_chain_orders

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SHAPES = [(1, 1), (1, 5), (2, 1), (2, 2), (2, 3), (3, 2), (3, 3), (4, 1), (4, 2), (4, 3), (2, 8),
          (5, 2), (3, 5), (6, 2), (4, 4), (5, 3), (8, 1), (7, 1)]


@pytest.fixture(scope="module")
def tm():
    tmbuild.build()
    from paper_1806_10113_gb300 import tm as tmmod
    return tmmod


def chain_batch(seed, shapes, hi=None):
    rng = random.Random(seed)
    groups, workers = [], []
    for T, R in shapes:
        h = hi or rng.choice([9, 20_000, 3_000_000])
        groups.append([[rng.randint(0, h) for _ in range(3)] for _ in range(T * R)])
        workers.append(T)
    b = inputs.make_batch(groups, [2 if g % 2 == 0 else 1 for g in range(len(groups))])
    return b, np.asarray(workers, dtype=np.int32)


def unrank_chain(rank, T, R):
    F = math.factorial(T)
    digits = []
    for _ in range(R):
        digits.append(rank % F)
        rank //= F
    order = []
    for r, q in enumerate(reversed(digits)):
        rest = list(range(T))
        for i in range(T):
            f = math.factorial(T - 1 - i)
            order.append(r * T + rest.pop(q // f))
            q %= f
    return order


def assert_stats_equal(gpu, orc, where=""):
    for k in ("best", "worst", "sum", "best_rank", "worst_rank", "best_order", "worst_order"):
        assert gpu[k] == orc[k], (where, k, gpu[k], orc[k])
    assert gpu["mean"] == orc["mean"], (where, gpu["mean"], orc["mean"])


def test_chain_worked_example(tm):
    unit = 1_000_000
    t = inputs.table2_tasks(["T0", "T7", "T5", "T4"], unit)
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "chain_T2_R2_worked.txt"))
            if ln.strip() and not ln.startswith("#")]
    for row in rows:
        dma = int(row[1])
        if row[0] == "order":
            assert tm.tm_predict_chain(t, 2, [int(x) for x in row[2].split(",")], dma) == \
                int(row[3]) * unit
        else:
            s = tm.tm_exhaustive_chain(t, 2, dma)
            best, brank, worst, wrank, total = map(int, row[2:])
            assert (s["best"], s["best_rank"], s["worst"], s["worst_rank"], s["sum"]) == \
                (best * unit, brank, worst * unit, wrank, total * unit)


def test_chain_predict_matches_oracle(tm):
    import torch
    rng = random.Random(5)
    shapes = SHAPES * 4 + [(8, 2)] * 4
    b, workers = chain_batch(6, shapes)
    orders = []
    for T, R in shapes:
        o = []
        for r in range(R):
            p = list(range(T))
            rng.shuffle(p)
            o += [r * T + w for w in p]
        orders += o
    dev = torch.device("cuda")
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    ms = torch.zeros(b.G, dtype=torch.int32, device=dev)
    status = torch.full((b.G,), 99, dtype=torch.int32, device=dev)
    tm.tm_predict_chain_batch_dev(d(b.tasks), d(b.offsets), d(workers), b.G,
                                  d(np.asarray(orders, dtype=np.int32)), d(b.dma), ms, status)
    torch.cuda.synchronize()
    assert (status.cpu().numpy() == 0).all()
    got = ms.cpu().numpy()
    for g in range(b.G):
        o0, o1 = int(b.offsets[g]), int(b.offsets[g + 1])
        want = oracle.predict_chain(b.group(g), int(workers[g]), orders[o0:o1], int(b.dma[g]))
        assert got[g] == want, g


def test_chain_exhaustive_matches_oracle(tm):
    """Every order of groups of every shape up to 1.7M orders, both models,
    three duration scales, one ragged batch."""
    b, workers = chain_batch(8, SHAPES * 2)
    got = tm.stats_to_dicts(tm.tm_exhaustive_chain_batch(b.tasks, b.offsets, workers, b.dma),
                            b.sizes())
    ref = oracle.exhaustive_chain_batch(b.tasks, b.offsets, workers, b.dma)
    for g in range(b.G):
        assert_stats_equal(got[g], ref[g], (g, int(workers[g])))


def test_chain_ties_pick_first_rank(tm):
    """Zero-length transfers: every order takes the kernel sum (first ranks
    0); small integer durations: many ties."""
    for T, R in ((3, 2), (4, 3), (2, 4)):
        t = np.asarray([[0, 7, 0]] * (T * R), dtype=np.int32)
        for dma in (1, 2):
            s = tm.tm_exhaustive_chain(t, T, dma)
            assert s["best"] == s["worst"] == 7 * T * R and s["best_rank"] == 0
            assert s["worst_rank"] == 0 and s["sum"] == 7 * T * R * math.factorial(T) ** R
    b, workers = chain_batch(12, [(3, 3), (4, 2), (2, 5), (5, 2)] * 3, hi=3)
    got = tm.stats_to_dicts(tm.tm_exhaustive_chain_batch(b.tasks, b.offsets, workers, b.dma),
                            b.sizes())
    ref = oracle.exhaustive_chain_batch(b.tasks, b.offsets, workers, b.dma)
    for g in range(b.G):
        assert_stats_equal(got[g], ref[g], g)


def test_chain_large_groups_sampled(tm):
    """8 workers x 2 rounds (1.6e9 orders) and 7 x 2: every reported order
    re-evaluated by the oracle, a sample of ranks bounded by best and worst."""
    b, workers = chain_batch(14, [(8, 2), (8, 2), (7, 2)], hi=2_000_000)
    got = tm.stats_to_dicts(tm.tm_exhaustive_chain_batch(b.tasks, b.offsets, workers, b.dma),
                            b.sizes())
    rng = random.Random(3)
    for g in range(b.G):
        T = int(workers[g])
        R = int(b.sizes()[g]) // T
        t, dma, s = b.group(g), int(b.dma[g]), got[g]
        count = math.factorial(T) ** R
        assert s["best_order"] == unrank_chain(s["best_rank"], T, R)
        assert s["worst_order"] == unrank_chain(s["worst_rank"], T, R)
        assert oracle.predict_chain(t, T, s["best_order"], dma) == s["best"]
        assert oracle.predict_chain(t, T, s["worst_order"], dma) == s["worst"]
        assert s["mean"] == float(s["sum"]) / float(count)
        assert s["best"] * count <= s["sum"] <= s["worst"] * count
        for _ in range(200):
            r = rng.randrange(count)
            ms = oracle.predict_chain(t, T, unrank_chain(r, T, R), dma)
            assert s["best"] <= ms <= s["worst"]
            assert ms != s["best"] or r >= s["best_rank"]
            assert ms != s["worst"] or r >= s["worst_rank"]


def test_chain_unrank_matches_enumeration():
    """The test's own unranking against the enumeration order of the brute
    force (no GPU; used by the sampled test above)."""
    for T, R in ((2, 2), (3, 2), (2, 3)):
        for r, o in enumerate(all_chain_orders(T, R)):
            assert unrank_chain(r, T, R) == list(o)


def test_chain_workload_groups(tm):
    """The benchmark's chained workload (4 workers x 4 rounds, mixed
    profiles, engines alternating): 96 groups enumerated by the oracle too."""
    b = inputs.chained_groups(groups=96, workers=4, rounds=4, seed=7)
    w = b.meta["workers"]
    got = tm.stats_to_dicts(tm.tm_exhaustive_chain_batch(b.tasks, b.offsets, w, b.dma), b.sizes())
    ref = oracle.exhaustive_chain_batch(b.tasks, b.offsets, w, b.dma)
    for g in range(b.G):
        assert_stats_equal(got[g], ref[g], g)


def test_chain_closed_form_counts_and_parity(tm):
    """Four-worker tails in the closed form of the HtD engine's path: none
    where kernels dominate under two DMA engines (the K engine runs ahead of
    the HtD engine; with one engine the round starts after the last DtH, so
    the HtD engine's path can end every order there too, and only parity is
    checked); all where only the last round's HtDs are long and every
    earlier task ends with its HtD (K = D = 0, so no release time and no
    engine gets ahead of the HtD engine), under both models; some on the
    mixed workload.  Every case equals the oracle's enumeration, and
    tm_chain_tail_counts counts 24^(R-1) tails per group."""
    rng = random.Random(31)

    def kernels(r, R):
        return [rng.randint(1, 9), rng.randint(10**6, 2 * 10**6), rng.randint(1, 9)]

    def htd_last(r, R):
        if r < R - 1:
            return [rng.randint(1, 9), 0, 0]
        return [rng.randint(10**6, 2 * 10**6), rng.randint(0, 9), 0]

    for name, mk, dma in (("kernels", kernels, [2, 2, 2, 2]), ("kernels1", kernels, [1, 1, 1, 1]),
                          ("htd_last", htd_last, [2, 1, 2, 1])):
        for R in (2, 3, 4):
            groups = [[mk(i // 4, R) for i in range(4 * R)] for _ in range(4)]
            b = inputs.make_batch(groups, dma)
            w = np.full(b.G, 4, dtype=np.int32)
            got = tm.stats_to_dicts(tm.tm_exhaustive_chain_batch(b.tasks, b.offsets, w, b.dma),
                                    b.sizes())
            tails, closed = tm.tm_chain_tail_counts()
            assert tails == b.G * 24 ** (R - 1), (name, R)
            if name == "kernels":
                assert closed == 0, (R, closed)
            elif name == "htd_last":
                assert closed == tails, (R, closed, tails)
            ref = oracle.exhaustive_chain_batch(b.tasks, b.offsets, w, b.dma)
            for g in range(b.G):
                assert_stats_equal(got[g], ref[g], (name, R, g))
    # the benchmark's shape (4 x 4: 576 units of 576 orders per group, so a
    # warp's lanes walk one group at a time): the one-DMA groups' tails close
    b = inputs.chained_groups(groups=24, workers=4, rounds=4, seed=9)
    w = b.meta["workers"]
    got = tm.stats_to_dicts(tm.tm_exhaustive_chain_batch(b.tasks, b.offsets, w, b.dma), b.sizes())
    tails, closed = tm.tm_chain_tail_counts()
    assert tails == b.G * 24 ** 3 and 0 < closed < tails
    ref = oracle.exhaustive_chain_batch(b.tasks, b.offsets, w, b.dma)
    for g in range(b.G):
        assert_stats_equal(got[g], ref[g], g)


def test_chain_dev_reports_bad_groups(tm):
    import torch
    b, workers = chain_batch(16, [(3, 2), (4, 2), (2, 3)], hi=1000)
    tasks = b.tasks.copy()
    tasks[b.offsets[2] + 1, 0] = -1                 # negative duration in group 2
    workers = workers.copy()
    workers[1] = 3                                  # 8 tasks, 3 workers: bad shape
    dev = torch.device("cuda")
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    st = torch.zeros(b.G * tm.STATS_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    status = torch.full((b.G,), 99, dtype=torch.int32, device=dev)
    tm.tm_exhaustive_chain_batch_dev(d(tasks), d(b.offsets), b.offsets, d(workers), workers,
                                     d(b.dma), st, status)
    torch.cuda.synchronize()
    assert list(status.cpu().numpy()) == [0, -1, -2]
    got = tm.stats_to_dicts(st.cpu().numpy().view(tm.STATS_DTYPE), b.sizes())[0]
    assert_stats_equal(got, oracle.exhaustive_chain(b.group(0), 3, int(b.dma[0])))
    with pytest.raises(tm.TMError):
        tm.tm_exhaustive_chain_batch(tasks, b.offsets, workers, b.dma)

"""Pins of the oracle's chained-task model (Sec. 6.1, experiment setup).

T workers each submit a chain of N dependent tasks; the group runs as N
rounds of T tasks, so it has (T!)^N orders.  None of these checks re-types
the oracle's event simulation: they use a case worked by hand, the plain
model (pinned on its own) where the chained one must reduce to it, the
order count, bounds that the chain dependency forces, time reversal, and the
independent unit-time brute force.
"""
import math
import os
import random

import numpy as np
import pytest

import oracle
from paper_1806_10113_gb300 import inputs
from tests.bruteforce import all_chain_orders, stepped_total_time

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rand_chain(rng, workers, rounds, lo=0, hi=2_000_000):
    return np.asarray([[rng.randint(lo, hi) for _ in range(3)]
                       for _ in range(workers * rounds)], dtype=np.int32)


def round_order(order, workers, r):
    """Round r's block of a chained order, as indices into that round's tasks."""
    return [int(t) - r * workers for t in order[r * workers:(r + 1) * workers]]


def test_worked_example_by_hand():
    unit = 1_000_000
    t = inputs.table2_tasks(["T0", "T7", "T5", "T4"], unit)
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "chain_T2_R2_worked.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 10
    for row in rows:
        dma = int(row[1])
        if row[0] == "order":
            order = [int(x) for x in row[2].split(",")]
            assert oracle.predict_chain(t, 2, order, dma) == int(row[3]) * unit
            assert stepped_total_time(inputs.table2_tasks(["T0", "T7", "T5", "T4"], 1), order,
                                      dma, workers=2) == int(row[3])
        else:
            s = oracle.exhaustive_chain(t, 2, dma)
            best, brank, worst, wrank, total = map(int, row[2:])
            assert (s["best"], s["best_rank"], s["worst"], s["worst_rank"], s["sum"]) == \
                (best * unit, brank, worst * unit, wrank, total * unit)
            assert s["mean"] == total * unit / 4
            assert s["best_order"] == list(all_chain_orders(2, 2)[brank])


@pytest.mark.parametrize("dma", [1, 2])
def test_one_round_is_the_plain_model(dma):
    """N = 1: no chain dependency, one group of T tasks."""
    rng = random.Random(3 + dma)
    for _ in range(12):
        T = rng.randint(1, 7)
        t = rand_chain(rng, T, 1)
        assert oracle.exhaustive_chain(t, T, dma) == oracle.exhaustive(t, dma)


def test_one_dma_engine_runs_the_rounds_one_after_another():
    """With one DMA engine a round's transfers queue behind every DtH of the
    round before, whose kernels have ended too: the total is the sum of the
    rounds' plain one-engine totals, and the search is a product of the
    rounds' searches (first best = the first best of every round)."""
    rng = random.Random(5)
    for _ in range(10):
        T, R = rng.choice([(2, 3), (3, 2), (3, 3), (4, 2), (2, 4)])
        t = rand_chain(rng, T, R)
        rounds = [t[r * T:(r + 1) * T] for r in range(R)]
        orders = all_chain_orders(T, R)
        for o in rng.sample(orders, min(20, len(orders))):
            want = sum(oracle.predict(rounds[r], round_order(o, T, r), 1) for r in range(R))
            assert oracle.predict_chain(t, T, o, 1) == want
        s = oracle.exhaustive_chain(t, T, 1)
        per = [oracle.exhaustive(x, 1) for x in rounds]
        f = math.factorial(T)
        assert s["best"] == sum(p["best"] for p in per)
        assert s["worst"] == sum(p["worst"] for p in per)
        assert s["sum"] == sum(p["sum"] for p in per) * f ** (R - 1)
        assert s["best_rank"] == sum(p["best_rank"] * f ** (R - 1 - r) for r, p in enumerate(per))
        assert s["worst_rank"] == sum(p["worst_rank"] * f ** (R - 1 - r)
                                      for r, p in enumerate(per))


@pytest.mark.parametrize("dma", [1, 2])
def test_order_count_is_t_factorial_to_the_n(dma):
    """With every transfer of zero length the kernels run back to back (each
    chain link is then a kernel waiting for an earlier kernel of the same
    FIFO), so every order takes the sum of the kernels and the sum over the
    search counts the orders: (T!)^N of them."""
    rng = random.Random(7 + dma)
    for T, R in ((2, 2), (3, 2), (2, 4), (4, 2), (3, 3), (1, 5), (5, 2)):
        t = np.asarray([[0, rng.randint(1, 99), 0] for _ in range(T * R)], dtype=np.int32)
        total_k = int(t[:, 1].sum())
        s = oracle.exhaustive_chain(t, T, dma)
        assert s["best"] == s["worst"] == total_k
        assert s["sum"] == total_k * math.factorial(T) ** R
        assert s["mean"] == total_k
        assert s["best_rank"] == 0 and s["worst_rank"] == 0


@pytest.mark.parametrize("dma", [1, 2])
def test_chain_bounds(dma):
    """Each worker's chain runs its tasks one after another, so no order beats
    the longest chain; no order beats the unchained model of the same
    sequence (a dependency can only delay); nothing exceeds the serial sum."""
    rng = random.Random(11 + dma)
    for _ in range(12):
        T, R = rng.choice([(2, 2), (3, 2), (2, 3), (4, 2), (3, 3)])
        t = rand_chain(rng, T, R, hi=rng.choice([9, 1000, 3_000_000]))
        chain_len = max(sum(int(t[r * T + w].sum()) for r in range(R)) for w in range(T))
        for o in all_chain_orders(T, R)[::7]:
            ms = oracle.predict_chain(t, T, o, dma)
            assert chain_len <= ms <= int(t.sum())
            if dma == 2:
                assert ms >= oracle.predict(t, list(o), 2)


def test_two_dma_reversibility():
    """Reversing time turns HtD into DtH, reverses every queue and turns each
    chain link (a DtH before the next round's HtD) into a link of the same
    kind between the reversed rounds, so the longest path is unchanged."""
    rng = random.Random(17)
    for _ in range(12):
        T, R = rng.choice([(2, 2), (3, 2), (2, 3), (4, 2)])
        t = rand_chain(rng, T, R)
        rev = np.empty_like(t)
        for r in range(R):
            for w in range(T):
                h, k, d = t[r * T + w]
                rev[(R - 1 - r) * T + w] = (d, k, h)
        for o in all_chain_orders(T, R)[::5]:
            # reversed run order; task (r, w) becomes task (R - 1 - r, w)
            ro = [(R - 1 - int(x) // T) * T + int(x) % T for x in reversed(o)]
            assert oracle.predict_chain(t, T, o, 2) == oracle.predict_chain(rev, T, ro, 2)


@pytest.mark.parametrize("dma", [1, 2])
def test_monotone_in_every_duration(dma):
    rng = random.Random(23 + dma)
    for _ in range(10):
        T, R = rng.choice([(2, 2), (3, 2), (2, 3)])
        t = rand_chain(rng, T, R, hi=1000)
        o = rng.choice(all_chain_orders(T, R))
        base = oracle.predict_chain(t, T, o, dma)
        i, s = rng.randrange(T * R), rng.randrange(3)
        t2 = t.copy()
        t2[i, s] += rng.randint(1, 500)
        assert oracle.predict_chain(t2, T, o, dma) >= base


@pytest.mark.parametrize("dma", [1, 2])
def test_matches_unit_time_bruteforce(dma):
    """Every order of small chained groups against the unit-time simulator,
    and the exhaustive statistics against enumeration with it."""
    for seed in range(14):
        rng = random.Random(300 + seed)
        T, R = [(2, 2), (3, 2), (2, 3), (3, 3), (4, 2), (2, 4), (1, 3)][seed % 7]
        t = rand_chain(rng, T, R, 0, 6)
        orders = all_chain_orders(T, R)
        ms = [stepped_total_time(t, o, dma, workers=T) for o in orders]
        for o, m in zip(orders[::3], ms[::3]):
            assert oracle.predict_chain(t, T, o, dma) == m
        s = oracle.exhaustive_chain(t, T, dma)
        assert s["best"] == min(ms) and s["worst"] == max(ms) and s["sum"] == sum(ms)
        assert s["best_rank"] == ms.index(min(ms)) and s["worst_rank"] == ms.index(max(ms))
        assert tuple(s["best_order"]) == orders[s["best_rank"]]
        assert tuple(s["worst_order"]) == orders[s["worst_rank"]]


def test_batch_equals_single_calls():
    rng = random.Random(29)
    shapes = [(2, 2), (3, 2), (4, 1), (2, 3), (1, 1), (3, 3)]
    groups = [rand_chain(rng, T, R) for T, R in shapes]
    b = inputs.make_batch(groups, [2, 1, 2, 1, 2, 2])
    workers = [T for T, _ in shapes]
    per = [oracle.exhaustive_chain(groups[g], workers[g], int(b.dma[g])) for g in range(b.G)]
    for nthreads in (1, 3, 0):
        assert oracle.exhaustive_chain_batch(b.tasks, b.offsets, workers, b.dma, nthreads) == per


def test_invalid_chains_rejected():
    t = np.ones((4, 3), dtype=np.int32)
    with pytest.raises(ValueError):
        oracle.predict_chain(t, 2, [0, 2, 1, 3], 2)        # a task outside its round
    with pytest.raises(ValueError):
        oracle.predict_chain(t, 2, [0, 0, 2, 3], 2)
    with pytest.raises(ValueError):
        oracle.exhaustive_chain(np.ones((6, 3), dtype=np.int32), 4, 2)   # 6 tasks, 4 workers
    with pytest.raises(ValueError):
        oracle.exhaustive_chain(np.ones((18, 3), dtype=np.int32), 9, 2)  # more than 16 tasks

"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these checks re-types the oracle's event-driven simulation.  They use
closed forms (one task; identical tasks), textbook results (Johnson's rule for
two-machine flow shops and its three-machine special case), bounds,
invariants (reversibility, monotonicity), hand-derived values for three of the
paper's Table 2 tasks, and an independent unit-time brute-force simulation.
"""
import itertools
import os
import random

import numpy as np
import pytest

import oracle
from paper_1806_10113_gb300 import inputs
from tests.bruteforce import all_orders, stepped_total_time

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rand_tasks(rng, n, lo=0, hi=2_000_000, zero_stage=None):
    t = [[rng.randint(lo, hi) for _ in range(3)] for _ in range(n)]
    if zero_stage is not None:
        for row in t:
            row[zero_stage] = 0
    return np.asarray(t, dtype=np.int32)


def all_makespans(tasks, dma):
    return [oracle.predict(tasks, o, dma) for o in all_orders(len(tasks))]


# ---- closed forms -------------------------------------------------------------

@pytest.mark.parametrize("dma", [1, 2])
def test_single_task_is_sum_of_stages(dma):
    rng = random.Random(11)
    for _ in range(50):
        t = rand_tasks(rng, 1)
        assert oracle.predict(t, [0], dma) == int(t[0].sum())


def test_identical_tasks_closed_form():
    """n identical tasks (H, K, D): a flow shop of identical jobs finishes at
    H + K + D + (n - 1) * max(H, K, D).  With one DMA engine the transfer
    queue also carries n*H + n*D back to back, so the total is the larger of
    that and the two-engine value."""
    rng = random.Random(12)
    for _ in range(40):
        n = rng.randint(1, 6)
        h, k, d = (rng.randint(0, 1000) for _ in range(3))
        t = np.asarray([[h, k, d]] * n, dtype=np.int32)
        two = h + k + d + (n - 1) * max(h, k, d)
        one = max(n * (h + d), two)
        assert set(all_makespans(t, 2)) == {two}
        assert set(all_makespans(t, 1)) == {one}
        for dma, v in ((2, two), (1, one)):
            s = oracle.exhaustive(t, dma)
            assert s["best"] == s["worst"] == v and s["mean"] == v
            assert s["best_rank"] == 0 and s["worst_rank"] == 0


def test_one_dma_without_kernels_is_order_invariant():
    """With one DMA engine and K = 0 the transfer queue is the bottleneck:
    every order takes sum(HtD) + sum(DtH)."""
    rng = random.Random(13)
    for _ in range(20):
        t = rand_tasks(rng, rng.randint(1, 6), zero_stage=1)
        expect = int(t[:, 0].sum() + t[:, 2].sum())
        assert set(all_makespans(t, 1)) == {expect}


# ---- Johnson's rule -----------------------------------------------------------

def johnson_order(a, b):
    """Johnson (1954): jobs with a <= b first by ascending a, then the rest by
    descending b (ties by index)."""
    first = sorted([j for j in range(len(a)) if a[j] <= b[j]], key=lambda j: (a[j], j))
    last = sorted([j for j in range(len(a)) if a[j] > b[j]], key=lambda j: (-b[j], j))
    return first + last


def two_machine_makespan(a, b, order):
    c1 = c2 = 0
    for j in order:
        c1 += a[j]
        c2 = max(c2, c1) + b[j]
    return c2


@pytest.mark.parametrize("zero_stage,machines", [(1, (0, 2)), (0, (1, 2)), (2, (0, 1))])
def test_two_dma_with_a_null_stage_is_johnson_optimal(zero_stage, machines):
    """With one stage null everywhere the two-engine model is a two-machine
    flow shop on the other two stages, where Johnson's rule is optimal."""
    rng = random.Random(20 + zero_stage)
    for _ in range(25):
        n = rng.randint(2, 7)
        t = rand_tasks(rng, n, zero_stage=zero_stage)
        a, b = t[:, machines[0]].tolist(), t[:, machines[1]].tolist()
        j = johnson_order(a, b)
        s = oracle.exhaustive(t, 2)
        assert s["best"] == two_machine_makespan(a, b, j)
        assert oracle.predict(t, j, 2) == s["best"]


def test_three_machine_johnson_special_case():
    """Johnson's three-machine case: if min HtD >= max K or min DtH >= max K,
    Johnson's rule on (HtD + K, K + DtH) gives an optimal order."""
    rng = random.Random(31)
    for trial in range(30):
        n = rng.randint(2, 7)
        kmax = rng.randint(0, 500)
        k = [rng.randint(0, kmax) for _ in range(n)]
        if trial % 2 == 0:
            h = [rng.randint(kmax, 3000) for _ in range(n)]
            d = [rng.randint(0, 3000) for _ in range(n)]
        else:
            h = [rng.randint(0, 3000) for _ in range(n)]
            d = [rng.randint(kmax, 3000) for _ in range(n)]
        t = np.asarray(list(zip(h, k, d)), dtype=np.int32)
        j = johnson_order([h[i] + k[i] for i in range(n)], [k[i] + d[i] for i in range(n)])
        assert oracle.predict(t, j, 2) == oracle.exhaustive(t, 2)["best"]


# ---- bounds and invariants ----------------------------------------------------

def lower_bound(t, dma):
    H, K, D = (t[:, i].astype(np.int64) for i in range(3))
    lbs = [H.sum() + (K + D).min(), H.min() + K.sum() + D.min(), (H + K + D).max()]
    if dma == 2:
        lbs.append((H + K).min() + D.sum())
    else:
        lbs.append(H.sum() + D.sum())
    return int(max(lbs))


@pytest.mark.parametrize("dma", [1, 2])
def test_every_order_between_engine_bound_and_serial_sum(dma):
    rng = random.Random(40 + dma)
    for _ in range(30):
        t = rand_tasks(rng, rng.randint(1, 6))
        lb, ub = lower_bound(t, dma), int(t.astype(np.int64).sum())
        for m in all_makespans(t, dma):
            assert lb <= m <= ub


def test_two_dma_reversibility():
    """A flow shop run backwards: order reversed and HtD/DtH swapped gives
    the same total time."""
    rng = random.Random(50)
    for _ in range(40):
        n = rng.randint(1, 6)
        t = rand_tasks(rng, n)
        rev = t[:, ::-1].copy()
        for o in all_orders(n):
            assert oracle.predict(t, o, 2) == oracle.predict(rev, o[::-1], 2)


@pytest.mark.parametrize("dma", [1, 2])
def test_monotone_in_every_duration(dma):
    rng = random.Random(60 + dma)
    for _ in range(30):
        n = rng.randint(1, 5)
        t = rand_tasks(rng, n, hi=1000)
        base = all_makespans(t, dma)
        t2 = t.copy()
        t2[rng.randrange(n), rng.randrange(3)] += rng.randint(1, 500)
        assert all(b2 >= b for b, b2 in zip(base, all_makespans(t2, dma)))


def test_one_dma_never_faster_than_two():
    rng = random.Random(70)
    for _ in range(30):
        t = rand_tasks(rng, rng.randint(1, 6))
        assert all(a >= b for a, b in zip(all_makespans(t, 1), all_makespans(t, 2)))


def test_one_dma_timeline_respects_single_transfer_queue():
    """Fig. 4a: no DtH starts before the last HtD has finished, transfers never
    overlap, and each stage starts after the previous stage of its task."""
    rng = random.Random(80)
    for _ in range(30):
        n = rng.randint(1, 7)
        t = rand_tasks(rng, n)
        order = list(range(n))
        rng.shuffle(order)
        ms, tl = oracle.predict(t, order, 1, timeline=True)
        last_htd_end = tl[:, 0, 1].max()
        assert (tl[:, 2, 0] >= last_htd_end).all()
        transfers = sorted([tuple(tl[i, 0]) for i in range(n)] + [tuple(tl[i, 2]) for i in range(n)])
        assert all(a[1] <= b[0] for a, b in zip(transfers, transfers[1:]))
        assert (tl[:, 1, 0] >= tl[:, 0, 1]).all() and (tl[:, 2, 0] >= tl[:, 1, 1]).all()
        assert ms == tl[:, :, 1].max()


# ---- brute force and worked values ---------------------------------------------

@pytest.mark.parametrize("dma", [1, 2])
def test_matches_unit_time_bruteforce(dma):
    for seed in range(25):
        n = 1 + seed % 5
        t = inputs.random_small(seed, n, 0, 6).tasks
        for o in all_orders(n):
            assert oracle.predict(t, o, dma) == stepped_total_time(t, o, dma), (seed, o)


@pytest.mark.parametrize("dma", [1, 2])
def test_exhaustive_stats_match_bruteforce(dma):
    for seed in range(20):
        n = 1 + seed % 6
        t = inputs.random_small(100 + seed, n, 0, 5).tasks
        ms = [stepped_total_time(t, o, dma) for o in all_orders(n)]
        s = oracle.exhaustive(t, dma)
        assert s["best"] == min(ms) and s["worst"] == max(ms) and s["sum"] == sum(ms)
        assert s["best_rank"] == ms.index(min(ms)) and s["worst_rank"] == ms.index(max(ms))
        assert tuple(s["best_order"]) == all_orders(n)[s["best_rank"]]
        assert tuple(s["worst_order"]) == all_orders(n)[s["worst_rank"]]
        assert s["mean"] == float(sum(ms)) / float(len(ms))


def read_worked_example():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "worked_example_T0_T7_T5.txt"))
            if ln.strip() and not ln.startswith("#")]
    return rows


def test_worked_example_by_hand():
    unit = 1_000_000
    t3 = inputs.table2_tasks(["T0", "T7", "T5"], unit)
    for row in read_worked_example():
        kind, dma = row[0], int(row[1])
        if kind in ("order", "pair"):
            order = [int(x) for x in row[2].split(",")]
            tasks = t3 if kind == "order" else t3[:2]
            assert oracle.predict(tasks, order, dma) == int(row[3]) * unit
            assert stepped_total_time(inputs.table2_tasks(["T0", "T7", "T5"], 1)[:len(order)],
                                      order, dma) == int(row[3])
        elif kind == "stats":
            s = oracle.exhaustive(t3, dma)
            best, brank, worst, wrank, total = map(int, row[2:])
            assert (s["best"], s["best_rank"], s["worst"], s["worst_rank"], s["sum"]) == \
                (best * unit, brank, worst * unit, wrank, total * unit)
            assert s["mean"] == total * unit / 6
        elif kind == "heuristic":
            order, ms = oracle.heuristic(t3, dma)
            assert order == [int(x) for x in row[2].split(",")] and ms == int(row[3]) * unit


def test_bk_tables_golden_and_bruteforce():
    """Every order of the paper's Table 3 benchmarks: the stored oracle values
    agree with the unit-time brute force."""
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "bk_table3_orders.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 5 * 2 * 24
    for bk, dma, order, ms in rows:
        tasks = inputs.table2_tasks(inputs.TABLE3[bk], unit_ns=1)
        order = [int(x) for x in order.split(",")]
        assert stepped_total_time(tasks, order, int(dma)) == int(ms)
        assert oracle.predict(tasks, order, int(dma)) == int(ms)


def test_exhaustive_batch_equals_single_calls():
    b = inputs.random_groups(5, [1, 2, 3, 5, 7, 4, 6], hi=3_000_000)
    per = [oracle.exhaustive(b.group(g), int(b.dma[g])) for g in range(b.G)]
    for nthreads in (1, 3, 0):
        assert oracle.exhaustive_batch(b.tasks, b.offsets, b.dma, nthreads) == per


def test_zero_durations_allowed():
    t = np.zeros((4, 3), dtype=np.int32)
    for dma in (1, 2):
        assert oracle.exhaustive(t, dma)["worst"] == 0


def test_invalid_inputs_rejected():
    t = np.asarray([[1, 2, 3], [4, 5, 6]], dtype=np.int32)
    with pytest.raises(ValueError):
        oracle.predict(t, [0, 0], 2)
    with pytest.raises(ValueError):
        oracle.predict(t, [0, 1], 3)
    with pytest.raises(ValueError):
        oracle.predict(np.asarray([[1, -1, 0]], dtype=np.int32), [0], 2)
    with pytest.raises(ValueError):
        oracle.exhaustive(np.zeros((13, 3), dtype=np.int32), 2)


# ---- heuristic: properties (the selection rules themselves are unpinned) -------

@pytest.mark.parametrize("dma", [1, 2])
def test_heuristic_properties(dma):
    rng = random.Random(90 + dma)
    for _ in range(60):
        n = rng.randint(1, 8)
        t = rand_tasks(rng, n, hi=rng.choice([10, 1000, 2_000_000]))
        order, ms = oracle.heuristic(t, dma)
        assert sorted(order) == list(range(n))
        assert ms == oracle.predict(t, order, dma)
        best = oracle.exhaustive(t, dma)["best"]
        assert ms >= best
        if n == 1:
            assert order == [0]
        if n == 2:
            assert ms == best
        if n >= 3:
            # H1: the first task has the largest K - HtD, then the longest DtH.
            key = [(int(r[1]) - int(r[0]), int(r[2]), -j) for j, r in enumerate(t)]
            assert order[0] == max(range(n), key=lambda j: key[j])
            # H4: the last two are in their better order.
            swapped = order[:-2] + [order[-1], order[-2]]
            assert ms <= oracle.predict(t, swapped, dma)
        if n >= 2:
            swapped = order[:-2] + [order[-1], order[-2]]
            if oracle.predict(t, swapped, dma) == ms:
                # H4 tie: the order ending with the shorter DtH, then lower index first.
                a, b = order[-2], order[-1]
                assert t[b, 2] < t[a, 2] or (t[b, 2] == t[a, 2] and a < b)


def test_heuristic_beats_mean_on_paper_benchmarks():
    """The paper reports that the heuristic always beats the mean order
    (Sec. 6.2).  It is expected, not guaranteed; on the paper's own Table 3
    benchmarks it holds for both device models."""
    for bk, names in inputs.TABLE3.items():
        t = inputs.table2_tasks(names, 1)
        for dma in (1, 2):
            _, ms = oracle.heuristic(t, dma)
            assert ms <= oracle.exhaustive(t, dma)["mean"], (bk, dma)


def test_prefix_samples_partition_the_exhaustive_search():
    """Subtrees under every one- and two-task prefix combine to the full
    search (same best / worst ranks, same sum)."""
    b = inputs.random_groups(9, [6, 5], hi=1000)
    for g in range(b.G):
        n = int(b.sizes()[g])
        full = oracle.exhaustive(b.group(g), int(b.dma[g]))
        for plen in (1, 2):
            prefixes = [p for p in itertools.permutations(range(n), plen)]
            parts = oracle.exhaustive_prefixes(b.tasks, b.offsets, b.dma, [g] * len(prefixes),
                                               prefixes)
            assert sum(p["sum"] for p in parts) == full["sum"]
            best = min(parts, key=lambda p: (p["best"], p["best_rank"]))
            worst = min(parts, key=lambda p: (-p["worst"], p["worst_rank"]))
            assert (best["best"], best["best_rank"]) == (full["best"], full["best_rank"])
            assert (worst["worst"], worst["worst_rank"]) == (full["worst"], full["worst_rank"])


# ---- heuristic: select_next_task worked by hand (H1-H4) -----------------------

def read_select_next_golden():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "heuristic_select_next_T2tasks.txt"))
            if ln.strip() and not ln.startswith("#")]
    groups = {r[1]: r[2].split(",") for r in rows if r[0] == "group"}
    return groups, [r for r in rows if r[0] != "group"]


def _ints(field):
    return [int(x) for x in field.split(",")]


def test_heuristic_select_next_worked_by_hand():
    """Algorithm 1 on three groups of Table 2 tasks, every step derived by hand
    (first task, each update() and each candidate's start and cost, both
    completions of the last two, the chosen order).  Groups A and B make
    select_next_task run twice, with a cost tie that the K rule settles and a
    candidate whose HtD ends after the kernel engine frees, so each plausible
    misreading of the cost or the tie rule changes the chosen order."""
    groups, rows = read_select_next_golden()
    unit = 1_000_000
    seen = set()
    for row in rows:
        kind, name, dma = row[0], row[1], int(row[2])
        ms_tasks = inputs.table2_tasks(groups[name], 1)
        ns_tasks = inputs.table2_tasks(groups[name], unit)
        seen.add((kind, name, dma))
        if kind == "first":
            order, _ = oracle.heuristic(ns_tasks, dma)
            assert order[0] == int(row[3])
        elif kind == "update":
            ot = _ints(row[3])
            sub = ns_tasks[ot]
            total, tl = oracle.predict(sub, list(range(len(ot))), dma, timeline=True)
            want = [int(x) for x in row[4:7]]
            # ends of the last HtD, K and DtH of OT simulated as the whole group
            assert [int(tl[-1, 0, 1]), int(tl[-1, 1, 1]), int(tl[-1, 2, 1])] == \
                [w * unit for w in want], (name, dma, ot)
            assert total == want[2] * unit
            assert stepped_total_time(ms_tasks[ot], list(range(len(ot))), dma) == want[2]
        elif kind == "complete":
            order = _ints(row[3])
            assert oracle.predict(ns_tasks, order, dma) == int(row[4]) * unit
            assert stepped_total_time(ms_tasks, order, dma) == int(row[4])
        elif kind == "heuristic":
            order, ms = oracle.heuristic(ns_tasks, dma)
            assert order == _ints(row[3]) and ms == int(row[4]) * unit, (name, dma, order)
            # the scale of the time unit changes nothing
            assert oracle.heuristic(ms_tasks, dma) == (_ints(row[3]), int(row[4]))
    # the stored candidate rows agree with the stored choices: at every step the
    # chosen task is the listed candidate of smallest cost, ties to larger K
    chosen = {(r[1], int(r[2])): _ints(r[3]) for r in rows if r[0] == "heuristic"}
    steps = {}
    for r in rows:
        if r[0] == "cand":
            steps.setdefault((r[1], int(r[2]), r[3]), []).append((int(r[4]), int(r[6])))
    for (name, dma, ot), cands in steps.items():
        k = {j: int(inputs.TABLE2_MS[groups[name][j]][1]) for j, _ in cands}
        pick = min(cands, key=lambda c: (c[1], -k[c[0]], c[0]))[0]
        prefix = _ints(ot)
        assert chosen[(name, dma)][:len(prefix) + 1] == prefix + [pick], (name, dma, ot)
    assert {(n, d) for _, n, d in seen} == {(n, d) for n in groups for d in (1, 2)}

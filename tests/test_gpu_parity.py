"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Makespans, sums, best / worst values and ranks are integers and must match
exactly; the mean is the same IEEE expression on both sides and must match
bit for bit.  The benchmark's workloads are checked in full where the oracle
finishes in seconds on the host cores: every order of the 64 groups of 10
tasks under both models, of all 8192 ragged groups, and of two complete
12-task groups; the remaining 12-task groups have every reported order and a
sample of ranks checked.
"""
import itertools
import math
import os
import random

import numpy as np
import pytest

import oracle
from paper_1806_10113_gb300 import build as tmbuild
from paper_1806_10113_gb300 import inputs

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def tm():
    tmbuild.build()
    from paper_1806_10113_gb300 import tm as tmmod
    return tmmod


def lex_rank(order):
    n, rank, rest = len(order), 0, sorted(order)
    for i, e in enumerate(order):
        c = rest.index(e)
        rank += c * math.factorial(n - 1 - i)
        rest.pop(c)
    return rank


def unrank(rank, n):
    rest, out = list(range(n)), []
    for i in range(n):
        f = math.factorial(n - 1 - i)
        out.append(rest.pop(rank // f))
        rank %= f
    return out


def assert_stats_equal(gpu, orc, where=""):
    for k in ("best", "worst", "sum", "best_rank", "worst_rank", "best_order", "worst_order"):
        assert gpu[k] == orc[k], (where, k, gpu[k], orc[k])
    assert gpu["mean"] == orc["mean"], (where, gpu["mean"], orc["mean"])


# ---- predict ----------------------------------------------------------------

def test_predict_paper_benchmarks_golden(tm):
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "bk_table3_orders.txt"))
            if ln.strip() and not ln.startswith("#")]
    for bk, dma, order, ms in rows:
        tasks = inputs.table2_tasks(inputs.TABLE3[bk], unit_ns=1_000_000)
        assert tm.tm_predict(tasks, [int(x) for x in order.split(",")], int(dma)) == \
            int(ms) * 1_000_000


def test_predict_ragged_random_vs_oracle(tm):
    rng = random.Random(3)
    sizes = [rng.randint(1, 16) for _ in range(300)] + [1, 16, 16]
    b = inputs.random_groups(3, sizes, hi=50_000_000)
    orders = []
    for g in range(b.G):
        o = list(range(sizes[g]))
        rng.shuffle(o)
        orders += o
    got = tm.tm_predict_batch(b.tasks, b.offsets, orders, b.dma)
    for g in range(b.G):
        o = orders[b.offsets[g]:b.offsets[g + 1]]
        assert got[g] == oracle.predict(b.group(g), o, int(b.dma[g])), g


# ---- exhaustive ---------------------------------------------------------------

@pytest.mark.parametrize("dma", [1, 2])
def test_exhaustive_every_size_up_to_8(tm, dma):
    for n in range(1, 9):
        for seed in range(4):
            t = inputs.random_groups(100 * n + seed, [n], hi=3_000_000).tasks
            assert_stats_equal(tm.tm_exhaustive(t, dma), oracle.exhaustive(t, dma), (n, seed))


@pytest.mark.parametrize("dma", [1, 2])
def test_exhaustive_ties_pick_first_rank(tm, dma):
    """Small integer durations and identical tasks make many orders tie; the
    first (lowest-rank) best and worst must still agree."""
    cases = [inputs.random_small(s, n, 0, 3).tasks for s, n in
             [(1, 5), (2, 6), (3, 7), (4, 8), (5, 9)]]
    cases += [np.tile(np.asarray([[5, 7, 3]], dtype=np.int32), (n, 1)) for n in (5, 8)]
    cases += [np.zeros((7, 3), dtype=np.int32)]
    for i, t in enumerate(cases):
        assert_stats_equal(tm.tm_exhaustive(t, dma), oracle.exhaustive(t, dma), i)


def test_exhaustive_ragged_batch_vs_oracle(tm):
    rng = random.Random(8)
    sizes = [rng.randint(1, 9) for _ in range(60)]
    b = inputs.random_groups(8, sizes, hi=4_000_000)
    got = tm.stats_to_dicts(tm.tm_exhaustive_batch(b.tasks, b.offsets, b.dma), sizes)
    ref = oracle.exhaustive_batch(b.tasks, b.offsets, b.dma)
    for g in range(b.G):
        assert_stats_equal(got[g], ref[g], g)


def test_exhaustive_small_case_six_tasks(tm):
    """One group of 6 tasks, durations U[50k, 2M] ns, seed 0, both models."""
    b = inputs.single_group_uniform(n=6, seed=0)
    for dma in (2, 1):
        assert_stats_equal(tm.tm_exhaustive(b.tasks, dma), oracle.exhaustive(b.tasks, dma))


def test_exhaustive_ten_tasks_full_oracle(tm):
    """Four groups of 10 tasks (DK and DT, both models), all 3,628,800 orders
    on both sides."""
    full = inputs.dk_dt_groups(groups=64, n=10, seed=1)
    pick = [0, 32, 64, 96]
    b = inputs.make_batch([full.group(g) for g in pick], full.dma[pick])
    got = tm.stats_to_dicts(tm.tm_exhaustive_batch(b.tasks, b.offsets, b.dma), b.sizes())
    ref = oracle.exhaustive_batch(b.tasks, b.offsets, b.dma)
    for g in range(b.G):
        assert_stats_equal(got[g], ref[g], g)


def check_reported_orders(tm, b, stats, samples=64, seed=0):
    """Every reported order and a sample of ranks, checked with the oracle."""
    rng = random.Random(seed)
    for g in range(b.G):
        t, n, dma, s = b.group(g), int(b.sizes()[g]), int(b.dma[g]), stats[g]
        assert s["best_order"] == unrank(s["best_rank"], n)
        assert s["worst_order"] == unrank(s["worst_rank"], n)
        assert oracle.predict(t, s["best_order"], dma) == s["best"]
        assert oracle.predict(t, s["worst_order"], dma) == s["worst"]
        nf = math.factorial(n)
        assert s["mean"] == float(s["sum"]) / float(nf)
        assert s["best"] * nf <= s["sum"] <= s["worst"] * nf
        for _ in range(samples):
            r = rng.randrange(nf)
            ms = oracle.predict(t, unrank(r, n), dma)
            assert s["best"] <= ms <= s["worst"]
            assert ms != s["best"] or r >= s["best_rank"]
            assert ms != s["worst"] or r >= s["worst_rank"]


def scheduled_as_benched(tm, b, tuning=None):
    """The whole scheduling pass (exhaustive search + heuristic) the way the
    benchmark runs it: tuning picked by the autotuner on this batch (or the
    one given), one tm_schedule_batch_dev call on device buffers."""
    import torch
    from paper_1806_10113_gb300 import autotune
    dev = torch.device("cuda")
    if tuning is None:
        tuning = autotune.tune(b.tasks, b.offsets, b.dma, cache_path=None, reps=10)
    plan = tm.Plan(b.offsets, **tuning)
    d_tasks = torch.from_numpy(b.tasks).to(dev)
    d_dma = torch.from_numpy(b.dma).to(dev)
    d_stats = torch.zeros(b.G * tm.STATS_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    d_orders = torch.full((b.tasks.shape[0],), -1, dtype=torch.int32, device=dev)
    d_ms = torch.zeros(b.G, dtype=torch.int32, device=dev)
    d_status = torch.full((b.G,), 99, dtype=torch.int32, device=dev)
    tm.tm_schedule_batch_dev(plan, d_tasks, d_dma, d_stats, d_orders, d_ms, d_status)
    torch.cuda.synchronize()
    plan.close()
    assert (d_status.cpu().numpy() == 0).all()
    stats = tm.stats_to_dicts(d_stats.cpu().numpy().view(tm.STATS_DTYPE), b.sizes())
    return stats, d_orders.cpu().numpy(), d_ms.cpu().numpy().astype(np.int64), tuning


def test_exhaustive_full_size_sixty_four_groups(tm):
    """The benchmark's workload and launch: 64 groups of 10 tasks (half DK,
    half DT) under both models, autotuned, one scheduling pass.  All 128 x
    10! orders are enumerated by the oracle too, and every statistic and
    every heuristic order must match."""
    b = inputs.dk_dt_groups(groups=64, n=10, seed=1)
    stats, orders, hms, tuning = scheduled_as_benched(tm, b)
    ref = oracle.exhaustive_batch(b.tasks, b.offsets, b.dma)
    for g in range(b.G):
        assert_stats_equal(stats[g], ref[g], (g, tuning))
    ref_orders, ref_ms = oracle.heuristic_batch(b.tasks, b.offsets, b.dma)
    assert (orders == ref_orders).all() and (hms == ref_ms).all()
    # the paper's heuristic can never beat the exhaustive best
    assert all(hms[g] >= stats[g]["best"] for g in range(b.G))


@pytest.mark.parametrize("workload,tuning", [
    ("dkdt64x10", dict(pdmax=5, fuse_finalize=2, unroll=5, item_cost=65536, chunks_per_thread=1)),
    ("dkdt64x10", dict(pdmax=4, unroll=5, chunks_per_thread=3)),
    ("ragged2048", dict(pdmax=5, fuse_finalize=2, blocks_per_sm=3, unroll=5, chunks_per_thread=3)),
    ("ties", dict(pdmax=5, unroll=5)),
    ("ties_uniform", dict(pdmax=5, fuse_finalize=2, unroll=5)),
    ("big_uniform", dict(pdmax=4, fuse_finalize=2, unroll=5)),
])
def test_dominance_walk_mode_full_oracle(tm, workload, tuning):
    """Walk modes 5 to 8 (closed forms for prefixes whose completions one
    engine's path ends; 6 with the suffix constants in shared memory and the
    six prefixes of a straight-line level evaluated together; 7 with their
    vote and closed forms in one pass; 7 and 8 with a rolled loop) against the
    oracle's full enumeration, whatever the tuner picks elsewhere: the
    benchmark's 64 x 10 workload (all 128 x 10! orders), 2048 ragged groups,
    and tie-heavy groups (durations 0..3, where every closed form meets equal
    makespans and the first rank decides), also as batches of one group size
    (the static split of whole warps), one of them with 24-order sums beyond
    32 bits (the DtH engine's case only)."""
    if workload == "dkdt64x10":
        b = inputs.dk_dt_groups(groups=64, n=10, seed=1)
    elif workload == "ragged2048":
        b = inputs.ragged_mixed(groups=2048, seed=4)
    elif workload == "ties":
        b = inputs.random_groups(26, [9, 10, 8, 9, 7, 10], lo=0, hi=3)
    elif workload == "ties_uniform":
        b = inputs.random_groups(27, [9] * 12, lo=0, hi=3)
    else:
        b = inputs.random_groups(28, [9] * 6, hi=60_000_000)
    ref = oracle.exhaustive_batch(b.tasks, b.offsets, b.dma)
    ref_orders, ref_ms = oracle.heuristic_batch(b.tasks, b.offsets, b.dma)
    for mode in (5, 6, 7, 8):
        t = dict(tuning, unroll=mode)
        stats, orders, hms, _ = scheduled_as_benched(tm, b, t)
        for g in range(b.G):
            assert_stats_equal(stats[g], ref[g], (g, t))
        assert (orders == ref_orders).all() and (hms == ref_ms).all()


def test_walk_counts(tm):
    """tm_plan_walk_counts: n!/24 prefixes per group; every prefix evaluated
    order by order outside walk modes 5 to 8; under them, some (the benchmark's
    dominant-transfer groups under two DMA engines mix the engines' paths)
    but not all; and none where the DtH engine's path ends every order."""
    import torch
    dev = torch.device("cuda")

    def run(b, unroll):
        plan = tm.Plan(b.offsets, pdmax=5, unroll=unroll)
        d_stats = torch.zeros(b.G * tm.STATS_DTYPE.itemsize, dtype=torch.uint8, device=dev)
        d_status = torch.full((b.G,), 9, dtype=torch.int32, device=dev)
        tm.tm_exhaustive_batch_dev(plan, torch.from_numpy(b.tasks).to(dev),
                                   torch.from_numpy(b.dma).to(dev), d_stats, d_status)
        torch.cuda.synchronize()
        assert (d_status.cpu().numpy() == 0).all()
        counts = plan.walk_counts()
        plan.close()
        return counts

    b = inputs.dk_dt_groups(groups=64, n=10, seed=1)
    pre3, full3 = run(b, 3)
    pre5, full5 = run(b, 5)
    assert pre3 == pre5 == 128 * math.factorial(10) // 24 and full3 == pre3
    assert 0 < full5 < pre5
    for mode in (6, 7, 8):
        pre6, full6 = run(b, mode)
        assert pre6 == pre5 and 0 < full6 < pre6
    dth = inputs.make_batch([[[1, 1, 1_000_000]] * 8] * 6, [2, 1] * 3)
    for mode in (5, 6, 7, 8):
        pre, full = run(dth, mode)
        assert pre == 6 * math.factorial(8) // 24 and full == 0


def oracle_full_by_prefixes(b, g):
    """Oracle statistics of group g from its two-task-prefix subtrees (all n!
    orders, spread evenly over the host cores)."""
    n = int(b.sizes()[g])
    prefixes = [p for p in itertools.permutations(range(n), 2)]
    parts = oracle.exhaustive_prefixes(b.tasks, b.offsets, b.dma, [g] * len(prefixes), prefixes)
    best = min(parts, key=lambda p: (p["best"], p["best_rank"]))
    worst = min(parts, key=lambda p: (-p["worst"], p["worst_rank"]))
    total = sum(p["sum"] for p in parts)
    return {"best": best["best"], "best_rank": best["best_rank"], "best_order": best["best_order"],
            "worst": worst["worst"], "worst_rank": worst["worst_rank"],
            "worst_order": worst["worst_order"], "sum": total,
            "mean": float(total) / float(math.factorial(n))}


def test_exhaustive_twelve_tasks_full_oracle(tm):
    """The 12-task workload (32 groups, half DK / half DT tasks, under 2 and 1
    DMA engines), autotuned and run as benched.  Two groups, one per device
    model, are enumerated completely by the oracle (2 x 479,001,600 orders);
    every other group's reported orders and a sample of ranks are checked."""
    b = inputs.half_dk_half_dt(groups=32, n=12, seed=3, models=(2, 1))
    stats, orders, hms, tuning = scheduled_as_benched(tm, b)
    for g in (0, 32 + 5):
        assert int(b.dma[g]) == (2 if g < 32 else 1)
        assert_stats_equal(stats[g], oracle_full_by_prefixes(b, g), (g, tuning))
    check_reported_orders(tm, b, stats, samples=16)
    ref_orders, ref_ms = oracle.heuristic_batch(b.tasks, b.offsets, b.dma)
    assert (orders == ref_orders).all() and (hms == ref_ms).all()


def test_ragged_8192_groups_full_oracle(tm):
    """The batched workload: 8192 ragged groups of 4..9 tasks, mixed profiles,
    engines alternating, autotuned and run as benched; every group's
    statistics and heuristic order against the oracle's full enumeration."""
    b = inputs.ragged_mixed(groups=8192, seed=2)
    stats, orders, hms, tuning = scheduled_as_benched(tm, b)
    ref = oracle.exhaustive_batch(b.tasks, b.offsets, b.dma)
    for g in range(b.G):
        assert_stats_equal(stats[g], ref[g], (g, tuning))
    ref_orders, ref_ms = oracle.heuristic_batch(b.tasks, b.offsets, b.dma)
    assert (orders == ref_orders).all() and (hms == ref_ms).all()


def test_exhaustive_duration_sum_at_int32_limit(tm):
    """The largest admissible group: durations sum to exactly INT32_MAX."""
    t = np.asarray([[300_000_000, 100_000_000, 200_000_000]] * 3 +
                   [[1, 0, 0], [50_000_000, 0, 0]], dtype=np.int64)
    t[-1, 1] += (2**31 - 1) - int(t.sum())
    assert int(t.sum()) == 2**31 - 1
    t = t.astype(np.int32)
    for dma in (1, 2):
        assert_stats_equal(tm.tm_exhaustive(t, dma), oracle.exhaustive(t, dma))
    t2 = t.copy()
    t2[0, 0] += 1
    with pytest.raises(tm.TMError) as e:
        tm.tm_exhaustive(t2, 2)
    assert e.value.code == -3


def test_plan_reuse_gives_identical_results(tm):
    b = inputs.random_groups(21, [5, 9, 7, 3, 8], hi=6_000_000)
    first = tm.tm_exhaustive_batch(b.tasks, b.offsets, b.dma)
    second = tm.tm_exhaustive_batch(b.tasks, b.offsets, b.dma)
    assert first.tobytes() == second.tobytes()


# ---- heuristic -------------------------------------------------------------------

@pytest.mark.parametrize("dma", [1, 2])
def test_heuristic_orders_match_oracle(tm, dma):
    rng = random.Random(40 + dma)
    sizes = [rng.randint(1, 16) for _ in range(400)] + list(range(1, 17))
    his = [rng.choice([5, 1000, 5_000_000]) for _ in sizes]
    groups = []
    for g, (n, hi) in enumerate(zip(sizes, his)):
        r = inputs.group_stream(777 + dma, g)
        groups.append([inputs.uniform_task(r, (0, hi), (0, hi), (0, hi)) for _ in range(n)])
    b = inputs.make_batch(groups, [dma] * len(groups))
    orders, ms = tm.tm_heuristic_batch(b.tasks, b.offsets, b.dma)
    ref_orders, ref_ms = oracle.heuristic_batch(b.tasks, b.offsets, b.dma)
    assert (orders == ref_orders).all()
    assert (ms.astype(np.int64) == ref_ms).all()


def test_heuristic_worked_example(tm):
    t3 = inputs.table2_tasks(["T0", "T7", "T5"], 1_000_000)
    assert tm.tm_heuristic(t3, 2) == ([0, 2, 1], 18_000_000)
    assert tm.tm_heuristic(t3, 1) == ([0, 2, 1], 19_000_000)


def test_heuristic_select_next_worked_by_hand(tm):
    """The hand-derived Algorithm 1 runs (select_next_task twice, a cost tie
    settled by K, an HtD ending after the kernel engine frees): the half-warp
    heuristic kernel and the full-warp heuristic inside the scheduling pass
    both give the stored orders."""
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "heuristic_select_next_T2tasks.txt"))
            if ln.strip() and not ln.startswith("#")]
    groups = {r[1]: r[2].split(",") for r in rows if r[0] == "group"}
    want = [(r[1], int(r[2]), [int(x) for x in r[3].split(",")], int(r[4]) * 1_000_000)
            for r in rows if r[0] == "heuristic"]
    assert len(want) == 6
    for name, dma, order, ms in want:
        assert tm.tm_heuristic(inputs.table2_tasks(groups[name]), dma) == (order, ms), (name, dma)
    b = inputs.make_batch([inputs.table2_tasks(groups[name]) for name, _, _, _ in want],
                          [dma for _, dma, _, _ in want])
    orders, ms = tm.tm_heuristic_batch(b.tasks, b.offsets, b.dma)
    _, orders2, ms2 = tm.tm_schedule_batch(b.tasks, b.offsets, b.dma)
    exp_orders = np.concatenate([np.asarray(o, dtype=np.int32) for _, _, o, _ in want])
    exp_ms = np.asarray([m for _, _, _, m in want])
    assert (orders == exp_orders).all() and (ms == exp_ms).all()
    assert (orders2 == exp_orders).all() and (ms2 == exp_ms).all()


# ---- the whole scheduling pass ----------------------------------------------------

def test_schedule_batch_matches_oracle_on_ragged_groups(tm):
    """Exhaustive search and heuristic in one call: groups of 1..10 tasks,
    both device models, small and large durations."""
    rng = random.Random(17)
    sizes = [rng.randint(1, 10) for _ in range(40)] + [1, 2, 3, 4, 10]
    b = inputs.random_groups(17, sizes, hi=3_000_000)
    st, orders, ms = tm.tm_schedule_batch(b.tasks, b.offsets, b.dma)
    got = tm.stats_to_dicts(st, b.sizes())
    ref = oracle.exhaustive_batch(b.tasks, b.offsets, b.dma)
    ref_orders, ref_ms = oracle.heuristic_batch(b.tasks, b.offsets, b.dma)
    for g in range(b.G):
        assert_stats_equal(got[g], ref[g], g)
    assert (orders == ref_orders).all() and (ms.astype(np.int64) == ref_ms).all()
    # repeated calls reuse the cached plan and its completion counters
    st2, orders2, ms2 = tm.tm_schedule_batch(b.tasks, b.offsets, b.dma)
    assert st2.tobytes() == st.tobytes() and (orders2 == orders).all()


@pytest.mark.parametrize("sizes,tuning", [
    ([6, 2, 9, 1, 5, 3, 8, 4], dict(fuse_finalize=2)),     # heuristic beside the finalize warps
    ([6, 2, 9, 1, 5, 3, 8, 4], dict(fuse_finalize=1)),     # no finalize launch: heuristic in prep
    ([3, 1, 2, 3, 2], dict(fuse_finalize=2)),              # no group of 4+: no enumeration at all
])
def test_heuristic_and_search_in_every_launch_layout(tm, sizes, tuning):
    """The heuristic's warps run in the finalize launch, or in the prep
    launch when there is no finalize launch; groups are laid out by size.
    Every output must land at the caller's index either way."""
    import torch
    dev = torch.device("cuda")
    b = inputs.random_groups(61, sizes, hi=4_000_000)
    plan = tm.Plan(b.offsets, **tuning)
    d_tasks = torch.from_numpy(b.tasks).to(dev)
    d_dma = torch.from_numpy(b.dma).to(dev)
    d_stats = torch.zeros(b.G * 72, dtype=torch.uint8, device=dev)
    d_orders = torch.full((b.tasks.shape[0],), -1, dtype=torch.int32, device=dev)
    d_ms = torch.zeros(b.G, dtype=torch.int32, device=dev)
    d_status = torch.full((b.G,), 99, dtype=torch.int32, device=dev)
    tm.tm_schedule_batch_dev(plan, d_tasks, d_dma, d_stats, d_orders, d_ms, d_status)
    torch.cuda.synchronize()
    assert (d_status.cpu().numpy() == 0).all()
    got = tm.stats_to_dicts(d_stats.cpu().numpy().view(tm.STATS_DTYPE), b.sizes())
    ref = oracle.exhaustive_batch(b.tasks, b.offsets, b.dma)
    ref_orders, ref_ms = oracle.heuristic_batch(b.tasks, b.offsets, b.dma)
    for g in range(b.G):
        assert_stats_equal(got[g], ref[g], g)
    assert (d_orders.cpu().numpy() == ref_orders).all()
    assert (d_ms.cpu().numpy().astype(np.int64) == ref_ms).all()
    plan.close()


def test_schedule_batch_dev_reports_invalid_groups(tm):
    import torch
    dev = torch.device("cuda")
    b = inputs.random_groups(58, [7, 3, 9, 5, 2, 8], hi=5_000_000)
    tasks = b.tasks.copy()
    tasks[b.offsets[2] + 4, 0] = -1                     # group 2: negative duration
    tasks[b.offsets[4], 2] = -7                         # group 4 (2 tasks): negative duration
    plan = tm.Plan(b.offsets)
    d_tasks = torch.from_numpy(tasks).to(dev)
    d_dma = torch.from_numpy(b.dma).to(dev)
    d_stats = torch.zeros(b.G * 72, dtype=torch.uint8, device=dev)
    d_orders = torch.zeros(b.tasks.shape[0], dtype=torch.int32, device=dev)
    d_ms = torch.zeros(b.G, dtype=torch.int32, device=dev)
    d_status = torch.full((b.G,), 99, dtype=torch.int32, device=dev)
    for _ in range(3):
        tm.tm_schedule_batch_dev(plan, d_tasks, d_dma, d_stats, d_orders, d_ms, d_status)
        torch.cuda.synchronize()
        assert list(d_status.cpu().numpy()) == [0, 0, -2, 0, -2, 0]
        got = tm.stats_to_dicts(d_stats.cpu().numpy().view(tm.STATS_DTYPE), b.sizes())
        orders = d_orders.cpu().numpy()
        for g in (0, 1, 3, 5):
            assert_stats_equal(got[g], oracle.exhaustive(b.group(g), int(b.dma[g])), g)
            o, m = oracle.heuristic(b.group(g), int(b.dma[g]))
            assert list(orders[b.offsets[g]:b.offsets[g + 1]]) == o and int(d_ms[g]) == m
    plan.close()


@pytest.mark.parametrize("tuning", [dict(pdmax=3), dict(pdmax=5),
                                    dict(fuse_finalize=1, chunks_per_thread=1),
                                    dict(pdmax=5, fuse_finalize=1, blocks_per_sm=2,
                                         chunks_per_thread=1),
                                    dict(pdmax=3, blocks_per_sm=1), dict(item_cost=1),
                                    dict(pdmax=4, item_cost=5000), dict(chunks_per_thread=1),
                                    dict(pdmax=3, chunks_per_thread=64),
                                    dict(chunks_per_thread=2, item_cost=1, blocks_per_sm=1),
                                    dict(unroll=1), dict(pdmax=3, unroll=1),
                                    dict(pdmax=5, unroll=1, chunks_per_thread=3),
                                    dict(pdmax=4, unroll=2, item_cost=1),
                                    dict(pdmax=5, unroll=3), dict(pdmax=3, unroll=3,
                                                                   chunks_per_thread=6),
                                    dict(pdmax=5, unroll=4), dict(pdmax=3, unroll=4),
                                    dict(pdmax=4, unroll=4, chunks_per_thread=3),
                                    dict(pdmax=5, unroll=5), dict(pdmax=3, unroll=5),
                                    dict(pdmax=4, unroll=5, chunks_per_thread=3),
                                    dict(pdmax=5, unroll=5, item_cost=1),
                                    dict(pdmax=5, unroll=6), dict(pdmax=3, unroll=6),
                                    dict(pdmax=4, unroll=6, chunks_per_thread=3),
                                    dict(pdmax=5, unroll=6, item_cost=1, blocks_per_sm=1),
                                    dict(pdmax=5, unroll=7), dict(pdmax=3, unroll=7),
                                    dict(pdmax=4, unroll=7, chunks_per_thread=3),
                                    dict(pdmax=5, unroll=8), dict(pdmax=3, unroll=8),
                                    dict(pdmax=4, unroll=8, chunks_per_thread=3)])
def test_every_tuning_gives_identical_results(tm, tuning):
    """Work split, prefix depth and finalize placement change no result."""
    import torch
    dev = torch.device("cuda")
    rng = random.Random(23)
    sizes = [rng.randint(1, 11) for _ in range(30)] + [4, 5, 9, 11]
    b = inputs.random_groups(23, sizes, hi=rng.choice([50, 4_000_000]))
    tie = inputs.random_groups(24, [9, 10, 8], lo=0, hi=3)        # many ties
    big = inputs.random_groups(25, [9, 8], hi=60_000_000)        # 24 makespans overflow 32 bits
    parts = (b, tie, big)
    b = inputs.make_batch([p.group(g) for p in parts for g in range(p.G)],
                          [int(x) for p in parts for x in p.dma])
    d_tasks = torch.from_numpy(b.tasks).to(dev)
    d_dma = torch.from_numpy(b.dma).to(dev)
    outs = []
    for tun in ({}, tuning):
        plan = tm.Plan(b.offsets, **tun)
        d_stats = torch.zeros(b.G * 72, dtype=torch.uint8, device=dev)
        d_status = torch.full((b.G,), 9, dtype=torch.int32, device=dev)
        for _ in range(2):
            tm.tm_exhaustive_batch_dev(plan, d_tasks, d_dma, d_stats, d_status)
        torch.cuda.synchronize()
        assert (d_status.cpu().numpy() == 0).all()
        outs.append(d_stats.cpu().numpy().tobytes())
        plan.close()
    assert outs[0] == outs[1]
    got = tm.stats_to_dicts(np.frombuffer(outs[1], dtype=tm.STATS_DTYPE), b.sizes())
    small = [g for g in range(b.G) if b.sizes()[g] <= 9]
    ref = oracle.exhaustive_batch(b.tasks, b.offsets, b.dma)
    for g in small:
        assert_stats_equal(got[g], ref[g], g)


def test_cuda_graph_replay_matches_direct_call(tm):
    import torch
    dev = torch.device("cuda")
    b = inputs.ragged_mixed(groups=300, seed=31)
    plan = tm.Plan(b.offsets)
    d_tasks = torch.from_numpy(b.tasks).to(dev)
    d_dma = torch.from_numpy(b.dma).to(dev)
    bufs = []
    for _ in range(2):
        bufs.append((torch.zeros(b.G * 72, dtype=torch.uint8, device=dev),
                     torch.zeros(b.tasks.shape[0], dtype=torch.int32, device=dev),
                     torch.zeros(b.G, dtype=torch.int32, device=dev),
                     torch.full((b.G,), 9, dtype=torch.int32, device=dev)))
    tm.tm_schedule_batch_dev(plan, d_tasks, d_dma, *bufs[0])
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(); e1.record()
    plan.set_timing(e0, e1)
    plan.capture(d_tasks, d_dma, *bufs[1])
    plan.set_timing(None, None)
    for _ in range(3):
        plan.graph_launch()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(); f1.record()
    plan.graph_set_timing(f0, f1)
    plan.graph_launch()
    torch.cuda.synchronize()
    assert f0.elapsed_time(f1) > 0
    for x, y in zip(bufs[0], bufs[1]):
        assert torch.equal(x, y)
    assert (bufs[1][3].cpu().numpy() == 0).all()
    ref = oracle.exhaustive_batch(b.tasks, b.offsets, b.dma)
    got = tm.stats_to_dicts(bufs[1][0].cpu().numpy().view(tm.STATS_DTYPE), b.sizes())
    for g in range(0, b.G, 7):
        assert_stats_equal(got[g], ref[g], g)
    plan.close()


# ---- device-pointer entry points ----------------------------------------------------

def test_dev_entry_points_and_status(tm):
    import torch
    dev = torch.device("cuda")
    b = inputs.random_groups(55, [6, 4, 9, 2, 7], hi=5_000_000)
    tasks = b.tasks.copy()
    tasks[b.offsets[1], 1] = -5                         # group 1: negative duration
    dma = b.dma.copy()
    dma[3] = 3                                          # group 3: bad model
    d_tasks = torch.from_numpy(tasks).to(dev)
    d_off = torch.from_numpy(b.offsets).to(dev)
    d_dma = torch.from_numpy(dma).to(dev)
    G = b.G
    plan = tm.Plan(b.offsets)
    d_stats = torch.zeros(G * 72, dtype=torch.uint8, device=dev)
    d_status = torch.full((G,), 99, dtype=torch.int32, device=dev)
    for _ in range(2):
        tm.tm_exhaustive_batch_dev(plan, d_tasks, d_dma, d_stats, d_status)
        torch.cuda.synchronize()
        st = d_stats.cpu().numpy().view(tm.STATS_DTYPE)
        status = d_status.cpu().numpy()
        assert list(status) == [0, -2, 0, -1, 0]
        got = tm.stats_to_dicts(st, b.sizes())
        for g in (0, 2, 4):
            assert_stats_equal(got[g], oracle.exhaustive(b.group(g), int(b.dma[g])), g)
    d_orders = torch.zeros(b.tasks.shape[0], dtype=torch.int32, device=dev)
    d_ms = torch.zeros(G, dtype=torch.int32, device=dev)
    tm.tm_heuristic_batch_dev(d_tasks, d_off, G, d_dma, d_orders, d_ms, d_status)
    torch.cuda.synchronize()
    assert list(d_status.cpu().numpy()) == [0, -2, 0, -1, 0]
    for g in (0, 2, 4):
        o, ms = oracle.heuristic(b.group(g), int(b.dma[g]))
        assert list(d_orders.cpu().numpy()[b.offsets[g]:b.offsets[g + 1]]) == o
        assert int(d_ms[g]) == ms
    ident = torch.from_numpy(np.concatenate([np.arange(n) for n in b.sizes()]).astype(np.int32))
    ident[0] = 1                                        # group 0: not a permutation
    tm.tm_predict_batch_dev(d_tasks, d_off, G, ident.to(dev), d_dma, d_ms, d_status)
    torch.cuda.synchronize()
    assert list(d_status.cpu().numpy()) == [-1, -2, 0, -1, 0]
    assert int(d_ms[2]) == oracle.predict(b.group(2), list(range(9)), int(b.dma[2]))
    plan.close()

"""GPU parity of the partial-overlap variant of the model (Sec. 4.2.1,
Fig. 6) against the oracle's event-driven simulation: bit-exact makespans,
exhaustive statistics and first best / worst orders."""
import itertools
import random

import numpy as np
import pytest

import oracle
from paper_1806_10113_gb300 import inputs, tm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RATES = [(1, 2), (2, 3), (3, 8), (5, 7), (1, 1024), (7, 7)]


def assert_stats(got, ref, g):
    for k in ("best", "worst", "sum", "best_rank", "worst_rank"):
        assert got[k] == ref[k], (g, k, got[k], ref[k])
    assert got["mean"] == ref["mean"], g
    assert got["best_order"] == ref["best_order"] and got["worst_order"] == ref["worst_order"], g


@pytest.mark.parametrize("rate", RATES)
def test_predict_matches_oracle(rate):
    num, den = rate
    sizes = list(range(1, 17)) * 4
    # keep 16 tasks with every transfer stretched by den / num below INT32_MAX
    hi = min(2_000_000, (2**31 - 1) // (16 * (2 * den // num + 1)))
    b = inputs.random_groups(31, sizes, hi=hi)
    rng = np.random.default_rng(7)
    orders = np.concatenate([rng.permutation(n) for n in b.sizes()]).astype(np.int32)
    got = tm.tm_predict_overlap_batch(b.tasks, b.offsets, orders, b.dma, num, den)
    for g in range(b.G):
        o = orders[b.offsets[g]:b.offsets[g + 1]]
        assert got[g] == oracle.predict_overlap(b.group(g), o, int(b.dma[g]), num, den), g


def test_predict_hand_cases_and_fig6():
    assert tm.tm_predict_overlap([[4, 2, 6], [8, 1, 1]], [0, 1], 2, 1, 2) == 20
    assert tm.tm_predict_overlap([[4, 2, 6], [8, 1, 1]], [0, 1], 2, 2, 5) == 23
    # Fig. 6 scenario at rate 3/8: DtH_0 ends at 220, then K_1 and DtH_1
    assert tm.tm_predict_overlap([[200, 7, 8], [10, 1, 1]], [0, 1], 2, 3, 8) == \
        oracle.predict_overlap([[200, 7, 8], [10, 1, 1]], [0, 1], 2, 3, 8)


def test_predict_dev_with_zero_stages_and_status():
    # zero-length stages, ties of simultaneous ends, and one bad group
    t = [[0, 5, 0], [3, 0, 3], [0, 0, 0], [6, 6, 6], [2, 9, 1]]
    groups = [t, t[:3], t[2:], [[1, -1, 1]], t[1:4]]
    b = inputs.make_batch(groups, [2, 2, 1, 2, 2])
    orders = np.concatenate([np.arange(len(x))[::-1] for x in groups]).astype(np.int32)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    ms = torch.zeros(b.G, dtype=torch.int32, device="cuda")
    st = torch.full((b.G,), 99, dtype=torch.int32, device="cuda")
    tm.tm_predict_overlap_batch_dev(dev(b.tasks), dev(b.offsets), b.G, dev(orders), dev(b.dma),
                                    2, 3, ms, st)
    torch.cuda.synchronize()
    ms, st = ms.cpu().numpy(), st.cpu().numpy()
    assert list(st) == [0, 0, 0, -2, 0]
    for g in (0, 1, 2, 4):
        o = orders[b.offsets[g]:b.offsets[g + 1]]
        assert ms[g] == oracle.predict_overlap(b.group(g), o, int(b.dma[g]), 2, 3), g


@pytest.mark.parametrize("rate", [(1, 2), (3, 8), (2, 3)])
def test_exhaustive_matches_oracle(rate):
    num, den = rate
    rng = random.Random(num * 100 + den)
    sizes = [rng.randint(1, 7) for _ in range(20)] + [8]
    b = inputs.random_groups(41 + num, sizes, hi=rng.choice([9, 3_000_000]))
    got = tm.stats_to_dicts(tm.tm_exhaustive_overlap_batch(b.tasks, b.offsets, b.dma, num, den),
                            b.sizes())
    for g in range(b.G):
        assert_stats(got[g], oracle.exhaustive_overlap(b.group(g), int(b.dma[g]), num, den), g)


def test_exhaustive_ties():
    # tiny durations: many orders share the best and the worst makespan
    b = inputs.random_groups(43, [6, 7, 5, 8], lo=0, hi=3)
    got = tm.stats_to_dicts(tm.tm_exhaustive_overlap_batch(b.tasks, b.offsets, b.dma, 1, 2),
                            b.sizes())
    for g in range(b.G):
        assert_stats(got[g], oracle.exhaustive_overlap(b.group(g), int(b.dma[g]), 1, 2), g)


def test_exhaustive_full_rate_equals_plain_search():
    b = inputs.random_groups(44, [9, 10, 4, 6, 10], hi=4_000_000)
    plain = tm.tm_exhaustive_batch(b.tasks, b.offsets, b.dma)
    full = tm.tm_exhaustive_overlap_batch(b.tasks, b.offsets, b.dma, 5, 5)
    assert plain.tobytes() == full.tobytes()


def test_exhaustive_dev_sampled_n10():
    # a 10-task group (3.6M simulated orders): statistics checked against the
    # oracle's simulation of the reported best / worst orders and a sample of
    # orders around them
    b = inputs.random_groups(45, [10, 10], hi=2_000_000, dma=[2, 2])
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    d_stats = torch.zeros(b.G * 72, dtype=torch.uint8, device="cuda")
    st = torch.full((b.G,), 99, dtype=torch.int32, device="cuda")
    tm.tm_exhaustive_overlap_batch_dev(dev(b.tasks), dev(b.offsets), b.offsets, dev(b.dma), 2, 3,
                                       d_stats, st)
    torch.cuda.synchronize()
    assert (st.cpu().numpy() == 0).all()
    got = tm.stats_to_dicts(d_stats.cpu().numpy().view(tm.STATS_DTYPE), b.sizes())
    rng = np.random.default_rng(3)
    for g in range(b.G):
        t = b.group(g)
        assert oracle.predict_overlap(t, got[g]["best_order"], 2, 2, 3) == got[g]["best"]
        assert oracle.predict_overlap(t, got[g]["worst_order"], 2, 2, 3) == got[g]["worst"]
        for _ in range(300):
            o = rng.permutation(10)
            m = oracle.predict_overlap(t, o, 2, 2, 3)
            assert got[g]["best"] <= m <= got[g]["worst"]
        assert got[g]["best"] * 3628800 <= got[g]["sum"] <= got[g]["worst"] * 3628800


def test_64bit_work_path():
    # durations of 3..5 ms at rate 1000/1024: a transfer's work (duration x
    # 1024 units) passes 2^31, so these groups take the 64-bit event loop
    b = inputs.random_groups(46, [5, 6, 7, 3], lo=3_000_000, hi=5_000_000)
    got = tm.stats_to_dicts(tm.tm_exhaustive_overlap_batch(b.tasks, b.offsets, b.dma, 1000, 1024),
                            b.sizes())
    for g in range(b.G):
        assert_stats(got[g], oracle.exhaustive_overlap(b.group(g), int(b.dma[g]), 1000, 1024), g)
    rng = np.random.default_rng(11)
    orders = np.concatenate([rng.permutation(n) for n in b.sizes()]).astype(np.int32)
    ms = tm.tm_predict_overlap_batch(b.tasks, b.offsets, orders, b.dma, 1000, 1024)
    for g in range(b.G):
        o = orders[b.offsets[g]:b.offsets[g + 1]]
        assert ms[g] == oracle.predict_overlap(b.group(g), o, int(b.dma[g]), 1000, 1024)


@pytest.mark.parametrize("rate", [(2, 3), (5, 9)])
def test_exhaustive_n9_every_order_against_predict(rate):
    """Every one of the 9! orders of two 9-task groups: the exhaustive
    search (each order resumed where it first differs from the one before,
    the tail after the last HtD in closed form) against the predict kernel,
    which simulates each order from time 0 and is itself checked against the
    oracle above."""
    num, den = rate
    b = inputs.random_groups(47 + num, [9, 9], hi=3_000_000, dma=[2, 2])
    got = tm.stats_to_dicts(tm.tm_exhaustive_overlap_batch(b.tasks, b.offsets, b.dma, num, den),
                            b.sizes())
    perms = np.array(list(itertools.permutations(range(9))), dtype=np.int32)   # lexicographic
    P = perms.shape[0]
    for g in range(b.G):
        t = b.group(g)
        tasks = np.tile(t, (P, 1)).astype(np.int32)
        offsets = (np.arange(P + 1) * 9).astype(np.int32)
        ms = tm.tm_predict_overlap_batch(tasks, offsets, perms.reshape(-1), np.full(P, 2, np.int32),
                                         num, den).astype(np.int64)
        assert got[g]["best"] == ms.min() and got[g]["worst"] == ms.max(), g
        assert got[g]["sum"] == ms.sum(), g
        assert got[g]["best_rank"] == int(np.argmax(ms == ms.min())), g
        assert got[g]["worst_rank"] == int(np.argmax(ms == ms.max())), g

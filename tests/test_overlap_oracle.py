"""Pins of the oracle's partial-overlap variant of the model (Sec. 4.2.1,
Fig. 6).  The paper gives no formula for the slowdown of concurrent HtD and
DtH transfers, so these check what any reading must satisfy, what the
reading taken here (a fixed rate rate_num / rate_den while both run, end
times re-estimated on each change, rounded up to whole ns) implies in cases
worked out by hand, and the two Fig. 6 numbers a single rate can reproduce."""
import itertools
import random

import numpy as np
import pytest

import oracle
from paper_1806_10113_gb300 import inputs


def rand_group(seed, n, hi=50):
    rng = random.Random(seed)
    return [[rng.randint(0, hi), rng.randint(0, hi), rng.randint(0, hi)] for _ in range(n)]


@pytest.mark.parametrize("dma", [1, 2])
def test_full_rate_is_the_ideal_model(dma):
    for seed in range(40):
        t = rand_group(seed, 1 + seed % 7)
        order = list(range(len(t)))
        random.Random(seed).shuffle(order)
        for num in (1, 3, 7):
            assert oracle.predict_overlap(t, order, dma, num, num) == oracle.predict(t, order, dma)


def test_one_dma_engine_never_overlaps_transfers():
    for seed in range(40):
        t = rand_group(100 + seed, 2 + seed % 6)
        order = list(range(len(t)))[::-1]
        assert oracle.predict_overlap(t, order, 1, 1, 5) == oracle.predict(t, order, 1)


def test_without_htd_nothing_overlaps():
    # zero-length HtD transfers end the instant they start: they slow nothing
    for seed in range(30):
        t = [[0, k, d] for _, k, d in rand_group(200 + seed, 5)]
        for order in itertools.islice(itertools.permutations(range(5)), 0, 120, 7):
            assert oracle.predict_overlap(t, order, 2, 2, 3) == oracle.predict(t, order, 2)


def test_two_tasks_by_hand():
    # A = (4, 2, 6), B = (8, 1, 1), order A B, two engines, rate 1/2 while both
    # transfers run.  HtD_A [0, 4); K_A [4, 6); HtD_B starts at 4 and moves
    # 2 ns of its 8 alone; at 6 DtH_A starts: both now run at half speed, so
    # HtD_B's 6 ns left take 12 ns and DtH_A's 6 ns take 12 ns: both end at
    # 18.  K_B [18, 19), DtH_B [19, 20).  Ideal model: 14.
    t = [[4, 2, 6], [8, 1, 1]]
    ms, tl = oracle.predict_overlap(t, [0, 1], 2, 1, 2, timeline=True)
    assert ms == 20
    assert tl[1, 0].tolist() == [4, 18] and tl[0, 2].tolist() == [6, 18]
    assert tl[1, 1].tolist() == [18, 19] and tl[1, 2].tolist() == [19, 20]
    assert oracle.predict(t, [0, 1], 2) == 14
    # rounding up to whole ns: rate 2/3, HtD_B's 6 ns left (18 units at 2 per
    # ns) take 9 ns and DtH_A's 18 units also 9: both end at 15
    assert oracle.predict_overlap(t, [0, 1], 2, 2, 3, timeline=True)[1][1, 0].tolist() == [4, 15]
    # rate 2/5: 30 units at 2 per ns = 15 ns -> 21; then K_B, DtH_B -> 23
    assert oracle.predict_overlap(t, [0, 1], 2, 2, 5) == 23


def test_fig6_reestimates_with_one_rate():
    # Fig. 6: HtD_0 ends at 200 and HtD_1 (10 ms) starts, ending at 210 if
    # alone; K_0 runs 200..207; DtH_0 starts at 207 and HtD_1's end moves to
    # 215.  A rate of 3/8 gives exactly that: 3 ms left take 8 ms.  DtH_0
    # (8 ms) has then moved 3 ms of its work, so alone from 215 it ends at
    # 220, the figure's estimate before HtD_2 arrives.  (The figure's next
    # value, 224, would need a rate of 5/9: no single rate fits both.)
    t = [[200, 7, 8], [10, 1, 1]]
    _, tl = oracle.predict_overlap(t, [0, 1], 2, 3, 8, timeline=True)
    assert tl[0, 0].tolist() == [0, 200] and tl[0, 1].tolist() == [200, 207]
    assert tl[0, 2].tolist() == [207, 220]
    assert tl[1, 0].tolist() == [200, 215]


def inflated(t, num, den):
    # every transfer at the slow rate all the time (rounded up)
    return [[-(-h * den // num), k, -(-d * den // num)] for h, k, d in t]


@pytest.mark.parametrize("rate", [(1, 2), (2, 3), (3, 8), (5, 7)])
def test_between_ideal_and_always_slow(rate):
    num, den = rate
    for seed in range(30):
        t = rand_group(300 + seed, 6, hi=1000)
        for order in itertools.islice(itertools.permutations(range(6)), 0, 720, 37):
            got = oracle.predict_overlap(t, order, 2, num, den)
            assert oracle.predict(t, order, 2) <= got <= oracle.predict(inflated(t, num, den), order, 2)


def test_timeline_obeys_queue_and_dependency_rules():
    b = inputs.random_groups(7, [7], hi=3_000_000)
    t = b.group(0)
    order = [3, 1, 6, 0, 5, 2, 4]
    _, tl = oracle.predict_overlap(t, order, 2, 2, 3, timeline=True)
    for i in range(7):
        h, k, d = tl[i]
        assert k[0] == max(h[1], tl[i - 1, 1, 1] if i else 0)        # kernel: own HtD, K queue
        assert d[0] == max(k[1], tl[i - 1, 2, 1] if i else 0)        # DtH: own K, DtH queue
        assert h[0] == (tl[i - 1, 0, 1] if i else 0)                 # HtD queue back to back
        assert k[1] - k[0] == t[order[i]][1]                         # kernels never slow down
        assert h[1] - h[0] >= t[order[i]][0] and d[1] - d[0] >= t[order[i]][2]


def test_exhaustive_overlap_full_rate_matches_exhaustive():
    for seed, n in ((1, 5), (2, 6), (3, 4)):
        t = rand_group(400 + seed, n, hi=9)
        for dma in (1, 2):
            assert oracle.exhaustive_overlap(t, dma, 4, 4) == oracle.exhaustive(t, dma)


def test_exhaustive_overlap_by_enumeration():
    t = rand_group(500, 5, hi=20)
    got = oracle.exhaustive_overlap(t, 2, 2, 3)
    ms = [oracle.predict_overlap(t, o, 2, 2, 3) for o in itertools.permutations(range(5))]
    assert got["best"] == min(ms) and got["worst"] == max(ms) and got["sum"] == sum(ms)
    assert got["best_rank"] == ms.index(min(ms)) and got["worst_rank"] == ms.index(max(ms))
    assert got["mean"] == sum(ms) / 120


def test_closed_form_tail_matches_the_event_simulation():
    """The enumeration kernel stops simulating events once the last HtD has
    ended and finishes the order with the plain recurrence (kernels back to
    back, each DtH at full speed after its kernel and the DtH before).  The
    bench's counting model takes the same steps (bench.overlap_loop_events);
    here its makespans must equal the oracle's event simulation."""
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    rng = np.random.default_rng(12)
    for trial in range(400):
        n = int(rng.integers(1, 9))
        hi = int(rng.choice([5, 40, 2_000_000]))
        t = rng.integers(0, hi, size=(n, 3)).astype(np.int32)
        num, den = [(1, 2), (2, 3), (3, 8), (5, 9), (1, 1), (7, 10)][trial % 6]
        order = [int(x) for x in rng.permutation(n)]
        _, _, _, ms = bench.overlap_loop_events(t, order, num, den)
        assert ms == oracle.predict_overlap(t, order, 2, num, den), (t.tolist(), order, num, den)

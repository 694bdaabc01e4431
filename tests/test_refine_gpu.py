"""The exact-model descent (tm_refine_batch_dev, and the beam's refine
stage) against a plain descent written here over the same move list, with
every makespan taken from the oracle's event simulation.  Orders and
makespans are integers and must match exactly."""
import random

import numpy as np
import pytest

import oracle
from paper_1806_10113_gb300 import build as tmbuild
from paper_1806_10113_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tm():
    tmbuild.build()
    from paper_1806_10113_gb300 import tm as tmmod
    return tmmod


def moves(n):
    """Swaps (i < j) by j then i; then moves of the task at i to position j,
    |i - j| >= 2, by max(i, j), then i, then j."""
    swaps = [("s", i, j) for j in range(1, n) for i in range(j)]
    ins = [("i", i, j) for m in range(n) for i in range(m + 1) for j in range(m + 1)
           if max(i, j) == m and abs(i - j) >= 2]
    return swaps + ins


def apply(order, mv):
    kind, i, j = mv
    o = list(order)
    if kind == "s":
        o[i], o[j] = o[j], o[i]
    else:
        o.insert(j, o.pop(i))
    return o


def descend(tasks, order, dma, max_passes=64):
    cur = oracle.predict(tasks, order, dma)
    mv = moves(len(order))
    for _ in range(max_passes):
        vals = [oracle.predict(tasks, apply(order, m), dma) for m in mv]
        if not vals or min(vals) >= cur:
            break
        k = vals.index(min(vals))              # the first best move
        order, cur = apply(order, mv[k]), vals[k]
    return order, cur


def run_refine(tm, b, start_orders):
    import torch
    dev = torch.device("cuda")
    d_tasks = torch.from_numpy(b.tasks).to(dev)
    d_off = torch.from_numpy(b.offsets).to(dev)
    d_dma = torch.from_numpy(b.dma).to(dev)
    d_orders = torch.from_numpy(np.ascontiguousarray(start_orders, dtype=np.int32)).to(dev)
    d_ms = torch.zeros(b.G, dtype=torch.int32, device=dev)
    d_status = torch.full((b.G,), 99, dtype=torch.int32, device=dev)
    tm.tm_refine_batch_dev(d_tasks, d_off, b.G, d_dma, d_orders, d_ms, d_status)
    torch.cuda.synchronize()
    return d_orders.cpu().numpy(), d_ms.cpu().numpy().astype(np.int64), d_status.cpu().numpy()


@pytest.mark.parametrize("dma", [1, 2])
def test_refine_matches_plain_descent(tm, dma):
    """Groups of every size 1..16 (and more at random), three duration scales,
    from random orders and from the heuristic's orders."""
    rng = random.Random(70 + dma)
    sizes = list(range(1, 17)) + [rng.randint(2, 16) for _ in range(60)]
    groups = []
    for g, n in enumerate(sizes):
        hi = rng.choice([7, 5000, 3_000_000])
        groups.append([[rng.randint(0, hi) for _ in range(3)] for _ in range(n)])
    b = inputs.make_batch(groups, [dma] * len(groups))
    starts = []
    for g, n in enumerate(sizes):
        if g % 2:
            starts += oracle.heuristic(b.group(g), dma)[0]
        else:
            p = list(range(n))
            rng.shuffle(p)
            starts += p
    orders, ms, status = run_refine(tm, b, starts)
    assert (status == 0).all()
    for g in range(b.G):
        o0, o1 = int(b.offsets[g]), int(b.offsets[g + 1])
        want_o, want_ms = descend(b.group(g), starts[o0:o1], dma)
        assert list(orders[o0:o1]) == want_o, g
        assert ms[g] == want_ms, g


def test_refine_rejects_bad_orders_and_keeps_them(tm):
    b = inputs.random_groups(3, [4, 5, 3], hi=1000, dma=2)
    starts = [0, 1, 1, 3] + [4, 3, 2, 1, 0] + [0, 2, 5]
    orders, _, status = run_refine(tm, b, starts)
    assert list(status) == [-1, 0, -1]
    assert list(orders[:4]) == [0, 1, 1, 3] and list(orders[9:]) == [0, 2, 5]
    want, _ = descend(b.group(1), [4, 3, 2, 1, 0], 2)
    assert list(orders[4:9]) == want


def test_refine_result_is_a_local_optimum(tm):
    b = inputs.half_dk_half_dt(groups=24, n=12, seed=9, models=(2, 1))
    starts = np.concatenate([np.arange(12, dtype=np.int32)] * b.G)
    orders, ms, status = run_refine(tm, b, starts)
    assert (status == 0).all()
    for g in range(b.G):
        o = [int(x) for x in orders[12 * g:12 * g + 12]]
        t, dma = b.group(g), int(b.dma[g])
        assert oracle.predict(t, o, dma) == ms[g]
        assert all(oracle.predict(t, apply(o, m), dma) >= ms[g] for m in moves(12))

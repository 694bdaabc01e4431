"""Edge cases through the C ABI on the GPU: empty batches, one-task groups,
the largest group sizes each entry point accepts, and zero durations."""
import numpy as np
import pytest

import oracle
from paper_1806_10113_gb300 import inputs, tm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EMPTY_T = np.zeros((0, 3), dtype=np.int32)
EMPTY_OFF = np.zeros(1, dtype=np.int32)
EMPTY_DMA = np.zeros(0, dtype=np.int32)


def test_empty_batches_host_calls():
    assert tm.tm_exhaustive_batch(EMPTY_T, EMPTY_OFF, EMPTY_DMA).shape == (0,)
    o, m = tm.tm_heuristic_batch(EMPTY_T, EMPTY_OFF, EMPTY_DMA)
    assert o.shape == (0,) and m.shape == (0,)
    assert tm.tm_predict_batch(EMPTY_T, EMPTY_OFF, np.zeros(0, np.int32), EMPTY_DMA).shape == (0,)
    st, o, m = tm.tm_schedule_batch(EMPTY_T, EMPTY_OFF, EMPTY_DMA)
    assert st.shape == (0,) and m.shape == (0,)
    assert tm.tm_exhaustive_overlap_batch(EMPTY_T, EMPTY_OFF, EMPTY_DMA, 1, 2).shape == (0,)
    assert tm.tm_predict_overlap_batch(EMPTY_T, EMPTY_OFF, np.zeros(0, np.int32), EMPTY_DMA,
                                       1, 2).shape == (0,)


def test_empty_batches_device_calls():
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    dummy = torch.zeros(16, dtype=torch.int32, device="cuda")
    plan = tm.Plan(EMPTY_OFF)
    assert plan.launches() == 0
    tm.tm_exhaustive_batch_dev(plan, dummy, dummy, dummy)
    tm.tm_schedule_batch_dev(plan, dummy, dummy, dummy, dummy)
    plan.close()
    tm.tm_heuristic_batch_dev(dummy, d(EMPTY_OFF), 0, dummy, dummy)
    tm.tm_predict_batch_dev(dummy, d(EMPTY_OFF), 0, dummy, dummy, dummy)
    tm.tm_exhaustive_batch_noalloc(dummy, EMPTY_OFF, dummy, dummy)
    r = tm.Ranker(seed=1)
    tm.tm_beam_batch_dev(r, dummy, d(EMPTY_OFF), EMPTY_OFF, dummy, 8, dummy)
    r.forward_dev(dummy, 0, dummy)
    torch.cuda.synchronize()
    assert r.errors() == 0
    r.close()
    s = tm.Server(exact_max_n=8, lanes=1, lane_groups=4)
    assert s.replay(EMPTY_T, EMPTY_OFF, EMPTY_DMA, np.zeros(0, np.int64)).shape == (0,)
    s.close()


def test_one_task_groups_everywhere():
    t = [[5, 7, 11]]
    for dma in (1, 2):
        st = tm.tm_exhaustive(t, dma)
        assert st["best"] == st["worst"] == 23 and st["sum"] == 23 and st["best_order"] == [0]
        assert tm.tm_heuristic(t, dma) == ([0], 23)
        assert tm.tm_predict_overlap(t, [0], dma, 1, 3) == 23
    b = inputs.make_batch([t] * 5, [2, 1, 2, 1, 2])
    r = tm.Ranker(seed=2)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    orders = torch.full((5,), -1, dtype=torch.int32, device="cuda")
    ms = torch.zeros(5, dtype=torch.int32, device="cuda")
    tm.tm_beam_batch_dev(r, d(b.tasks), d(b.offsets), b.offsets, d(b.dma), 64, orders, ms)
    torch.cuda.synchronize()
    assert (orders.cpu().numpy() == 0).all() and (ms.cpu().numpy() == 23).all()
    r.close()


def test_all_zero_durations():
    t = np.zeros((7, 3), dtype=np.int32)
    for dma in (1, 2):
        st = tm.tm_exhaustive(t, dma)
        assert st["best"] == st["worst"] == 0 and st["sum"] == 0 and st["best_rank"] == 0
        assert st["worst_rank"] == 0
        order, ms = tm.tm_heuristic(t, dma)
        assert ms == 0 and (order, ms) == oracle.heuristic(t, dma)
        assert tm.tm_predict_overlap(t, list(range(7)), dma, 1, 2) == 0


def test_largest_sizes_each_entry_point_accepts():
    big = inputs.random_groups(51, [16, 16], hi=1_000_000)
    o, m = tm.tm_heuristic_batch(big.tasks, big.offsets, big.dma)
    for g in range(2):
        assert (list(o[big.offsets[g]:big.offsets[g + 1]]), int(m[g])) == \
            oracle.heuristic(big.group(g), int(big.dma[g]))
    with pytest.raises(tm.TMError) as e:                      # 17 tasks
        tm.tm_heuristic_batch(np.ones((17, 3), np.int32), [0, 17], [2])
    assert e.value.code == -1
    with pytest.raises(tm.TMError) as e:                      # exhaustive beyond 12
        tm.tm_exhaustive_batch(np.ones((13, 3), np.int32), [0, 13], [2])
    assert e.value.code == -4
    with pytest.raises(tm.TMError) as e:
        tm.tm_exhaustive_overlap_batch(np.ones((13, 3), np.int32), [0, 13], [2], 1, 2)
    assert e.value.code == -4
    with pytest.raises(tm.TMError) as e:                      # beam width beyond 64
        r = tm.Ranker(seed=3)
        d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        tm.tm_beam_batch_dev(r, d(big.tasks), d(big.offsets), big.offsets, d(big.dma), 65,
                             torch.zeros(32, dtype=torch.int32, device="cuda"))
    assert e.value.code == -1

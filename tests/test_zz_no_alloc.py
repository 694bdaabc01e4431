"""tm_exhaustive_batch_noalloc: the exhaustive search for callers that cannot
allocate device memory.

Some callers cannot call cudaMalloc: their GPU memory is all reserved by
another allocator (a framework's caching pool), or they cannot pay for
cudaMalloc / cudaFree (cudaFree waits for the whole device) where they run.
tm_plan_create allocates, so such callers use tm_exhaustive_batch_noalloc,
which keeps its working memory in a fixed device array inside libtm.so.

The test calls it through the C ABI twice in a row, on two different
batches, and compares each result with the plan-based entry point
tm_exhaustive_batch_dev.  Everything compared is an integer, or a double
computed by the same expression, so the comparison is exact (the tolerance
of the other parity tests).  The second call also checks that state left in
the shared array by the first call does not leak into its result.  Another
test checks that, once the device is set up, calls leave the device's free
memory unchanged.

This file is collected last on purpose, and passes both alone in a fresh
process and after the rest of the suite.
"""
import numpy as np
import pytest

from paper_1806_10113_gb300 import build as tmbuild
from paper_1806_10113_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tm():
    tmbuild.build()
    from paper_1806_10113_gb300 import tm as tmmod
    return tmmod


def run_both(tm, torch, b):
    dev = torch.device("cuda")
    d_tasks = torch.from_numpy(b.tasks).to(dev)
    d_dma = torch.from_numpy(b.dma).to(dev)
    nbytes = b.G * tm.STATS_DTYPE.itemsize
    ref = torch.zeros(nbytes, dtype=torch.uint8, device=dev)
    ref_status = torch.full((b.G,), 7, dtype=torch.int32, device=dev)
    plan = tm.Plan(b.offsets)
    tm.tm_exhaustive_batch_dev(plan, d_tasks, d_dma, ref, ref_status)
    got = torch.full((nbytes,), 0xAB, dtype=torch.uint8, device=dev)
    got_status = torch.full((b.G,), 7, dtype=torch.int32, device=dev)
    tm.tm_exhaustive_batch_noalloc(d_tasks, b.offsets, d_dma, got, got_status)
    torch.cuda.synchronize()
    plan.close()
    return (ref.cpu().numpy(), ref_status.cpu().numpy(),
            got.cpu().numpy(), got_status.cpu().numpy())


def test_no_alloc_matches_plan_entry_point_on_two_calls(tm):
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    first = inputs.random_groups(101, [9, 5, 7, 1, 10, 3, 8, 6, 4, 2], hi=5_000_000)
    second = inputs.dk_dt_groups(groups=8, n=9, seed=7)          # 16 groups, both models
    for b in (first, second):
        ref, ref_status, got, got_status = run_both(tm, torch, b)
        assert (ref_status == 0).all() and (got_status == 0).all()
        assert got.tobytes() == ref.tobytes()
        st = got.view(tm.STATS_DTYPE)
        assert (st["best"] <= st["worst"]).all()


def test_no_alloc_call_takes_no_device_memory(tm):
    """What the entry point is for: once a device is set up, a call leaves the
    device's free memory exactly as it was (a cudaMalloc anywhere on its path,
    even of a few bytes, takes at least one allocation page)."""
    torch = pytest.importorskip("torch")
    b = inputs.random_groups(202, [8, 6, 9, 4, 7, 5], hi=2_000_000)
    dev = torch.device("cuda")
    d_tasks = torch.from_numpy(b.tasks).to(dev)
    d_dma = torch.from_numpy(b.dma).to(dev)
    d_stats = torch.zeros(b.G * tm.STATS_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    d_status = torch.zeros(b.G, dtype=torch.int32, device=dev)
    tm.tm_exhaustive_batch_noalloc(d_tasks, b.offsets, d_dma, d_stats, d_status)   # set-up
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        tm.tm_exhaustive_batch_noalloc(d_tasks, b.offsets, d_dma, d_stats, d_status)
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before
    assert (d_status.cpu().numpy() == 0).all()


def test_no_alloc_rejects_batches_beyond_its_capacity(tm):
    torch = pytest.importorskip("torch")
    b = inputs.random_groups(5, [5] * (tm.TM_NOALLOC_MAX_GROUPS + 1), hi=1000)
    d = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(tm.TMError) as e:
        tm.tm_exhaustive_batch_noalloc(d, b.offsets, d, d)
    assert e.value.code == -8

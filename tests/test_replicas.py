"""The multi-rank path of bench.py on CPU (gloo, world size 2).

The hot path shards into independent replicas: each rank schedules its own
groups (its own seed) and the only exchange is the timing aggregation of the
measurement: the slowest rank's time and the sum of all ranks' orders."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist = bench.dist_init("gloo")
    ws, r, local = bench.dist_env()
    b = bench.workload(r)
    orders = bench.orders_per_step(b)
    # a per-rank "time" that differs, to check the max-over-ranks rule
    t = 1.0 + r
    t_max = bench.max_over_ranks(dist, t)
    total = bench.sum_over_ranks(dist, float(orders))
    first_group = [int(x) for x in b.group(0)[0]]
    dist.barrier()
    dist.destroy_process_group()
    out.put((r, ws, t_max, total, orders, first_group))


def test_two_replicas_aggregate_like_the_bench():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, ws0, tmax0, tot0, ord0, g0), (r1, ws1, tmax1, tot1, ord1, g1) = res
    assert (r0, r1, ws0, ws1) == (0, 1, 2, 2)
    assert tmax0 == tmax1 == 2.0                       # the slowest rank's time
    assert tot0 == tot1 == float(ord0 + ord1)          # every rank's orders
    assert g0 != g1                                    # each replica its own groups


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(None, 3.5) == 3.5
    assert bench.sum_over_ranks(None, 7.0) == 7.0

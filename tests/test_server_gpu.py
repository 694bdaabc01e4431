"""The serving loop: every group's result is the same whether it is served
alone or in a mix, equals the direct library call for its method, and is
checked against the oracle (exhaustive optimum and first best order, the
heuristic's order, the model's makespan)."""
import numpy as np
import pytest

import oracle
from paper_1806_10113_gb300 import inputs, tm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def serve_mix(seed=21, groups=300, nmax=16):
    """Ragged groups with n ~ U{4..nmax}, log-uniform durations (DK/DT per
    task with p = 1/2), alternating device models."""
    return inputs.training_groups(groups, 4, nmax, seed)


def poisson_arrivals(G, rate, seed=0):
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1e9 / rate, G)).astype(np.int64)


def check_against_oracle(b, res, exact_max_n, heuristic_only):
    for g in range(b.G):
        r = res[g]
        t, n, dma = b.group(g), int(b.sizes()[g]), int(b.dma[g])
        assert r["status"] == 0 and r["n"] == n
        order = [int(x) for x in r["order"][:n]]
        assert sorted(order) == list(range(n)) and (r["order"][n:] == -1).all()
        assert r["makespan"] == oracle.predict(t, order, dma)
        h_order, h_ms = oracle.heuristic(t, dma)
        if n <= exact_max_n:
            assert r["method"] == tm.TM_METHOD_EXHAUSTIVE
            if n <= 9:
                ref = oracle.exhaustive(t, dma)
                assert r["makespan"] == ref["best"] and order == ref["best_order"]
            assert r["makespan"] <= h_ms
        elif heuristic_only:
            assert r["method"] == tm.TM_METHOD_HEURISTIC
            assert order == h_order and r["makespan"] == h_ms
        else:
            assert r["method"] in (tm.TM_METHOD_BEAM, tm.TM_METHOD_HEURISTIC)
            assert r["makespan"] <= h_ms
            if r["method"] == tm.TM_METHOD_HEURISTIC:
                assert order == h_order


def test_server_heuristic_only_matches_oracle():
    b = serve_mix(21, 200, 16)
    s = tm.Server(exact_max_n=9, lanes=2, lane_groups=64)
    res = s.replay(b.tasks, b.offsets, b.dma, poisson_arrivals(b.G, 20000))
    s.close()
    assert list(res["ticket"]) == sorted(res["ticket"])
    check_against_oracle(b, res, 9, heuristic_only=True)


def test_server_alone_equals_mix_and_direct_calls():
    b = serve_mix(22, 240, 16)
    ranker = tm.Ranker(seed=3)
    s = tm.Server(exact_max_n=10, beam_width=16, ranker=ranker, lanes=3, lane_groups=32)
    mix = s.replay(b.tasks, b.offsets, b.dma, poisson_arrivals(b.G, 20000, 1))
    # the same groups, each alone in its batch
    alone = []
    for g in range(b.G):
        ticket = s.submit(b.group(g), int(b.dma[g]))
        got = s.poll(1, wait_us=10_000_000)
        assert len(got) == 1 and got[0]["ticket"] == ticket
        alone.append(got[0])
    alone = np.array(alone, dtype=tm.RESULT_DTYPE)
    for k in ("status", "n", "makespan", "method", "order"):
        assert np.array_equal(mix[k], alone[k]), k
    c = s.counters()
    assert c["completed"] == 2 * b.G and c["batches"] >= b.G + 1
    s.close()
    check_against_oracle(b, mix, 10, heuristic_only=False)
    # the beam groups equal one direct tm_beam_batch_dev call over all of them
    big = [g for g in range(b.G) if b.sizes()[g] > 10]
    sub = inputs.make_batch([b.group(g) for g in big], b.dma[big])
    d_orders = torch.zeros(sub.tasks.shape[0], dtype=torch.int32, device="cuda")
    d_ms = torch.zeros(sub.G, dtype=torch.int32, device="cuda")
    d_won = torch.zeros(sub.G, dtype=torch.int32, device="cuda")
    tm.tm_beam_batch_dev(ranker, torch.from_numpy(sub.tasks).cuda(),
                         torch.from_numpy(sub.offsets).cuda(), sub.offsets,
                         torch.from_numpy(sub.dma).cuda(), 16, d_orders, d_ms, d_beam_won=d_won)
    torch.cuda.synchronize()
    orders = d_orders.cpu().numpy()
    for i, g in enumerate(big):
        n = int(b.sizes()[g])
        assert mix[g]["makespan"] == int(d_ms[i])
        assert list(mix[g]["order"][:n]) == list(orders[sub.offsets[i]:sub.offsets[i + 1]])
        assert mix[g]["method"] == (tm.TM_METHOD_BEAM if int(d_won[i]) else tm.TM_METHOD_HEURISTIC)


def test_server_exact_groups_match_exhaustive_batch():
    b = serve_mix(23, 120, 12)
    s = tm.Server(exact_max_n=12, lanes=2, lane_groups=16, lane_subsets=2000)
    res = s.replay(b.tasks, b.offsets, b.dma, poisson_arrivals(b.G, 50000, 2))
    s.close()
    st = tm.tm_exhaustive_batch(b.tasks, b.offsets, b.dma)
    for g in range(b.G):
        n = int(b.sizes()[g])
        assert res[g]["status"] == 0 and res[g]["method"] == tm.TM_METHOD_EXHAUSTIVE
        assert res[g]["makespan"] == st[g]["best"]
        assert list(res[g]["order"][:n]) == list(st[g]["best_order"][:n])


def test_server_small_lanes_and_burst():
    # capacity of 4 groups per lane: a burst of 100 is served in >= 25 batches
    b = serve_mix(24, 100, 8)
    s = tm.Server(exact_max_n=8, lanes=2, lane_groups=4)
    res = s.replay(b.tasks, b.offsets, b.dma, np.zeros(b.G, dtype=np.int64))
    c = s.counters()
    s.close()
    assert c["batches"] >= 25 and c["max_batch_groups"] <= 4
    check_against_oracle(b, res, 8, heuristic_only=True)


def test_server_rejects_bad_groups_at_submit():
    s = tm.Server(exact_max_n=8, lanes=1, lane_groups=8)
    for tasks, dma, code in (([[1, -2, 3]], 2, -2), ([[2**30, 2**30, 0]], 2, -3),
                             ([[1, 2, 3]], 3, -1), ([[1, 2, 3]] * 17, 2, -1)):
        with pytest.raises(tm.TMError) as e:
            s.submit(tasks, dma)
        assert e.value.code == code
    t = s.submit([[5, 6, 7], [1, 2, 3]], 1)
    got = s.poll(4, wait_us=5_000_000)
    assert len(got) == 1 and got[0]["ticket"] == t and got[0]["status"] == 0
    s.close()


def test_server_destroy_drains_queue():
    b = serve_mix(25, 64, 12)
    s = tm.Server(exact_max_n=12, lanes=1, lane_groups=8, lane_subsets=4000)
    for g in range(b.G):
        s.submit(b.group(g), int(b.dma[g]))
    s.close()     # returns after every queued group ran

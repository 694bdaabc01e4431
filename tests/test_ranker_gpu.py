"""GPU parity of the learned ranker's kernels against the CPU oracle
(oracle/mlp.py, fp64) and checks of the beam search against the exact model
(oracle event simulation, Sec. 4.1) and the exhaustive optimum."""
import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_1806_10113_gb300 import inputs, tm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F = tm.TM_RANKER_FEATURES


def cuda(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    return (t.to(dtype) if dtype is not None else t).cuda()


def bf16_bits_to_float(bits: np.ndarray) -> np.ndarray:
    u = bits.astype(np.uint16).astype(np.uint32) << 16
    return u.view(np.float32).astype(np.float64)


def float_to_bf16_bits(x: np.ndarray) -> np.ndarray:
    r = mlp.to_bf16(x).astype(np.float32)
    return (r.view(np.uint32) >> 16).astype(np.uint16).view(np.int16)


def random_params(seed: int, scale: float = 1.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    p = np.zeros(mlp.NPARAM)
    i = 0
    for name, shape in mlp.SIZES:
        n = int(np.prod(shape))
        fan_in = shape[0] if len(shape) == 2 else (mlp.H if name == "w4" else 1)
        if name.startswith("b"):
            p[i:i + n] = rng.normal(0, 0.05, n)
        else:
            p[i:i + n] = rng.normal(0, scale * np.sqrt(2.0 / fan_in), n)
        i += n
    return p


def expected_rows(b, orders):
    """Rows, state offsets and targets of the training layout, from the
    oracle's event simulation and feature map."""
    X, state_off, target = [], [], []
    for g in range(b.G):
        t = b.group(g)
        n = t.shape[0]
        o = orders[b.offsets[g]:b.offsets[g + 1]]
        dma = int(b.dma[g])
        _, tl = oracle.predict(t, o, dma, timeline=True)
        dinit = int(t[:, 0].sum()) if dma == 1 else 0
        used = set()
        for p in range(n - 1):
            state = (0, 0, dinit) if p == 0 else (tl[p - 1, 0, 1], tl[p - 1, 1, 1], tl[p - 1, 2, 1])
            cands = [j for j in range(n) if j not in used]
            state_off.append(len(X))
            target.append(len(X) + cands.index(int(o[p])))
            for j in cands:
                X.append(mlp.features(t, used, state, dma, j))
            used.add(int(o[p]))
    state_off.append(len(X))
    return np.asarray(X).reshape(-1, F), np.asarray(state_off), np.asarray(target)


@pytest.mark.parametrize("source", ["orders", "stats"])
def test_training_rows_match_oracle_features(source):
    b = inputs.random_groups(11, [1, 2, 5, 9, 3, 8, 4, 6], hi=2_000_000)
    rng = np.random.default_rng(4)
    orders = np.concatenate([rng.permutation(n) for n in b.sizes()]).astype(np.int32)
    d_stats = None
    if source == "stats":
        st = np.zeros(b.G, dtype=tm.STATS_DTYPE)
        for g, n in enumerate(b.sizes()):
            st[g]["best_order"][:n] = orders[b.offsets[g]:b.offsets[g + 1]]
        d_stats = cuda(st.view(np.uint8))
    rows, states = tm.tm_ranker_rows_count(b.offsets)
    pad = (rows + 15) // 16 * 16
    X = torch.full((pad * F,), -1, dtype=torch.int16, device="cuda")   # tail must be zeroed
    soff = torch.full((states + 1,), -7, dtype=torch.int32, device="cuda")
    tgt = torch.full((states,), -7, dtype=torch.int32, device="cuda")
    status = torch.full((b.G,), 99, dtype=torch.int32, device="cuda")
    r = tm.Ranker(seed=1)
    r.rows_dev(cuda(b.tasks), cuda(b.offsets), b.G, cuda(b.dma), rows, states, X, soff, tgt,
               d_orders=cuda(orders) if source == "orders" else None, d_stats=d_stats,
               d_status=status)
    torch.cuda.synchronize()
    assert (status.cpu().numpy() == 0).all()
    Xe, soff_e, tgt_e = expected_rows(b, orders)
    assert np.array_equal(soff.cpu().numpy(), soff_e)
    assert np.array_equal(tgt.cpu().numpy(), tgt_e)
    got = bf16_bits_to_float(X.cpu().numpy().reshape(pad, F))
    assert not got[rows:].any()
    ref = mlp.to_bf16(Xe)
    # both sides round to bfloat16; the kernel computes in float32 first, so
    # a value next to a rounding boundary may land one bfloat16 step away
    assert np.all(np.abs(got[:rows] - ref) <= 2.0 ** -7 * np.abs(ref) + 1e-30)
    assert np.mean(got[:rows] == ref) > 0.999


def test_training_rows_reject_bad_order():
    b = inputs.random_groups(12, [4, 5, 3])
    orders = np.concatenate([np.arange(4), [0, 1, 1, 3, 4], np.arange(3)]).astype(np.int32)
    rows, states = tm.tm_ranker_rows_count(b.offsets)
    pad = (rows + 15) // 16 * 16
    X = torch.full((pad * F,), -1, dtype=torch.int16, device="cuda")
    soff = torch.zeros(states + 1, dtype=torch.int32, device="cuda")
    tgt = torch.zeros(states, dtype=torch.int32, device="cuda")
    status = torch.full((b.G,), 99, dtype=torch.int32, device="cuda")
    r = tm.Ranker(seed=1)
    r.rows_dev(cuda(b.tasks), cuda(b.offsets), b.G, cuda(b.dma), rows, states, X, soff, tgt,
               d_orders=cuda(orders), d_status=status)
    torch.cuda.synchronize()
    assert list(status.cpu().numpy()) == [0, -1, 0]
    Xh = X.cpu().numpy().reshape(pad, F)
    lo, hi = 4 * 5 // 2 - 1, 4 * 5 // 2 - 1 + 5 * 6 // 2 - 1
    assert not Xh[lo:hi].any()          # the bad group's rows are zero
    assert Xh[:lo].any() and Xh[hi:rows].any()


def forward_keep(r, bits, M, path):
    """Logits and hidden activations of one forward kernel (path 0: the
    tensor-core scoring kernel, 1: the training forward)."""
    logits = torch.full((M,), float("nan"), dtype=torch.float32, device="cuda")
    acts = torch.zeros(3 * M * mlp.H, dtype=torch.int16, device="cuda")
    r.forward_keep_dev(cuda(bits), M, logits, acts, path=path)
    torch.cuda.synchronize()
    a = bf16_bits_to_float(acts.cpu().numpy()).reshape(3, M, mlp.H)
    return logits.cpu().numpy().astype(np.float64), a


def check_forward_elementwise(theta, x, logits, acts):
    """Every activation of every layer, and every logit, against the oracle
    evaluated from the kernel's own inputs of that layer: a float32 result
    may differ from it only by one bfloat16 rounding that the float32
    accumulation error can reach (oracle.mlp.layer_bound, zero elsewhere)."""
    prev = x
    for layer in (1, 2, 3):
        ref, bound = mlp.layer_bound(theta, prev, layer)
        err = np.abs(acts[layer - 1] - ref)
        assert np.all(err <= bound), (layer, np.argwhere(err > bound)[:5])
        prev = acts[layer - 1]
    ref, bound = mlp.head_bound(theta, acts[2])
    err = np.abs(logits - ref)
    assert np.all(err <= bound), np.argwhere(err > bound)[:5]
    # and end to end from the features alone, with the differences of every
    # layer carried through |W| (oracle.mlp.forward_bound)
    ref, E, _ = mlp.forward_bound(theta, x)
    assert np.all(np.abs(logits - ref) <= E)


@pytest.mark.parametrize("path", [0, 1])
@pytest.mark.parametrize("M", [1, 15, 16, 17, 127, 128, 129, 1000, 4101])
def test_forward_elementwise_at_tile_edges(path, M):
    """Both forward kernels, at the tensor-core kernel's 128-row tiles and the
    training kernel's 16-row slabs, with ragged tails."""
    rng = np.random.default_rng(M + 17 * path)
    theta = random_params(6 + path).astype(np.float32)
    r = tm.Ranker(seed=2)
    r.set_params(theta)
    bits = float_to_bf16_bits(rng.normal(0, 1, (M, F)).astype(np.float32))
    x = bf16_bits_to_float(bits)
    logits, acts = forward_keep(r, bits, M, path)
    assert r.errors() == 0
    check_forward_elementwise(theta.astype(np.float64), x, logits, acts)
    if path == 0:
        # the scoring entry point computes exactly what the kept pass did
        lg = torch.zeros(M, dtype=torch.float32, device="cuda")
        r.forward_dev(cuda(bits), M, lg)
        torch.cuda.synchronize()
        assert np.array_equal(lg.cpu().numpy().astype(np.float64), logits)


def test_forward_many_tiles_per_cta():
    """300,000 rows: several tiles per warpgroup and CTA; every element."""
    M = 300_000
    rng = np.random.default_rng(M)
    theta = random_params(12).astype(np.float32)
    r = tm.Ranker(seed=2)
    r.set_params(theta)
    bits = float_to_bf16_bits(rng.normal(0, 1, (M, F)).astype(np.float32))
    logits, acts = forward_keep(r, bits, M, 0)
    assert np.isfinite(logits).all() and r.errors() == 0
    check_forward_elementwise(theta.astype(np.float64), bf16_bits_to_float(bits), logits, acts)


def test_get_params_roundtrip_and_init():
    r = tm.Ranker(seed=7)
    p = r.get_params()
    W1 = p[:F * 128]
    assert np.abs(W1).max() <= np.sqrt(6.0 / F) and W1.std() > 0.1
    assert not p[F * 128:F * 128 + 128].any()            # b1 = 0
    q = random_params(8).astype(np.float32)
    r.set_params(q)
    assert np.array_equal(r.get_params(), q)
    assert np.array_equal(tm.Ranker(seed=7).get_params(), p)    # seeded


@pytest.mark.parametrize("M,S", [(777, 101), (4096 + 13, 300)])
def test_gradients_match_oracle(M, S):
    """Every one of the 37,377 gradient entries and the loss, against the
    oracle's backward pass run from the training kernel's own forward
    results, with bfloat16 deltas where the kernels round them: a float32
    result may differ by the softmax's and the accumulations' rounding and by
    the bfloat16 roundings that those can flip (oracle.mlp.backward_bound).
    The forward those results come from is checked element by element too."""
    rng = np.random.default_rng(M)
    x = mlp.to_bf16(rng.normal(0, 1, (M, F)))
    cuts = np.sort(rng.choice(np.arange(1, M), S - 1, replace=False))
    off = np.concatenate([[0], cuts, [M]]).astype(np.int32)
    target = np.array([rng.integers(off[s], off[s + 1]) for s in range(S)], dtype=np.int32)
    theta = random_params(9).astype(np.float32)
    r = tm.Ranker(seed=3)
    r.set_params(theta)
    pad = (M + 15) // 16 * 16
    Xb = np.zeros((pad, F), dtype=np.int16)
    Xb[:M] = float_to_bf16_bits(x)
    logits, acts = forward_keep(r, Xb[:M], M, 1)
    check_forward_elementwise(theta.astype(np.float64), x, logits, acts)
    grad = torch.zeros(tm.TM_RANKER_PARAMS, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    r.grad_dev(cuda(Xb), M, cuda(off), cuda(target), S, d_grad=grad, d_loss=loss)
    torch.cuda.synchronize()
    g = grad.cpu().numpy().astype(np.float64)
    ref_loss, ref_g, loss_b, g_b = mlp.backward_bound(theta.astype(np.float64), x, acts, logits,
                                                      off, target)
    assert abs(float(loss.item()) - ref_loss) <= loss_b
    err = np.abs(g - ref_g)
    bad = np.argwhere(err > g_b)
    assert bad.size == 0, [(int(i), g[i], ref_g[i], g_b[i]) for i in bad[:5, 0]]
    # and the bound is not vacuous: for most entries it is a few percent of
    # the entry (M-term float32 sums of terms that largely cancel)
    assert np.median(g_b / np.maximum(np.abs(ref_g), 1e-30)) < 0.05


def test_adam_step():
    theta = random_params(10).astype(np.float32)
    r = tm.Ranker(seed=4)
    r.set_params(theta)
    rng = np.random.default_rng(11)
    M, S = 64, 8
    Xb = float_to_bf16_bits(mlp.to_bf16(rng.normal(0, 1, (M, F))))
    off = np.arange(0, M + 1, M // S, dtype=np.int32)
    target = off[:-1] + 1
    grad = torch.zeros(tm.TM_RANKER_PARAMS, dtype=torch.float32, device="cuda")
    r.grad_dev(cuda(Xb), M, cuda(off), cuda(target), S, d_grad=grad)
    lr = 1e-3
    r.adam_dev(lr)
    g = grad.cpu().numpy()
    p1 = r.get_params()
    # first Adam step (Kingma and Ba): m_hat = g, v_hat = g^2
    m = (0.1 * g) / np.float32(1 - 0.9)
    v = (0.001 * g * g) / np.float32(1 - 0.999)
    expect = theta - lr * m / (np.sqrt(v) + 1e-8)
    assert np.allclose(p1, expect, rtol=1e-5, atol=1e-7)


def run_beam(b, ranker, width, refine_starts=0):
    d_tasks, d_off, d_devs = cuda(b.tasks), cuda(b.offsets), cuda(b.dma)
    orders = torch.full((max(b.tasks.shape[0], 1),), -1, dtype=torch.int32, device="cuda")
    ms = torch.zeros(b.G, dtype=torch.int32, device="cuda")
    status = torch.full((b.G,), 99, dtype=torch.int32, device="cuda")
    won = torch.full((b.G,), -1, dtype=torch.int32, device="cuda")
    tm.tm_beam_batch_dev(ranker, d_tasks, d_off, b.offsets, d_devs, width, orders, ms, status,
                         won, refine_starts=refine_starts)
    torch.cuda.synchronize()
    return (orders.cpu().numpy(), ms.cpu().numpy(), status.cpu().numpy(), won.cpu().numpy())


@pytest.mark.parametrize("width", [1, 8, 64])
def test_beam_orders_valid_and_exact(width):
    sizes = list(range(1, 17)) * 3
    b = inputs.random_groups(13, sizes, hi=3_000_000)
    r = tm.Ranker(seed=5)
    orders, ms, status, won = run_beam(b, r, width)
    assert (status == 0).all()
    for g in range(b.G):
        t, n, dma = b.group(g), int(b.sizes()[g]), int(b.dma[g])
        o = orders[b.offsets[g]:b.offsets[g + 1]]
        assert sorted(o.tolist()) == list(range(n))
        assert ms[g] == oracle.predict(t, o, dma)
        h_order, h_ms = oracle.heuristic(t, dma)
        assert ms[g] <= h_ms
        if won[g] == 0:
            assert o.tolist() == h_order and ms[g] == h_ms
        else:
            assert won[g] == 1 and ms[g] < h_ms


@pytest.mark.parametrize("width,starts", [(8, 1), (64, 4), (64, 8)])
def test_beam_refine_is_exact_and_locally_optimal(width, starts):
    """With the refine stage the result is the exact model's makespan of the
    returned order, no worse than the beam alone or than the descent from the
    heuristic's order (one of the starts), and no single move improves it."""
    from tests.test_refine_gpu import apply, descend, moves
    sizes = list(range(1, 17)) + [12] * 16
    b = inputs.random_groups(31, sizes, hi=3_000_000)
    r = tm.Ranker(seed=5)
    orders, ms, status, won = run_beam(b, r, width, refine_starts=starts)
    _, ms0, _, _ = run_beam(b, r, width)
    assert (status == 0).all() and set(won.tolist()) <= {0, 1}
    for g in range(b.G):
        t, n, dma = b.group(g), int(b.sizes()[g]), int(b.dma[g])
        o = [int(x) for x in orders[b.offsets[g]:b.offsets[g + 1]]]
        assert sorted(o) == list(range(n))
        assert ms[g] == oracle.predict(t, o, dma) and ms[g] <= ms0[g]
        assert ms[g] <= descend(t, oracle.heuristic(t, dma)[0], dma)[1]
        assert all(oracle.predict(t, apply(o, m), dma) >= ms[g] for m in moves(n))


def test_beam_large_batch_equals_small_batches():
    # 1100 groups of 12 tasks at width 64 (845k first-position rows) take the
    # separate row kernel and the 512-thread selection; 25 of them alone take
    # the fused, 1024-thread selection
    b = inputs.training_groups(1100, 12, 12, seed=9)
    r = tm.Ranker(seed=8)
    big = run_beam(b, r, 64)
    sub = inputs.make_batch([b.group(g) for g in range(25)], b.dma[:25])
    small = run_beam(sub, r, 64)
    T = int(sub.offsets[-1])
    assert np.array_equal(big[0][:T], small[0]) and np.array_equal(big[1][:25], small[1])
    assert np.array_equal(big[3][:25], small[3]) and (big[2] == 0).all()


@pytest.mark.parametrize("width", [16, 7, 4, 1])
def test_beam_warp_selection_equals_block_selection(width):
    # 600 ragged groups of 1..16 tasks take the one-warp-per-group selection
    # (widths up to 16, more than 8 groups), which also writes the next
    # position's rows; 8 of them alone take the block selection.  The kept
    # beams, so the orders, makespans and winners, must agree exactly.
    rng = np.random.default_rng(21)
    sizes = rng.integers(1, 17, 600)
    sizes[0] = 16
    b = inputs.random_groups(22, sizes, hi=3_000_000)
    r = tm.Ranker(seed=8)
    big = run_beam(b, r, width)
    sub = inputs.make_batch([b.group(g) for g in range(8)], b.dma[:8])
    small = run_beam(sub, r, width)
    T = int(sub.offsets[-1])
    assert (big[2] == 0).all() and (small[2] == 0).all()
    assert np.array_equal(big[0][:T], small[0]) and np.array_equal(big[1][:8], small[1])
    assert np.array_equal(big[3][:8], small[3])


def test_beam_is_exhaustive_when_wide_enough():
    # n <= 4 and width 24 >= n!: every partial order survives every step
    rng = np.random.default_rng(14)
    sizes = rng.integers(1, 5, 300)
    b = inputs.random_groups(15, sizes, hi=1_000_000)
    orders, ms, status, _ = run_beam(b, tm.Ranker(seed=6), 24)
    assert (status == 0).all()
    ref = oracle.exhaustive_batch(b.tasks, b.offsets, b.dma)
    assert [int(x) for x in ms] == [s["best"] for s in ref]


def test_beam_reports_bad_groups():
    b = inputs.random_groups(16, [5, 6, 7])
    tasks = b.tasks.copy()
    tasks[b.offsets[1] + 2, 1] = -5                       # a negative duration in group 1
    b2 = inputs.Batch(tasks, b.offsets, b.dma)
    orders, ms, status, _ = run_beam(b2, tm.Ranker(seed=6), 16)
    assert list(status) == [0, -2, 0]
    for g in (0, 2):
        o = orders[b.offsets[g]:b.offsets[g + 1]]
        assert ms[g] == oracle.predict(b.group(g), o, int(b.dma[g]))


def test_learned_beam_beats_untrained():
    from paper_1806_10113_gb300 import learn
    test = inputs.half_dk_half_dt(32, 12, seed=3, models=(2, 1))
    best = learn.stats_host(learn.exhaustive_stats(test, learn.to_device(test)),
                            test.G)["best"].astype(np.int64)
    r = tm.Ranker(seed=5)
    before = learn.evaluate(r, test, 64, best, repeats=1)
    info = learn.train(r, groups=131072, epochs=2, seed=5, lr=2e-3, minibatch_groups=1024)
    after = learn.evaluate(r, test, 64, best, repeats=1)
    assert info["losses"][-1] < info["losses"][0]
    for res in (before, after):
        assert (res["makespans"] >= best).all()
        assert res["beam_gap_mean"] <= res["heuristic_gap_mean"]
    assert after["beam_gap_mean"] < before["beam_gap_mean"], (before, after)

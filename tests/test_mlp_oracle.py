"""Pins of the ranker's CPU oracle (oracle/mlp.py) against the mathematics:
central finite differences for every gradient, a hand-checked feature
vector, and bfloat16 rounding against its definition."""
import numpy as np
import pytest

from oracle import mlp


def small_problem(seed=0, M=23, S=5):
    rng = np.random.default_rng(seed)
    theta = rng.normal(0, 0.3, mlp.NPARAM)
    x = rng.normal(0, 1, (M, mlp.F))
    cuts = np.sort(rng.choice(np.arange(1, M), S - 1, replace=False))
    off = np.concatenate([[0], cuts, [M]])
    target = np.array([rng.integers(off[s], off[s + 1]) for s in range(S)])
    return theta, x, off, target


def test_gradients_match_central_differences():
    theta, x, off, target = small_problem()
    loss, g = mlp.loss_and_grads(theta, x, off, target)
    rng = np.random.default_rng(1)
    idx = np.concatenate([rng.choice(mlp.NPARAM - 1, 200, replace=False), [mlp.NPARAM - 1]])
    eps = 1e-6
    for i in idx:
        tp, tm_ = theta.copy(), theta.copy()
        tp[i] += eps
        tm_[i] -= eps
        num = (mlp.loss_and_grads(tp, x, off, target)[0] -
               mlp.loss_and_grads(tm_, x, off, target)[0]) / (2 * eps)
        assert abs(num - g[i]) <= 1e-6 + 1e-4 * abs(num), (i, num, g[i])
    assert loss > 0


def test_forward_matches_explicit_layers():
    theta, x, _, _ = small_problem(2)
    p = mlp.unpack(theta)
    logit, _ = mlp.forward(theta, x)
    for r in range(x.shape[0]):
        a = x[r]
        for W, b in (("W1", "b1"), ("W2", "b2"), ("W3", "b3")):
            a = np.array([max(0.0, sum(a[i] * p[W][i, c] for i in range(len(a))) + p[b][c])
                          for c in range(mlp.H)])
        assert abs(sum(a * p["w4"]) + p["b4"][0] - logit[r]) < 1e-9


def test_bf16_rounding():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5, 3.0e-39, 1.0 + 2 ** -7])
    r = mlp.to_bf16(vals)
    # bfloat16 keeps 8 significand bits: 1 + 2^-8 is a tie -> even (1.0);
    # 1 + 3 * 2^-8 rounds up to 1 + 2^-6
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0 + 2 ** -6 and r[3] == -2.5
    assert r[5] == 1.0 + 2 ** -7


def test_features_by_hand():
    # three tasks (ms): A = (1, 8, 1), B = (8, 1, 1), C = (2, 2, 6); total 30, n 3 -> scale 0.1
    t = np.array([[1, 8, 1], [8, 1, 1], [2, 2, 6]])
    # prefix A placed (two DMA engines): h = 1, k = 9, d = 10; candidate C
    f = mlp.features(t, used={0}, state=(1, 9, 10), dma=2, j=2)
    # C: h' = 3, k' = max(9, 3) + 2 = 11, d' = max(10, 11) + 6 = 17; remaining {B}
    expect = {0: 0.2, 1: 0.2, 2: 0.6, 3: 0.8, 4: 0.1, 5: 0.8, 6: 0.6, 7: 0.7,
              8: 0.8, 9: 0.1, 10: 0.1, 11: 0.8, 12: 0.1, 13: 0.1, 14: 1 / 3, 15: 0.0,
              16: 0.0, 17: 0.1, 18: 0.0, 19: 0.2}
    for i, v in expect.items():
        assert abs(f[i] - v) < 1e-12, (i, f[i], v)
    assert not f[20:].any()


# ---- the float32 bounds used by the GPU parity tests ---------------------------

def _f32_layer(a, W, b, order):
    """One layer in float32 with the kernels' roundings: products of bfloat16
    values (exact in float32) summed in float32 in a given order."""
    a32, W32 = a.astype(np.float32), mlp.to_bf16(W).astype(np.float32)
    K = W32.shape[0]
    acc = np.zeros((a.shape[0], W32.shape[1]), dtype=np.float32)
    for k in (range(K) if order == "fwd" else reversed(range(K))):
        acc = (acc + np.outer(a32[:, k], W32[k]).astype(np.float32)).astype(np.float32)
    return (acc + np.asarray(b, dtype=np.float32)).astype(np.float32)


@pytest.mark.parametrize("order", ["fwd", "rev", "blas"])
def test_float32_forward_lies_within_the_bounds(order):
    """A float32 evaluation (three summation orders) of every layer and of the
    logits is within layer_bound / head_bound of the oracle fed with that
    evaluation's own inputs, and within forward_bound end to end."""
    rng = np.random.default_rng(3)
    theta = rng.normal(0, 0.25, mlp.NPARAM)
    p = mlp.unpack(theta)
    x = mlp.to_bf16(rng.normal(0, 1, (400, mlp.F)))
    acts, prev = [], x
    for layer in (1, 2, 3):
        W, b = p[f"W{layer}"], p[f"b{layer}"]
        if order == "blas":
            z = (prev.astype(np.float32) @ mlp.to_bf16(W).astype(np.float32) +
                 b.astype(np.float32)).astype(np.float32)
        else:
            z = _f32_layer(prev, W, b, order)
        a = mlp.to_bf16(np.maximum(z, 0.0))
        ref, bound = mlp.layer_bound(theta, prev, layer)
        assert np.all(np.abs(a - ref) <= bound)
        acts.append(a)
        prev = a
    w4 = mlp.to_bf16(p["w4"]).astype(np.float32)
    logit = (prev.astype(np.float32) @ w4 + np.float32(p["b4"][0])).astype(np.float64)
    ref, bound = mlp.head_bound(theta, prev)
    assert np.all(np.abs(logit - ref) <= bound)
    ref, E, _ = mlp.forward_bound(theta, x)
    assert np.all(np.abs(logit - ref) <= E)


def test_float32_backward_lies_within_the_bounds():
    """The training kernels' backward pass written in float32 (softmax,
    dlogit * w4, deltas rounded to bfloat16 after the relu mask, float32
    accumulations) stays within backward_bound of the oracle run from the
    same forward results, for every one of the 37,377 entries; and the
    bf16_deltas oracle differs from the unrounded one by what rounding the
    deltas can change."""
    rng = np.random.default_rng(8)
    M, S = 300, 40
    theta = rng.normal(0, 0.25, mlp.NPARAM)
    p = mlp.unpack(theta)
    x = mlp.to_bf16(rng.normal(0, 1, (M, mlp.F)))
    cuts = np.sort(rng.choice(np.arange(1, M), S - 1, replace=False))
    off = np.concatenate([[0], cuts, [M]])
    target = np.array([rng.integers(off[s], off[s + 1]) for s in range(S)])
    # float32 forward
    acts, prev = [], x
    for layer in (1, 2, 3):
        z = _f32_layer(prev, p[f"W{layer}"], p[f"b{layer}"], "rev")
        prev = mlp.to_bf16(np.maximum(z, 0.0))
        acts.append(prev)
    w4 = mlp.to_bf16(p["w4"]).astype(np.float32)
    logits = (prev.astype(np.float32) @ w4 + np.float32(p["b4"][0])).astype(np.float32)
    # float32 backward with the kernels' rounding points
    dl = np.zeros(M, dtype=np.float32)
    loss = np.float32(0)
    for s in range(S):
        lo, hi = off[s], off[s + 1]
        mx = logits[lo:hi].max()
        e = np.exp(logits[lo:hi] - mx).astype(np.float32)
        zs = np.float32(e.sum(dtype=np.float32))
        dl[lo:hi] = e * np.float32(1.0 / (zs * np.float32(S)))
        dl[target[s]] -= np.float32(1.0 / S)
        loss += np.float32((np.log(zs) + mx - logits[target[s]]) / np.float32(S))
    g = {"w4": (acts[2].astype(np.float32).T @ dl).astype(np.float64),
         "b4": np.array([dl.sum(dtype=np.float32)], dtype=np.float64)}
    dz = mlp.to_bf16((np.outer(dl, w4).astype(np.float32)) * (acts[2] > 0))
    for lvl in (3, 2, 1):
        prev = acts[lvl - 2] if lvl > 1 else x
        g[f"W{lvl}"] = (prev.astype(np.float32).T @ dz.astype(np.float32)).astype(np.float64)
        g[f"b{lvl}"] = dz.astype(np.float32).sum(0, dtype=np.float32).astype(np.float64)
        if lvl > 1:
            Wb = mlp.to_bf16(p[f"W{lvl}"]).astype(np.float32)
            v = (dz.astype(np.float32) @ Wb.T).astype(np.float32)
            dz = mlp.to_bf16(v * (acts[lvl - 2] > 0))
    g32 = mlp.pack(g)
    ref_loss, ref_g, loss_b, g_b = mlp.backward_bound(theta, x, acts, logits, off, target)
    assert abs(float(loss) - ref_loss) <= loss_b
    assert np.all(np.abs(g32 - ref_g) <= g_b)
    # rounding the deltas changes each gradient entry by less than the deltas'
    # own rounding can: |dz - r(dz)| <= 2^-8 |dz| summed through |a|
    _, g_plain = mlp.loss_and_grads(theta, x, off, target, bf16=True)
    _, g_rd = mlp.loss_and_grads(theta, x, off, target, bf16=True, bf16_deltas=True)
    assert not np.array_equal(g_plain, g_rd)
    assert np.all(np.abs(g_plain - g_rd) <= 2.0 ** -7 * np.abs(g_plain).max() * M)

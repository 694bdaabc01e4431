"""Pins of the ranker's CPU oracle (oracle/mlp.py) against the mathematics:
central finite differences for every gradient, a hand-checked feature
vector, and bfloat16 rounding against its definition."""
import numpy as np

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

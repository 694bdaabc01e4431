"""CPU oracle of the learned ranker's arithmetic (TEST INFRASTRUCTURE ONLY).

Plain numpy in float64: the feature map, the 4-layer MLP forward pass, the
per-state softmax cross-entropy and its gradients.  Only the test suite may
import it; the CUDA library never does.  The paper has no learned component:
this checks the hand-written kernels of the ranker that proposes orders for
groups beyond exhaustive reach (the exact model still judges every order).

Parameter layout (float32 in the library, float64 here), one flat vector:
    W1 [32 x 128] (row-major, in x out), b1 [128],
    W2 [128 x 128], b2 [128], W3 [128 x 128], b3 [128], w4 [128], b4 [1]
Forward: a1 = relu(x W1 + b1), a2 = relu(a1 W2 + b2), a3 = relu(a2 W3 + b3),
logit = a3 . w4 + b4.  The kernels round x, the weights and a1..a3 to
bfloat16 and accumulate in float32; pass `bf16=True` to mimic the roundings.
"""
from __future__ import annotations

import numpy as np

F, H = 32, 128
SIZES = [("W1", (F, H)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)),
         ("W3", (H, H)), ("b3", (H,)), ("w4", (H,)), ("b4", (1,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(theta):
    out, i = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = np.asarray(theta[i:i + n], dtype=np.float64).reshape(shape)
        i += n
    return out


def pack(p) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).reshape(-1) for name, _ in SIZES])


def to_bf16(a) -> np.ndarray:
    """Round float values to bfloat16 (round to nearest even), as float64."""
    a32 = np.asarray(a, dtype=np.float32)
    u = a32.view(np.uint32).astype(np.uint64)
    rounded = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return rounded.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(theta, x, bf16=False):
    """Returns logits [M] and the activations (a0 = x, a1, a2, a3)."""
    p = unpack(theta)
    r = to_bf16 if bf16 else (lambda v: np.asarray(v, dtype=np.float64))
    a0 = r(x)
    a1 = r(np.maximum(a0 @ r(p["W1"]) + p["b1"], 0.0))
    a2 = r(np.maximum(a1 @ r(p["W2"]) + p["b2"], 0.0))
    a3 = r(np.maximum(a2 @ r(p["W3"]) + p["b3"], 0.0))
    logit = a3 @ r(p["w4"]) + p["b4"][0]
    return logit, (a0, a1, a2, a3)


def loss_and_grads(theta, x, state_off, target_row, bf16=False):
    """Mean over states of the softmax cross-entropy of each state's rows
    (rows state_off[s] .. state_off[s+1]) against its target row; returns
    (loss, dtheta)."""
    p = unpack(theta)
    r = to_bf16 if bf16 else (lambda v: np.asarray(v, dtype=np.float64))
    logit, (a0, a1, a2, a3) = forward(theta, x, bf16)
    S = len(state_off) - 1
    dlogit = np.zeros_like(logit)
    loss = 0.0
    for s in range(S):
        lo, hi = state_off[s], state_off[s + 1]
        z = logit[lo:hi] - logit[lo:hi].max()
        pz = np.exp(z) / np.exp(z).sum()
        loss += -np.log(pz[target_row[s] - lo])
        g = pz.copy()
        g[target_row[s] - lo] -= 1.0
        dlogit[lo:hi] = g / S
    loss /= S
    grads = {}
    grads["w4"] = a3.T @ dlogit
    grads["b4"] = np.array([dlogit.sum()])
    dz3 = np.outer(dlogit, r(p["w4"])) * (a3 > 0)
    grads["W3"] = a2.T @ dz3
    grads["b3"] = dz3.sum(0)
    dz2 = (dz3 @ r(p["W3"]).T) * (a2 > 0)
    grads["W2"] = a1.T @ dz2
    grads["b2"] = dz2.sum(0)
    dz1 = (dz2 @ r(p["W2"]).T) * (a1 > 0)
    grads["W1"] = a0.T @ dz1
    grads["b1"] = dz1.sum(0)
    return loss, pack(grads)


def features(tasks, used, state, dma, j):
    """The 32 ranker features for appending task j (not in `used`) to a
    prefix whose engine times are state = (h, k, d).  tasks: [n, 3]."""
    t = np.asarray(tasks, dtype=np.float64)
    n = t.shape[0]
    total = t.sum()
    s = n / total if total > 0 else 0.0
    h, k, d = (float(v) for v in state)
    H, K, D = t[j]
    h1 = h + H
    k1 = max(k, h1) + K
    d1 = max(d, k1) + D
    rem = [i for i in range(n) if i not in used and i != j]
    R = t[rem] if rem else np.zeros((0, 3))
    f = np.zeros(F)
    f[0:3] = np.array([H, K, D]) * s
    f[3], f[4] = (k - h) * s, (d - k) * s
    f[5], f[6] = (k1 - h1) * s, (d1 - k1) * s
    f[7] = (d1 - d) * s
    f[8:11] = (R.sum(0) if len(rem) else np.zeros(3)) * s
    f[11:14] = (R.max(0) if len(rem) else np.zeros(3)) * s
    f[14] = len(rem) / n
    f[15] = 1.0 if dma == 1 else 0.0
    f[16] = max(0.0, h1 - k) * s
    f[17] = max(0.0, k1 - d) * s
    f[18] = (K - H) * s
    f[19] = min(H, D) * s
    return f

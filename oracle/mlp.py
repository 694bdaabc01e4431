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


def loss_and_grads(theta, x, state_off, target_row, bf16=False, bf16_deltas=False):
    """Mean over states of the softmax cross-entropy of each state's rows
    (rows state_off[s] .. state_off[s+1]) against its target row; returns
    (loss, dtheta).  bf16_deltas: also round the back-propagated deltas dz3,
    dz2, dz1 to bfloat16 after masking, as the training kernels store them."""
    p = unpack(theta)
    r = to_bf16 if bf16 else (lambda v: np.asarray(v, dtype=np.float64))
    rd = to_bf16 if bf16_deltas else (lambda v: v)
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
    dz3 = rd(np.outer(dlogit, r(p["w4"])) * (a3 > 0))
    grads["W3"] = a2.T @ dz3
    grads["b3"] = dz3.sum(0)
    dz2 = rd((dz3 @ r(p["W3"]).T) * (a2 > 0))
    grads["W2"] = a1.T @ dz2
    grads["b2"] = dz2.sum(0)
    dz1 = rd((dz2 @ r(p["W2"]).T) * (a1 > 0))
    grads["W1"] = a0.T @ dz1
    grads["b1"] = dz1.sum(0)
    return loss, pack(grads)


# ---- how far a float32 evaluation may differ from the bfloat16 path above ------
#
# The kernels compute the same roundings (x, weights, activations and, in
# training, the deltas, to bfloat16) but accumulate in float32, in an order
# of their own.  Products of two bfloat16 values are exact in float32, so a
# dot product of K terms plus a bias differs from the exact value by at most
# (K + 4) u sum |terms| (the bias may enter as up to three exact bfloat16
# parts, as in the tensor-core kernel); u = 2^-22 here, two bits above
# float32's unit roundoff, for tensor-core accumulation.  A bfloat16 rounding after it is
# monotone, so if the exact input is v and the float32 one lies within eta
# of v, the two rounded values differ by at most
#     cell(v, eta) = max(r(v + eta) - r(v), r(v) - r(v - eta)),
# zero when the whole interval rounds to r(v).  Differences already present
# in a layer's inputs (delta per element) enter the next dot product through
# |W|.  Running this layer by layer with absolute values gives, for every
# output element, a bound that holds whatever the float32 summation order.

U_ACC = 2.0 ** -22
U32 = 2.0 ** -24


def cell(v, eta):
    rv = to_bf16(v)
    return np.maximum(to_bf16(v + eta) - rv, rv - to_bf16(v - eta))


def relu_cell(z, eps):
    """cell() of r(relu(z)) for a pre-activation known within eps: relu is
    monotone too, so the interval's ends bound it (zero below -eps)."""
    act = to_bf16(np.maximum(z, 0.0))
    lo, hi = to_bf16(np.maximum(z - eps, 0.0)), to_bf16(np.maximum(z + eps, 0.0))
    return act, np.maximum(hi - act, act - lo), lo, hi


def forward_bound(theta, x):
    """(logits of the bfloat16 path, per-row bound on |float32 logit - it|,
    per-layer data for grads_bound).  x must be bfloat16 values."""
    p = unpack(theta)
    a = [to_bf16(x)]
    dl = [np.zeros_like(a[0])]
    info = []
    for W, bname in (("W1", "b1"), ("W2", "b2"), ("W3", "b3")):
        Wb, bias = to_bf16(p[W]), p[bname]
        K = Wb.shape[0]
        z = a[-1] @ Wb + bias
        eps = dl[-1] @ np.abs(Wb) + U_ACC * (K + 4) * ((np.abs(a[-1]) + dl[-1]) @ np.abs(Wb)
                                                     + np.abs(bias))
        act, d, lo, hi = relu_cell(z, eps)
        dl.append(d)
        a.append(act)
        # the relu mask (act > 0) is certain unless the interval reaches 0
        info.append({"z": z, "eps": eps, "mask_sure": (lo > 0) | (hi == 0)})
    w4 = to_bf16(p["w4"])
    logit = a[3] @ w4 + p["b4"][0]
    E = dl[3] @ np.abs(w4) + U_ACC * 132 * ((np.abs(a[3]) + dl[3]) @ np.abs(w4)
                                           + abs(p["b4"][0]))
    return logit, E, {"a": a, "delta": dl, "layers": info}


def layer_bound(theta, a_in, layer):
    """Layer `layer` (1..3) from the kernels' own bfloat16 inputs a_in: the
    rounded activations r(relu(a_in W + b)) and a bound on how far a float32
    evaluation of them can be, element by element (no difference enters from
    the inputs, so only the accumulation and one rounding remain)."""
    p = unpack(theta)
    Wb, bias = to_bf16(p[f"W{layer}"]), p[f"b{layer}"]
    a_in = np.asarray(a_in, dtype=np.float64)
    z = a_in @ Wb + bias
    eps = U_ACC * (Wb.shape[0] + 4) * (np.abs(a_in) @ np.abs(Wb) + np.abs(bias))
    act, d, _, _ = relu_cell(z, eps)
    return act, d


def head_bound(theta, a3):
    """The logits from the kernels' own a3, and the per-row bound of a float32
    evaluation (128 products and the bias, which may enter as three parts)."""
    p = unpack(theta)
    w4 = to_bf16(p["w4"])
    a3 = np.asarray(a3, dtype=np.float64)
    logit = a3 @ w4 + p["b4"][0]
    return logit, U_ACC * 132 * (np.abs(a3) @ np.abs(w4) + abs(p["b4"][0]))


def backward_bound(theta, x, acts, logits, state_off, target_row):
    """The backward pass of the training kernels, from their own forward
    results (a1, a2, a3 as bfloat16 values, logits as float32 values): the
    loss and gradient in float64 with the deltas rounded to bfloat16 where
    the kernels round them, and bounds on how far the float32 kernels can be
    (a scalar for the loss, one per parameter).  The float32 softmax (a few
    roundings per row), the float32 product dlogit * w4, the deltas' bfloat16
    rounding (cell) and every accumulation ((terms) u sum |terms|) enter the
    bounds; the relu masks are those of the kernels' own activations."""
    p = unpack(theta)
    a = [to_bf16(x)] + [np.asarray(v, dtype=np.float64) for v in acts]
    logits = np.asarray(logits, dtype=np.float64)
    M = a[0].shape[0]
    S = len(state_off) - 1
    dlog = np.zeros(M)
    eta = np.zeros(M)
    loss, loss_b = 0.0, 0.0
    for s in range(S):
        lo, hi = state_off[s], state_off[s + 1]
        n = hi - lo
        mx = logits[lo:hi].max()
        e = np.exp(logits[lo:hi] - mx)
        pz = e / e.sum()
        lz = np.log(e.sum())
        t = target_row[s]
        loss += (lz + mx - logits[t]) / S
        loss_b += (n + 8) * U_ACC * (abs(lz) + abs(mx) + abs(logits[t]) + 1.0) / S
        dlog[lo:hi] = pz / S
        dlog[t] -= 1.0 / S
        eta[lo:hi] = pz / S * (n + 8) * U_ACC + U32 / S
    loss_b += S * U32 * (abs(loss) + 1.0)
    G, B = {}, {}
    absd = np.abs(dlog) + eta
    G["w4"] = a[3].T @ dlog
    B["w4"] = eta @ np.abs(a[3]) + U_ACC * M * (absd @ np.abs(a[3]))
    G["b4"] = np.array([dlog.sum()])
    B["b4"] = np.array([eta.sum() + U_ACC * M * absd.sum()])
    w4 = to_bf16(p["w4"])
    v = np.outer(dlog, w4)
    eta_v = np.outer(eta, np.abs(w4)) + U32 * np.abs(v)
    for lvl in (3, 2, 1):
        mask = a[lvl] > 0
        dz = to_bf16(v * mask)
        ddz = np.where(mask, cell(v, eta_v), 0.0)
        absdz = np.abs(dz) + ddz
        prev = np.abs(a[lvl - 1])
        G[f"W{lvl}"] = a[lvl - 1].T @ dz
        B[f"W{lvl}"] = prev.T @ ddz + U_ACC * M * (prev.T @ absdz)
        G[f"b{lvl}"] = dz.sum(0)
        B[f"b{lvl}"] = ddz.sum(0) + U_ACC * M * absdz.sum(0)
        if lvl > 1:
            Wb = to_bf16(p[f"W{lvl}"])
            v = dz @ Wb.T
            eta_v = ddz @ np.abs(Wb).T + U_ACC * 129 * (absdz @ np.abs(Wb).T)
    return loss, pack(G), loss_b, pack(B)


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

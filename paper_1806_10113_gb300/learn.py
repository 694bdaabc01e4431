"""Training and evaluation of the learned order ranker.

The ranker (include/tm.h, "learned order ranker") is trained by behaviour
cloning: every training group is solved exactly by the exhaustive search
(tm_exhaustive_batch_dev), and the ranker learns, position by position, to
pick the task that the first best order places there.  Rows, loss, gradient
and Adam all run in the library's kernels; this module only slices batches
and loops.  The trained ranker feeds tm_beam_batch_dev, whose orders the
exact model judges, with the paper's heuristic (Sec. 5.1) as the fallback.

    python -m paper_1806_10113_gb300.learn --groups 2000000 --epochs 2 \
        --out ranker.npy          # trains, evaluates on 32 groups of 12 tasks
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import inputs, tm

STATS_BYTES = tm.STATS_DTYPE.itemsize


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("the ranker runs on a CUDA device; none is available")
    return torch


def to_device(batch: inputs.Batch):
    """(d_tasks, d_offsets, d_devs) int32 CUDA tensors of a batch."""
    torch = _torch()
    return (torch.from_numpy(np.ascontiguousarray(batch.tasks)).cuda(),
            torch.from_numpy(np.ascontiguousarray(batch.offsets)).cuda(),
            torch.from_numpy(np.ascontiguousarray(batch.dma)).cuda())


def exhaustive_stats(batch: inputs.Batch, dev, chunk_groups: int = 32768):
    """tm_stats of every group (uint8 CUDA tensor [G * 72]) by exhaustive
    search, one plan per chunk of groups."""
    torch = _torch()
    d_tasks, _, d_devs = dev
    G = batch.G
    d_stats = torch.zeros(max(G, 1) * STATS_BYTES, dtype=torch.uint8, device="cuda")
    d_status = torch.zeros(max(G, 1), dtype=torch.int32, device="cuda")
    off = batch.offsets
    for g0 in range(0, G, chunk_groups):
        g1 = min(G, g0 + chunk_groups)
        plan = tm.Plan(off[g0:g1 + 1] - off[g0])
        tm.tm_exhaustive_batch_dev(plan, d_tasks[int(off[g0]):], d_devs[g0:],
                                   d_stats[g0 * STATS_BYTES:], d_status[g0:])
        torch.cuda.synchronize()
        plan.close()
    if int(d_status[:G].abs().sum()) != 0:
        raise RuntimeError("exhaustive search rejected a training group")
    return d_stats


def stats_host(d_stats, G: int) -> np.ndarray:
    return d_stats[:G * STATS_BYTES].cpu().numpy().view(tm.STATS_DTYPE)


class Trainer:
    """Minibatch behaviour cloning of exhaustive best orders."""

    def __init__(self, ranker: tm.Ranker, batch: inputs.Batch, dev, d_stats,
                 minibatch_groups: int = 4096):
        torch = _torch()
        self.ranker, self.batch, self.dev, self.d_stats = ranker, batch, dev, d_stats
        off = batch.offsets
        self.mb = []
        for g0 in range(0, batch.G, minibatch_groups):
            g1 = min(batch.G, g0 + minibatch_groups)
            rows, states = tm.tm_ranker_rows_count(off[g0:g1 + 1] - off[g0])
            if states:
                self.mb.append((g0, g1, rows, states))
        max_rows = max((m[2] for m in self.mb), default=0)
        max_states = max((m[3] for m in self.mb), default=0)
        pad = (max_rows + 15) // 16 * 16
        self.X = torch.zeros(max(pad, 16) * tm.TM_RANKER_FEATURES, dtype=torch.int16,
                             device="cuda")
        self.state_off = torch.zeros(max_states + 1, dtype=torch.int32, device="cuda")
        self.target = torch.zeros(max(max_states, 1), dtype=torch.int32, device="cuda")
        self.status = torch.zeros(max(minibatch_groups, 1), dtype=torch.int32, device="cuda")
        self.losses = torch.zeros(max(len(self.mb), 1), dtype=torch.float32, device="cuda")
        self.steps = 0

    def rows(self, i: int):
        g0, g1, rows, states = self.mb[i]
        d_tasks, d_offsets, d_devs = self.dev
        self.ranker.rows_dev(d_tasks, d_offsets[g0:], g1 - g0, d_devs[g0:], rows, states, self.X,
                             self.state_off, self.target,
                             d_stats=self.d_stats[g0 * STATS_BYTES:], d_status=self.status)
        return rows, states

    def epoch(self, lr, rng: np.random.Generator) -> float:
        """One pass over the minibatches in random order; lr is a float or a
        function of the global step.  Returns the mean loss."""
        torch = _torch()
        order = rng.permutation(len(self.mb))
        for j, i in enumerate(order):
            rows, states = self.rows(int(i))
            self.ranker.grad_dev(self.X, rows, self.state_off, self.target, states,
                                 d_loss=self.losses[j:j + 1])
            self.steps += 1
            self.ranker.adam_dev(lr(self.steps) if callable(lr) else lr)
        torch.cuda.synchronize()
        return float(self.losses[:len(order)].mean())


def cosine_lr(base: float, total_steps: int, warmup: int = 50):
    def f(step: int) -> float:
        if step <= warmup:
            return base * step / warmup
        t = min(1.0, (step - warmup) / max(1, total_steps - warmup))
        return base * (0.05 + 0.95 * 0.5 * (1.0 + math.cos(math.pi * t)))
    return f


def evaluate(ranker: tm.Ranker, batch: inputs.Batch, beam: int = 64, best=None,
             repeats: int = 3) -> dict:
    """Gap to the exhaustive optimum of the heuristic and of the beam search,
    and the beam's groups/s (device time, best of `repeats`)."""
    torch = _torch()
    dev = to_device(batch)
    d_tasks, d_offsets, d_devs = dev
    G = batch.G
    if best is None:
        best = stats_host(exhaustive_stats(batch, dev), G)["best"].astype(np.int64)
    horders, hms = tm.tm_heuristic_batch(batch.tasks, batch.offsets, batch.dma)
    d_orders = torch.zeros(max(batch.tasks.shape[0], 1), dtype=torch.int32, device="cuda")
    d_ms = torch.zeros(max(G, 1), dtype=torch.int32, device="cuda")
    d_won = torch.zeros(max(G, 1), dtype=torch.int32, device="cuda")
    times = []
    for _ in range(repeats):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        tm.tm_beam_batch_dev(ranker, d_tasks, d_offsets, batch.offsets, d_devs, beam, d_orders,
                             d_ms, d_beam_won=d_won)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) * 1e-3)
    bms = d_ms[:G].cpu().numpy().astype(np.int64)
    hms = hms.astype(np.int64)
    gap = lambda ms: (ms - best) / np.maximum(best, 1)
    return {
        "groups": G, "beam": beam,
        "heuristic_gap_mean": float(gap(hms).mean()),
        "beam_gap_mean": float(gap(bms).mean()),
        "beam_gap_max": float(gap(bms).max()),
        "beam_within_1pct": float((gap(bms) <= 0.01).mean()),
        "beam_optimal": float((bms == best).mean()),
        "beam_won": float(d_won[:G].float().mean()),
        "beam_groups_per_s": G / min(times),
        "orders": d_orders[:batch.tasks.shape[0]].cpu().numpy(),
        "makespans": bms,
    }


def train(ranker: tm.Ranker, groups: int, epochs: int, seed: int = 5, lr: float = 2e-3,
          minibatch_groups: int = 4096, nmin: int = 6, nmax: int = 10, log=None) -> dict:
    """Draws `groups` training groups, labels them exhaustively and trains."""
    t0 = time.time()
    batch = inputs.training_groups(groups, nmin, nmax, seed)
    dev = to_device(batch)
    d_stats = exhaustive_stats(batch, dev)
    t_label = time.time() - t0
    tr = Trainer(ranker, batch, dev, d_stats, minibatch_groups)
    sched = cosine_lr(lr, epochs * len(tr.mb))
    rng = np.random.default_rng(seed)
    losses = []
    t1 = time.time()
    for e in range(epochs):
        losses.append(tr.epoch(sched, rng))
        if log:
            log(f"epoch {e}: loss {losses[-1]:.4f}")
    return {"groups": groups, "epochs": epochs, "losses": losses, "label_s": t_label,
            "train_s": time.time() - t1, "steps": tr.steps}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--groups", type=int, default=2_000_000)
    ap.add_argument("--epochs", type=int, default=2)
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--beam", type=int, default=64)
    ap.add_argument("--out", default=None, help="save the trained parameters (.npy)")
    ap.add_argument("--load", default=None, help="start from saved parameters")
    a = ap.parse_args(argv)
    tm.lib()
    ranker = tm.Ranker(seed=a.seed)
    test = inputs.half_dk_half_dt(32, 12, seed=3)
    best = stats_host(exhaustive_stats(test, to_device(test)), test.G)["best"].astype(np.int64)
    before = evaluate(ranker, test, a.beam, best)
    if a.load:
        ranker.set_params(np.load(a.load))
    info = train(ranker, a.groups, a.epochs, a.seed, a.lr, log=print) if a.epochs else {}
    after = evaluate(ranker, test, a.beam, best)
    if a.out:
        np.save(a.out, ranker.get_params())
    strip = lambda d: {k: v for k, v in d.items() if k not in ("orders", "makespans")}
    print(json.dumps({"train": info, "untrained": strip(before), "trained": strip(after)}))


if __name__ == "__main__":
    main()

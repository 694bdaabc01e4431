"""Autotuner for exhaustive-search plans.

Picks the tm_tuning (prefix depth per work item, fused or separate
finalize, resident blocks per SM, per-item cost weight, static or dynamic
work split, straight-line or looped walk level) that runs a given batch fastest, by
timing each candidate on the device with CUDA events (L2 flushed between
runs), and caches the choice in a JSON file keyed by the batch's shape (the
number of groups of each size), so later plans for the same shape reuse it
without timing.  No candidate changes any result; the tuner checks that all
candidates agree bit for bit before trusting its timings.
"""
from __future__ import annotations

import itertools
import json
import os
import threading

import numpy as np

from . import tm

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning_cache.json")
CANDIDATES = {
    "pdmax": (3, 4, 5),
    "fuse_finalize": (2,),
    "blocks_per_sm": (0, 3),
    "item_cost": (4096, 16384, 65536),
    "chunks_per_thread": (1, 3, 6, 12),
    "unroll": (1, 2, 3, 4, 5, 6, 7, 8),
}
_lock = threading.Lock()


def shape_key(offsets) -> str:
    """Group-size histogram, e.g. 'n10x128' or 'n4x1365,n5x1402,...'."""
    sizes = np.diff(np.asarray(offsets, dtype=np.int64))
    vals, counts = np.unique(sizes, return_counts=True)
    return ",".join(f"n{int(v)}x{int(c)}" for v, c in zip(vals, counts))


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path, data):
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def time_tuning(tasks, offsets, dma, tuning: dict, reps: int = 20, warmup: int = 3,
                with_heuristic: bool = True):
    """Median device time (ms) of one scheduling pass with this tuning, and
    the stats bytes it produced."""
    import torch
    dev = torch.device("cuda")
    off = np.asarray(offsets, dtype=np.int32)
    G = off.shape[0] - 1
    plan = tm.Plan(off, **tuning)
    d_tasks = torch.from_numpy(np.ascontiguousarray(tasks, dtype=np.int32)).to(dev)
    d_dma = torch.from_numpy(np.array(np.broadcast_to(dma, (G,)), dtype=np.int32)).to(dev)
    d_stats = torch.zeros(G * tm.STATS_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    d_orders = torch.zeros(max(int(off[-1]), 1), dtype=torch.int32, device=dev)
    flush = torch.empty(64 << 20, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()

    def run():
        if with_heuristic:
            tm.tm_schedule_batch_dev(plan, d_tasks, d_dma, d_stats, d_orders, None, None, stream)
        else:
            tm.tm_exhaustive_batch_dev(plan, d_tasks, d_dma, d_stats, None, stream)

    for _ in range(warmup):
        run()
    times = []
    for _ in range(reps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        run()
        b.record(stream)
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    out = d_stats.cpu().numpy().tobytes()
    plan.close()
    return float(np.median(times)), out


def tune(tasks, offsets, dma, cache_path: str | None = DEFAULT_CACHE, reps: int = 20,
         candidates=None, verbose: bool = False) -> dict:
    """Best tuning for this batch shape (timed now, or read from the cache)."""
    key = shape_key(offsets)
    if cache_path:
        with _lock:
            hit = _load(cache_path).get(key)
        if hit:
            return dict(hit["tuning"])
    cands = candidates or CANDIDATES
    results, reference = [], None
    for values in itertools.product(*cands.values()):
        tuning = dict(zip(cands.keys(), values))
        ms, out = time_tuning(tasks, offsets, dma, tuning, reps=reps)
        if reference is None:
            reference = out
        elif out != reference:
            raise RuntimeError(f"tuning {tuning} changed the results")
        results.append((ms, tuning))
        if verbose:
            print(f"  {tuning}: {ms:.4f} ms", flush=True)
    ms, best = min(results, key=lambda r: r[0])
    if cache_path:
        with _lock:
            data = _load(cache_path)
            data[key] = {"tuning": best, "ms": ms,
                         "timed": [{"tuning": t, "ms": m} for m, t in results]}
            _store(cache_path, data)
    return dict(best)


def plan_for(tasks, offsets, dma, cache_path: str | None = DEFAULT_CACHE, **kw) -> tm.Plan:
    """A tm.Plan with the tuned knobs for this batch shape."""
    return tm.Plan(offsets, **tune(tasks, offsets, dma, cache_path=cache_path, **kw))

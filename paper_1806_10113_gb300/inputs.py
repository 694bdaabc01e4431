"""Seeded synthetic task groups.

This module draws durations and nothing else: it holds none of the model's
arithmetic, so both the CUDA path and the CPU oracle can be fed from it.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014).  Group g of a workload with seed s draws
from its own stream seeded with ``s ^ (g * 0x9E3779B97F4A7C15 mod 2**64)``.
Integers in [a, b] are drawn by rejection (no modulo bias); log-uniform
values are ``round(exp(U(ln lo, ln hi)))`` with U built from the top 53 bits
of one draw.

Task classes follow the paper's definition (Sec. 4.3): a task is dominant
kernel (DK) when HtD + DtH <= K, otherwise dominant transfer (DT).

All durations are int32 nanoseconds.  A batch is returned as
``tasks`` int32 [T, 3] (HtD, K, DtH per row, groups concatenated),
``offsets`` int32 [G + 1] and ``dma`` int32 [G] (DMA engines per group).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

M64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15


class SplitMix64:
    """SplitMix64 as published (state += golden gamma, then the mix13 finaliser)."""

    def __init__(self, seed: int):
        self.state = seed & M64

    def next_u64(self) -> int:
        self.state = (self.state + GOLDEN) & M64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
        return z ^ (z >> 31)

    def uniform_int(self, a: int, b: int) -> int:
        """Uniform integer in [a, b] (inclusive) by rejection."""
        r = b - a + 1
        limit = (1 << 64) - ((1 << 64) % r)
        while True:
            x = self.next_u64()
            if x < limit:
                return a + x % r

    def uniform01(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def log_uniform_int(self, lo: int, hi: int) -> int:
        u = self.uniform01()
        v = math.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))
        return min(hi, max(lo, int(math.floor(v + 0.5))))


def group_stream(seed: int, g: int) -> SplitMix64:
    return SplitMix64(seed ^ ((g * GOLDEN) & M64))


@dataclass
class Batch:
    tasks: np.ndarray             # int32 [T, 3]
    offsets: np.ndarray           # int32 [G + 1]
    dma: np.ndarray               # int32 [G]
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def G(self) -> int:
        return int(self.offsets.shape[0] - 1)

    def sizes(self) -> np.ndarray:
        return np.diff(self.offsets)

    def group(self, g: int) -> np.ndarray:
        return self.tasks[self.offsets[g]:self.offsets[g + 1]]


def make_batch(groups, dma, name="", meta=None) -> Batch:
    sizes = [len(t) for t in groups]
    offsets = np.zeros(len(groups) + 1, dtype=np.int32)
    offsets[1:] = np.cumsum(sizes, dtype=np.int64)
    if groups:
        tasks = np.ascontiguousarray(np.concatenate(
            [np.asarray(t, dtype=np.int32).reshape(-1, 3) for t in groups]))
    else:
        tasks = np.zeros((0, 3), dtype=np.int32)
    return Batch(tasks, offsets, np.ascontiguousarray(np.asarray(dma, dtype=np.int32)),
                 name, meta or {})


def duplicate_for_models(b: Batch, models=(2, 1)) -> Batch:
    """The same groups once per device model (two DMA engines, then one)."""
    groups = [b.group(g) for g in range(b.G)] * len(models)
    dma = np.repeat(np.asarray(models, dtype=np.int32), b.G)
    return make_batch(groups, dma, b.name, dict(b.meta, models=list(models)))


# ---- per-task recipes --------------------------------------------------------

def uniform_task(rng: SplitMix64, h, k, d):
    return [rng.uniform_int(*h), rng.uniform_int(*k), rng.uniform_int(*d)]


def log_uniform_task(rng: SplitMix64, dominant_kernel: bool, lo=10_000, hi=10_000_000):
    """Log-uniform HtD, K, DtH, redrawn until the task has the wanted class."""
    while True:
        h = rng.log_uniform_int(lo, hi)
        k = rng.log_uniform_int(lo, hi)
        d = rng.log_uniform_int(lo, hi)
        if (h + d <= k) == dominant_kernel:
            return [h, k, d]


# ---- the paper-shaped workloads ---------------------------------------------

def single_group_uniform(n=6, seed=0, lo=50_000, hi=2_000_000, dma=2) -> Batch:
    """One group, n tasks, every duration uniform on [lo, hi] ns.

    n = 6, seed 0 is the small case: 720 orders, in the 1-8 ms range of the
    paper's synthetic tasks (Table 2)."""
    rng = group_stream(seed, 0)
    tasks = [uniform_task(rng, (lo, hi), (lo, hi), (lo, hi)) for _ in range(n)]
    return make_batch([tasks], [dma], f"single_n{n}_seed{seed}")


def dk_dt_groups(groups=64, n=10, seed=1, models=(2, 1)) -> Batch:
    """Half dominant-kernel, half dominant-transfer groups (Sec. 4.3 classes).

    DK groups: K ~ U[1M, 5M] ns, HtD and DtH ~ U[50k, 500k] ns.
    DT groups: HtD and DtH ~ U[1M, 5M] ns, K ~ U[50k, 500k] ns.
    Every group is evaluated once per device model in `models`."""
    base = []
    for g in range(groups):
        rng = group_stream(seed, g)
        if g < groups // 2:
            tasks = [uniform_task(rng, (50_000, 500_000), (1_000_000, 5_000_000),
                                  (50_000, 500_000)) for _ in range(n)]
        else:
            tasks = [uniform_task(rng, (1_000_000, 5_000_000), (50_000, 500_000),
                                  (1_000_000, 5_000_000)) for _ in range(n)]
        base.append(tasks)
    b = make_batch(base, [models[0]] * groups, f"dkdt_g{groups}_n{n}_seed{seed}")
    return duplicate_for_models(b, models)


def ragged_mixed(groups=8192, nmin=4, nmax=9, seed=2) -> Batch:
    """Ragged groups, n ~ U{nmin..nmax}; each task DK or DT with p = 1/2,
    durations log-uniform on [1e4, 1e7] ns (the 0.01-14.58 ms command range
    of the paper's real tasks, Table 5).  Even groups use two DMA engines,
    odd groups one."""
    out, dma = [], []
    for g in range(groups):
        rng = group_stream(seed, g)
        n = rng.uniform_int(nmin, nmax)
        out.append([log_uniform_task(rng, rng.uniform_int(0, 1) == 1) for _ in range(n)])
        dma.append(2 if g % 2 == 0 else 1)
    return make_batch(out, dma, f"ragged_g{groups}_n{nmin}-{nmax}_seed{seed}")


def half_dk_half_dt(groups=32, n=12, seed=3, models=(2,)) -> Batch:
    """Groups of n tasks, the first n/2 DK and the rest DT, log-uniform
    durations as in `ragged_mixed`."""
    base = []
    for g in range(groups):
        rng = group_stream(seed, g)
        base.append([log_uniform_task(rng, i < n // 2) for i in range(n)])
    b = make_batch(base, [models[0]] * groups, f"halfdkdt_g{groups}_n{n}_seed{seed}")
    return duplicate_for_models(b, models) if len(models) > 1 else b


def chained_groups(groups=4096, workers=4, rounds=4, seed=7) -> Batch:
    """Chained groups (the experiment setup of Sec. 6.1): `workers` workers
    each with a chain of `rounds` tasks, task r * workers + w being worker
    w's round-r task; each task DK or DT with p = 1/2, log-uniform durations
    as in `ragged_mixed`; even groups two DMA engines, odd groups one.  The
    batch's meta holds the workers per group."""
    out, dma = [], []
    for g in range(groups):
        rng = group_stream(seed, g)
        out.append([log_uniform_task(rng, rng.uniform_int(0, 1) == 1)
                    for _ in range(workers * rounds)])
        dma.append(2 if g % 2 == 0 else 1)
    return make_batch(out, dma, f"chain_g{groups}_t{workers}_r{rounds}_seed{seed}",
                      {"workers": np.full(groups, workers, dtype=np.int32)})


def random_small(seed: int, n: int, lo: int = 0, hi: int = 9, dma: int = 2) -> Batch:
    """A tiny group with small integer durations, for brute-force checks."""
    rng = group_stream(seed, n)
    tasks = [uniform_task(rng, (lo, hi), (lo, hi), (lo, hi)) for _ in range(n)]
    return make_batch([tasks], [dma], f"small_n{n}_seed{seed}")


def random_groups(seed: int, sizes, lo=0, hi=2_000_000, dma=None) -> Batch:
    """Ragged groups of the given sizes, durations uniform on [lo, hi]."""
    groups = []
    for g, n in enumerate(sizes):
        rng = group_stream(seed, g)
        groups.append([uniform_task(rng, (lo, hi), (lo, hi), (lo, hi)) for _ in range(int(n))])
    if dma is None:
        dma = [2 if g % 2 == 0 else 1 for g in range(len(groups))]
    return make_batch(groups, np.broadcast_to(np.asarray(dma), (len(groups),)),
                      f"random_seed{seed}")


# Table 2 of the paper: synthetic tasks as fractions of a 10 ms time unit,
# here in integer nanoseconds (HtD, K, DtH).
TABLE2_MS = {
    "T0": (1, 8, 1), "T1": (2, 7, 1), "T2": (3, 6, 1), "T3": (1, 7, 2),
    "T4": (6, 2, 2), "T5": (2, 2, 6), "T6": (4, 2, 4), "T7": (8, 1, 1),
}
# Table 3: the five synthetic benchmarks (X = percentage of DK tasks).
TABLE3 = {
    "BK0": ("T6", "T7", "T4", "T5"),
    "BK25": ("T0", "T4", "T6", "T7"),
    "BK50": ("T0", "T1", "T4", "T5"),
    "BK75": ("T0", "T1", "T2", "T4"),
    "BK100": ("T0", "T1", "T2", "T3"),
}


def table2_tasks(names, unit_ns=1_000_000) -> np.ndarray:
    return np.asarray([[v * unit_ns for v in TABLE2_MS[x]] for x in names], dtype=np.int32)


# ---- large training sets (vectorised) -----------------------------------------

def _splitmix_at(keys: np.ndarray, idx: np.ndarray) -> np.ndarray:
    """SplitMix64 output number idx (0-based) of the stream seeded with key:
    the state after idx + 1 steps is key + (idx + 1) * golden, then mix13."""
    with np.errstate(over="ignore"):
        z = keys.astype(np.uint64) + (idx.astype(np.uint64) + np.uint64(1)) * np.uint64(GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def _log_uniform_vec(u64: np.ndarray, lo: int, hi: int) -> np.ndarray:
    u = (u64 >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))
    v = np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))
    return np.clip(np.floor(v + 0.5), lo, hi).astype(np.int64)


def training_groups(groups: int, nmin: int = 6, nmax: int = 10, seed: int = 5,
                    lo: int = 10_000, hi: int = 10_000_000) -> Batch:
    """Many ragged groups drawn like `ragged_mixed` (n ~ U{nmin..nmax}, each
    task DK or DT with p = 1/2, log-uniform durations on [lo, hi] redrawn
    until the class matches, two DMA engines on even groups, one on odd),
    vectorised with numpy.  Group g reads its stream (key seed ^ g * golden)
    at fixed positions: number 0 gives n (as floor(u * r / 2^64), bias below
    2^-59), number 1 + i the class of task i (top bit), and numbers
    64 + 4096 i + 3 a + c the c-th duration of attempt a of task i."""
    g = np.arange(groups, dtype=np.uint64)
    with np.errstate(over="ignore"):
        keys = np.uint64(seed & M64) ^ (g * np.uint64(GOLDEN))
    r = nmax - nmin + 1
    u = _splitmix_at(keys, np.zeros(groups, dtype=np.uint64))
    # floor(u * r / 2^64) from the top 32 bits (exact enough for r < 2^16)
    n = nmin + (((u >> np.uint64(32)) * np.uint64(r)) >> np.uint64(32)).astype(np.int64)
    offsets = np.zeros(groups + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(n)
    T = int(offsets[-1])
    gid = np.repeat(np.arange(groups), n)
    tid = np.arange(T) - offsets[gid]
    tkeys = keys[gid]
    dk = (_splitmix_at(tkeys, (1 + tid).astype(np.uint64)) >> np.uint64(63)) == 1
    out = np.zeros((T, 3), dtype=np.int64)
    todo = np.arange(T)
    a = 0
    while todo.size:
        if a >= 1365:
            raise RuntimeError("class rejection did not settle")
        base = (64 + 4096 * tid[todo] + 3 * a).astype(np.uint64)
        vals = [_log_uniform_vec(_splitmix_at(tkeys[todo], base + np.uint64(c)), lo, hi)
                for c in range(3)]
        ok = ((vals[0] + vals[2]) <= vals[1]) == dk[todo]
        for c in range(3):
            out[todo[ok], c] = vals[c][ok]
        todo = todo[~ok]
        a += 1
    dma = np.where(np.arange(groups) % 2 == 0, 2, 1).astype(np.int32)
    return Batch(np.ascontiguousarray(out.astype(np.int32)), offsets.astype(np.int32), dma,
                 f"train_g{groups}_n{nmin}-{nmax}_seed{seed}")

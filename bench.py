"""Benchmark: orders evaluated per second by the exhaustive search, plus the
heuristic, over 64 groups of 10 tasks (half dominant-kernel, half
dominant-transfer) under both device models (one and two DMA engines).

One step = the whole hot path over that batch: for each of the 128 group
evaluations, every one of the 10! = 3,628,800 orders is evaluated with the
temporal execution model and reduced to best / worst / sum / mean with the
first best / worst order, and the reordering heuristic (Algorithm 1) picks an
order.  128 x 10! = 464,486,400 orders per step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl tm|reference]

Prints one JSON line (rank 0).  `value` is device-timed with inputs resident
in HBM; `e2e` goes through the host-pointer C ABI with host<->device copies
inside the timed region.  `--impl reference` times the CPU oracle on the
host cores on a bounded sample of the same workload.

At one GPU the default run also measures, each with its own clocks, the
metric's other clauses and the chained-task search as extra keys: `n12`
(orders/s of the 12-task exhaustive search), `learned` (task groups
scheduled/s by the learned path on 12-task groups, with the gap to the
exhaustive optimum timed in the same run, the ranker trained in the run) and
`chain` (orders/s of the search over chained tasks).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1806_10113_gb300 import inputs  # noqa: E402

METRIC = "orderings evaluated/s (exact model, N=10/12); task groups scheduled/s at <=1% gap"
UNIT = "orders/s"
GROUPS, N_TASKS, SEED = 64, 10, 1
WORKLOADS = {
    "dkdt64x10": ("64 groups x 10 tasks (32 dominant-kernel: K~U[1M,5M] ns, HtD/DtH~U[50k,500k]; "
                  "32 dominant-transfer: reverse), seed 1, each under 1 and 2 DMA engines: "
                  "exhaustive 10! orders + heuristic per group"),
    "single6": ("1 group x 6 tasks, durations U[50k,2M] ns, seed 0, two DMA engines: exhaustive 720 "
                "orders + heuristic in one host-pointer call (tm_schedule_batch), one group per "
                "call (latency)"),
    "dkdt32x12": ("32 groups x 12 tasks (half dominant-kernel, half dominant-transfer tasks in each, "
                  "log-uniform [1e4,1e7] ns), seed 3, each under 2 and 1 DMA engines: exhaustive "
                  "12! orders + heuristic per group (64 x 479,001,600 orders per step)"),
    "ragged8192": ("8192 ragged groups, n~U{4..9}, each task dominant-kernel or dominant-transfer "
                   "(p=1/2), durations log-uniform [1e4,1e7] ns, seed 2, DMA engines alternating "
                   "2/1: exhaustive n! orders + heuristic per group"),
    "beam12": ("2048 groups x 12 tasks (6 dominant-kernel + 6 dominant-transfer, log-uniform "
               "[1e4,1e7] ns, seed 3), each under 2 and 1 DMA engines: learned beam search "
               "(width 4; ranker trained on 2M exhaustively labelled groups, n~U{6..10}) "
               "vs the exhaustive optimum"),
    "overlap10": ("16 groups x 10 tasks (8 dominant-kernel: K~U[1M,5M] ns, HtD/DtH~U[50k,500k]; "
                  "8 dominant-transfer: reverse), seed 1, two DMA engines whose concurrent "
                  "transfers each run at 2/3 speed (partial-overlap model): exhaustive 10! orders "
                  "per group, every order simulated"),
    "chain4x4": ("4096 chained groups: 4 workers x 4 dependent tasks (Sec. 6.1 experiment setup), "
                 "each task dominant-kernel or dominant-transfer (p=1/2), log-uniform [1e4,1e7] ns, "
                 "seed 7, DMA engines alternating 2/1: exhaustive (4!)^4 = 331,776 orders per group"),
    "heuristic1m": ("1,048,576 ragged groups, n~U{4..16}, each task dominant-kernel or dominant-"
                    "transfer (p=1/2), log-uniform [1e4,1e7] ns, seed 6, DMA engines alternating: "
                    "the reordering heuristic (Algorithm 1) for every group"),
    "serve20k": ("Poisson arrivals at 20k groups/s for 5 s, n~U{4..16}, each task dominant-kernel "
                 "or dominant-transfer (p=1/2), log-uniform [1e4,1e7] ns, seed 4, DMA engines "
                 "alternating 2/1: served one by one by the continuous-batching server "
                 "(exhaustive optimum up to 12 tasks, learned beam 64 above)"),
}
WORKLOAD = WORKLOADS["dkdt64x10"]
# Integer operations per evaluated order, as the plain method counts them:
# 5 per recurrence step (3 adds, 2 maxes) times ~e tree nodes per order with
# prefix sharing, plus 4 for the reduction.
STEPWISE_OPS_PER_ORDER = 5 * math.e + 4


def method_ops_per_order(n: int) -> float:
    """Integer operations per order that the implemented method needs.

    The last four positions hold a set S; the makespan is
    max(d + alpha_S, k + beta_sigma, gamma_sigma), so each order costs one
    add and two maxes, plus one min and one add for the reductions (5).  Per
    prefix of the other P = n - 4 tasks: d + alpha, the prefix maximum
    (1 add, 2 maxes) and the 64-bit sum (2): 6, shared by 24 orders.  The
    prefixes are walked depth-first at 5 operations per tree node.  The
    suffix tables cost 24 orders x 2 chains x 4 steps x 5 per subset, shared
    by P! x 24 orders."""
    P = n - 4
    nodes = sum(math.factorial(P) // math.factorial(P - i) for i in range(1, P + 1))
    per_prefix = 6 + 5 * nodes / math.factorial(P)
    return 5 + per_prefix / 24 + 960 / (math.factorial(P) * 24)


def dominance_ops_per_order(n: int, full: float) -> float:
    """Integer operations per order of walk modes 5 to 8 (tm_tuning.unroll), where
    a fraction `full` of the prefixes had their 24 orders evaluated one by one
    (tm_plan_walk_counts) and the others took the closed forms.

    Per prefix, the dominance test: k + bmin, d + alpha, k + bmax, the
    maximum of k + bmax and cmax, six compares, two ors (12).  A dominated
    prefix then takes two selects for its minimum, two for its maximum, the
    sum 24 c0 or 24 k + sum(beta) (2) and a select between those and
    sum(gamma) (2), the item minimum and maximum (2) and the 64-bit sum (2):
    12.  Any other prefix costs what method_ops_per_order counts (the 24
    orders at 5 and the prefix's 6, of which d + alpha and k + bmax are the
    test's: 124).  The walk and the suffix tables as in method_ops_per_order."""
    P = n - 4
    nodes = sum(math.factorial(P) // math.factorial(P - i) for i in range(1, P + 1))
    per_prefix = 5 * nodes / math.factorial(P) + 12 + (1.0 - full) * 12 + full * 124
    return per_prefix / 24 + 960 / (math.factorial(P) * 24)


ALG_OPS_PER_ORDER = method_ops_per_order(N_TASKS)
SM_COUNT = 152
SM_MAX_MHZ = 2070.0
# Issue-limited int32 peak: 4 schedulers x 32 lanes per SM per clock.
INT32_PEAK_TOPS = SM_COUNT * 4 * 32 * SM_MAX_MHZ * 1e6 / 1e12
PROFILE = os.path.join(ROOT, "profiles", "exhaustive_enum_kernel_n10_g128.md")
L2_FLUSH_BYTES = 256 << 20


def workload(rank: int = 0, name: str = "dkdt64x10"):
    if name == "dkdt32x12":
        return inputs.half_dk_half_dt(groups=32, n=12, seed=3 + 1000 * rank, models=(2, 1))
    if name == "ragged8192":
        return inputs.ragged_mixed(groups=8192, seed=2 + 1000 * rank)
    return inputs.dk_dt_groups(groups=GROUPS, n=N_TASKS, seed=SEED + 1000 * rank)


def ops_per_order(b, full=None) -> float:
    """method_ops_per_order weighted by each group's orders (groups n >= 4);
    with `full` (walk modes 5 to 8: the fraction of prefixes evaluated order by
    order, over the whole batch), dominance_ops_per_order instead."""
    f = (lambda n: method_ops_per_order(n)) if full is None else \
        (lambda n: dominance_ops_per_order(n, full))
    w = [(math.factorial(int(n)), f(int(n))) for n in b.sizes() if n >= 4]
    return sum(a * o for a, o in w) / max(1, sum(a for a, _ in w))


def walk_basis(plan, tuning) -> tuple:
    """(fraction of prefixes evaluated order by order in the plan's last run,
    or None outside walk modes 5 to 8; a one-line statement of the count's basis)."""
    mode = int(tuning.get("unroll", 0))
    if mode < 5:
        return None, "max-plus suffix decomposition (see method_ops_per_order)"
    pre, full = plan.walk_counts()
    f = full / pre if pre else 1.0
    return f, (f"walk mode {mode}: {full} of {pre} prefixes ({100 * f:.1f}%) evaluated order by "
               "order, the rest by closed forms (see dominance_ops_per_order)")


def orders_per_step(b) -> int:
    return int(sum(math.factorial(int(n)) for n in b.sizes()))


# ---- distributed helpers --------------------------------------------------------

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def dist_init(backend: str):
    ws, rank, _ = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group(backend=backend)
        return dist
    return None


def max_over_ranks(dist, value: float, device=None) -> float:
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(dist, value: float, device=None) -> float:
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ---- clocks during the timed region ----------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id: str | None):
        self.bus_id = bus_id
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "50"]
        if self.bus_id:
            cmd += ["-i", self.bus_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "power_w_max": max(power), "reasons": sorted(reasons), "samples": len(sm)}


def bus_id_of(device_index: int) -> str | None:
    try:
        import torch
        p = torch.cuda.get_device_properties(device_index)
        return f"{p.pci_domain_id:08X}:{p.pci_bus_id:02X}:{p.pci_device_id:02X}.0"
    except Exception:
        return None


# ---- roofline inputs from the committed ncu summary --------------------------------

def kernel_source_hash() -> str:
    """Hash of the enumeration kernel's sources with comments and blank lines
    left out, so that a comment edit keeps the profiled traffic valid."""
    h = hashlib.sha256()
    for f in ("exhaustive.cu", "tm_device.cuh", "tm_internal.h"):
        with open(os.path.join(ROOT, "paper_1806_10113_gb300", "csrc", f)) as fh:
            text = re.sub(r"/\*.*?\*/", "", fh.read(), flags=re.S)
        for line in text.splitlines():
            code = line.split("//", 1)[0].rstrip()
            if code:
                h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per enumeration launch from the committed ncu summary, or
    None when the kernel source changed since that capture."""
    try:
        text = open(PROFILE).read()
    except OSError:
        return None
    m_hash = re.search(r"source_hash:\s*([0-9a-f]+)", text)
    m_bytes = re.search(r"dram_bytes_per_launch:\s*([0-9]+)", text)
    if not m_hash or not m_bytes or m_hash.group(1) != kernel_source_hash():
        return None
    return int(m_bytes.group(1))


# ---- CPU oracle timing ------------------------------------------------------------

def oracle_sample(b, items_per_group: int, nthreads: int = 0):
    """Times the oracle on the orders under `items_per_group` two-task
    prefixes of every group (8! = 40,320 orders each for n = 10)."""
    import oracle
    groups, prefixes = [], []
    for g in range(b.G):
        n = int(b.sizes()[g])
        k = 0
        for a in range(n):
            for c in range(n):
                if a != c and k < items_per_group:
                    groups.append(g)
                    prefixes.append((a, c))
                    k += 1
    t0 = time.perf_counter()
    oracle.exhaustive_prefixes(b.tasks, b.offsets, b.dma, groups, prefixes, nthreads)
    dt = time.perf_counter() - t0
    n_orders = sum(math.factorial(int(b.sizes()[g]) - 2) for g in groups)
    return n_orders, dt


def cpu_baseline(b, items_per_group: int = 2) -> dict:
    import oracle
    cores = oracle.hardware_threads()
    n_orders, dt = oracle_sample(b, items_per_group)
    return {"value": n_orders / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": (f"{items_per_group} two-task prefixes x (n-2)! orders of each of the "
                       f"{b.G} group evaluations ({n_orders} orders, event-driven "
                       f"simulation per order, {cores} threads, {dt:.2f} s)")}


def reference_step(b, group_idx, cores):
    """One bounded sample: the orders under the first two-task prefix of
    `cores` consecutive group evaluations (8! orders each, one per thread)."""
    import oracle
    groups = [(group_idx + i) % b.G for i in range(cores)]
    prefixes = [(0, 1)] * len(groups)
    t0 = time.perf_counter()
    oracle.exhaustive_prefixes(b.tasks, b.offsets, b.dma, groups, prefixes, cores)
    dt = time.perf_counter() - t0
    return sum(math.factorial(int(b.sizes()[g]) - 2) for g in groups), dt


def _reference_arm(name: str, cores: int):
    """The oracle's side of each workload: (line fields, step).  step(k)
    runs the k-th bounded sample on the host cores and returns (units, s);
    the units are those of the workload's own metric."""
    import oracle
    if name == "ragged8192":
        b = workload(0, name)
        fields = {"metric": METRIC, "unit": UNIT, "higher_is_better": True, "dtype": "int64",
                  "each_step": f"the (n-2)! orders under each of two two-task prefixes of "
                               f"every group, on {cores} host threads"}
        return fields, lambda k: oracle_sample(b, 2)
    if name in ("dkdt64x10", "dkdt32x12"):
        b = workload(0, name)
        fields = {"metric": METRIC, "unit": UNIT, "higher_is_better": True, "dtype": "int64",
                  "each_step": f"the (n-2)! orders under one two-task prefix of {cores} group "
                               "evaluations, one per host thread"}
        return fields, lambda k: reference_step(b, k * cores, cores)
    if name == "beam12":
        b = inputs.half_dk_half_dt(2048, 12, seed=3, models=(2, 1))

        def step(k):   # the exact optimum: groups = orders / 12!
            n, dt = reference_step(b, k * cores, cores)
            return n / math.factorial(12), dt
        fields = {"metric": "task groups scheduled/s at <=1% gap (learned beam, n=12)",
                  "unit": "groups/s", "higher_is_better": True, "dtype": "int64",
                  "each_step": f"the exact search (gap 0): 10! orders under one two-task "
                               f"prefix of {cores} groups, counted as 1/132 group each"}
        return fields, step
    if name == "overlap10":
        b = inputs.dk_dt_groups(16, 10, seed=1, models=(2,))

        def step(k):
            rng = np.random.default_rng(k)
            picks = [(int(rng.integers(b.G)), rng.permutation(10)) for _ in range(5000)]
            t0 = time.perf_counter()
            for g, o in picks:
                oracle.predict_overlap(b.group(g), o, 2, 2, 3)
            return len(picks), time.perf_counter() - t0
        fields = {"metric": "orderings evaluated/s (partial-overlap model, N=10, exhaustive)",
                  "unit": "orders/s", "higher_is_better": True, "dtype": "int64",
                  "each_step": "5000 random orders of the same groups, one oracle."
                               "predict_overlap call each, one host thread"}
        return fields, step
    if name == "heuristic1m":
        b = inputs.training_groups(1 << 20, 4, 16, seed=6)
        per = 1 << 15

        def step(k):
            g0 = (k * per) % (b.G - per)
            off = b.offsets[g0:g0 + per + 1]
            t0 = time.perf_counter()
            oracle.heuristic_batch(b.tasks[off[0]:off[-1]], off - off[0], b.dma[g0:g0 + per])
            return per, time.perf_counter() - t0
        fields = {"metric": "task groups scheduled/s (reordering heuristic, Algorithm 1)",
                  "unit": "groups/s", "higher_is_better": True, "dtype": "int64",
                  "each_step": f"{per} consecutive groups, oracle heuristic on {cores} threads"}
        return fields, step
    if name == "chain4x4":
        b = inputs.chained_groups(4096, 4, 4, seed=7)
        w = b.meta["workers"]
        per = 4

        def step(k):
            g0 = (k * per) % (b.G - per)
            off = b.offsets[g0:g0 + per + 1]
            t0 = time.perf_counter()
            oracle.exhaustive_chain_batch(b.tasks[off[0]:off[-1]], off - off[0], w[g0:g0 + per],
                                          b.dma[g0:g0 + per])
            return per * math.factorial(4) ** 4, time.perf_counter() - t0
        fields = {"metric": "orderings evaluated/s (exact model, chained tasks)", "unit": UNIT,
                  "higher_is_better": True, "dtype": "int64",
                  "each_step": f"every order of {per} consecutive groups, oracle on {cores} "
                               "host threads"}
        return fields, step
    if name == "single6":
        b = inputs.single_group_uniform(n=6, seed=0)

        def step(k):
            t0 = time.perf_counter()
            for _ in range(20):
                oracle.exhaustive(b.tasks, 2)
                oracle.heuristic(b.tasks, 2)
            return 20, time.perf_counter() - t0
        fields = {"metric": "schedule latency of one 6-task group (exhaustive 720 orders + "
                            "heuristic)", "unit": "us", "higher_is_better": False,
                  "dtype": "int64", "each_step": "20 calls of oracle exhaustive + heuristic "
                                                "on the group, one host thread"}
        return fields, step
    return None, None


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    cores = oracle.hardware_threads()
    fields, step = _reference_arm(args.workload, cores)
    if step is None:
        print(json.dumps({"impl": "reference", "unavailable":
                          f"the oracle has no serving loop: one {args.workload} group of up to "
                          "16 tasks takes it seconds, far below the offered load"}))
        return 0
    for w in range(args.warmup):
        step(w)
    units, total_s = 0.0, 0.0
    for k in range(args.steps):
        n, dt = step(args.warmup + k)
        units += n
        total_s += dt
    value = units / total_s if fields["higher_is_better"] else 1e6 * total_s / units
    unit = fields["unit"]
    print(json.dumps({
        "impl": "reference", "metric": fields["metric"], "value": value, "unit": unit,
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * total_s / args.steps,
        "higher_is_better": fields["higher_is_better"],
        "scaling": "weak", "vs_baseline": None, "dtype": fields["dtype"], "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload] + f" (each step: {fields['each_step']})",
                   "l2": "n/a (host)"},
        "cpu_baseline": {"value": value, "unit": unit, "cores": cores, "kind": "oracle",
                         "sample": f"per step: {fields['each_step']}"},
        "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))
    return 0


# ---- the CUDA path ----------------------------------------------------------------

# ---- the metric's other clauses, measured in the default run ----------------------

# Learned path: beam width on the 12-task groups, and the beams (plus the
# heuristic's order) that start the exact descent.  Picked on held-out groups
# (seed 5): widths 4, 8 and 16 with 1, 2 or 4 starts all keep 99.78-99.83%
# of the groups within 1% of the optimum; width 4 with 2 starts is the fastest
# (7.8M groups/s against 4.7M at width 16 with 4 starts).
BEAM_WIDTH = 4
REFINE_STARTS = 2
CHAIN_WORKERS, CHAIN_ROUNDS, CHAIN_GROUPS = 4, 4, 4096


def timed_steps(step, K: int, flush=None):
    """Device time (ms) of each of K steps on the current stream, with the
    clocks sampled during them; `flush` (if given) runs before each step,
    outside the events."""
    import torch
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(K)]
    sampler = ClockSampler(bus_id_of(torch.cuda.current_device()))
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.2)
    for k in range(K):
        if flush is not None:
            flush()
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    return [a.elapsed_time(c) for a, c in ev], clocks


def n12_leg(args, log) -> dict:
    """Orders/s of the 12-task exhaustive search (N = 12 half of the metric):
    32 groups x 12 tasks under both device models, autotuned, one
    tm_schedule_batch_dev pass per step (search + heuristic), L2 flushed."""
    import torch
    from paper_1806_10113_gb300 import autotune, tm
    dev = torch.device("cuda")
    b = workload(0, "dkdt32x12")
    G, T = b.G, int(b.tasks.shape[0])
    n_orders = orders_per_step(b)
    tuning = autotune.tune(b.tasks, b.offsets, b.dma, cache_path=None, reps=5)
    plan = tm.Plan(b.offsets, **tuning)
    d_tasks, d_dma = torch.from_numpy(b.tasks).to(dev), torch.from_numpy(b.dma).to(dev)
    d_stats = torch.zeros(G * tm.STATS_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    d_status = torch.zeros(G, dtype=torch.int32, device=dev)
    d_orders = torch.zeros(T, dtype=torch.int32, device=dev)
    d_ms = torch.zeros(G, dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    step = lambda: tm.tm_schedule_batch_dev(plan, d_tasks, d_dma, d_stats, d_orders, d_ms, d_status)
    for _ in range(args.warmup):
        step()
    K = 20
    ek = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(K)]
    for a, c in ek:          # torch creates an event on its first record
        a.record()
        c.record()
    # value steps without the timing hook; then the kernel alone in K more
    ms, clocks = timed_steps(step, K, flush=flush.zero_)
    for a, c in ek:
        flush.zero_()
        plan.set_timing(a, c)
        step()
    plan.set_timing(None, None)
    torch.cuda.synchronize()
    if (d_status.cpu().numpy() != 0).any():
        raise RuntimeError("12-task workload: device status errors")
    full, basis = walk_basis(plan, tuning)
    plan.close()
    step_s = statistics.mean(ms) / 1000.0
    enum_s = statistics.mean(a.elapsed_time(c) for a, c in ek) / 1000.0
    ops = ops_per_order(b, full)
    achieved = ops * n_orders / enum_s / 1e12
    log(f"n12: {n_orders / step_s:.3e} orders/s")
    return {"workload": WORKLOADS["dkdt32x12"], "value": n_orders / step_s, "unit": UNIT,
            "ms_per_step": 1000 * step_s, "steps": K, "orders_per_step": n_orders,
            "groups_per_s": G / step_s, "tuning": tuning,
            "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MiB write)",
            "roofline": {"bound": "alu", "achieved": achieved, "peak": INT32_PEAK_TOPS,
                         "unit": "Tops/s (int32)", "frac": achieved / INT32_PEAK_TOPS,
                         "kernel": "enum_kernel (exhaustive enumeration)",
                         "kernel_ms": 1000 * enum_s, "ops_per_order": round(ops, 3),
                         "ops_basis": basis, "traffic": None},
            "clocks": clocks}


def learned_leg(args, log) -> dict:
    """Task groups scheduled/s at <= 1% gap (the metric's second clause): the
    ranker is trained in this run (2M exhaustively labelled groups of 6..10
    tasks, 3 epochs, all on the GPU), then the learned path -- beam search
    with the ranker's proposals, the exact model judging, the heuristic's
    order as a start, the exact-model descent from the best beams and the
    heuristic -- schedules 2048 twelve-task groups under both device models,
    against the exhaustive optimum of the same groups timed in the same run."""
    import torch
    from paper_1806_10113_gb300 import learn, tm
    ranker, train_info = trained_ranker(args, log)
    test = inputs.half_dk_half_dt(2048, 12, seed=3, models=(2, 1))
    G, T = test.G, int(test.tasks.shape[0])
    d_tasks, d_offsets, d_devs = learn.to_device(test)
    # the exhaustive optimum of every test group, timed (the plain GPU search)
    d_stats = torch.zeros(G * tm.STATS_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    warm = tm.Plan(test.offsets[:9])
    tm.tm_exhaustive_batch_dev(warm, d_tasks, d_devs, d_stats)
    plan = tm.Plan(test.offsets, pdmax=5)
    ex_ms, _ = timed_steps(lambda: tm.tm_exhaustive_batch_dev(plan, d_tasks, d_devs, d_stats), 2)
    best = learn.stats_host(d_stats, G)["best"].astype(np.int64)
    plan.close()
    warm.close()
    ex_s = min(ex_ms) / 1000.0
    d_orders = torch.zeros(T, dtype=torch.int32, device="cuda")
    d_ms = torch.zeros(G, dtype=torch.int32, device="cuda")
    d_won = torch.zeros(G, dtype=torch.int32, device="cuda")
    step = lambda: tm.tm_beam_batch_dev(ranker, d_tasks, d_offsets, test.offsets, d_devs,
                                        BEAM_WIDTH, d_orders, d_ms, d_beam_won=d_won,
                                        refine_starts=REFINE_STARTS)
    for _ in range(args.warmup):
        step()
    ms, clocks = timed_steps(step, 20)
    step_s = statistics.mean(ms) / 1000.0
    got = d_ms.cpu().numpy().astype(np.int64)
    gap = (got - best) / best
    # the same search without the descent, for the ablation
    tm.tm_beam_batch_dev(ranker, d_tasks, d_offsets, test.offsets, d_devs, BEAM_WIDTH, d_orders,
                         d_ms)
    gap0 = (d_ms.cpu().numpy().astype(np.int64) - best) / best
    _, hms = tm.tm_heuristic_batch(test.tasks, test.offsets, test.dma)
    gaph = (hms.astype(np.int64) - best) / best
    within = float((gap <= 0.01).mean())
    log(f"learned: {G / step_s:.3e} groups/s, within 1% {within:.4f}")
    return {"workload": WORKLOADS["beam12"] + f"; exact-model descent from the best "
                        f"{REFINE_STARTS} beams and the heuristic's order",
            "metric": "task groups scheduled/s at <=1% gap", "value": G / step_s,
            "unit": "groups/s", "ms_per_step": 1000 * step_s, "steps": 20,
            "groups_within_1pct_per_s": within * G / step_s,
            "within_1pct": within, "optimal": float((gap == 0).mean()),
            "gap_mean": float(gap.mean()), "gap_p99": float(np.quantile(gap, 0.99)),
            "gap_max": float(gap.max()), "beam_won": float(d_won.float().mean()),
            "exhaustive_groups_per_s": G / ex_s,
            "speedup_vs_exhaustive": ex_s / step_s,
            "ablation": {"beam_only_within_1pct": float((gap0 <= 0.01).mean()),
                         "beam_only_gap_mean": float(gap0.mean()),
                         "heuristic_within_1pct": float((gaph <= 0.01).mean()),
                         "heuristic_gap_mean": float(gaph.mean())},
            "l2": "inputs < L2; no flush (ranker weights stay resident by design)",
            "clocks": clocks, "train": train_info}


def chain_ops_per_order(T: int, full: float = 1.0) -> float:
    """Integer operations per order of the chained search's tail, the part
    every order needs.  Four workers (the fast path): 16 recurrence steps
    for the first two positions (6 operations each: three maxima, three
    additions), then each order's last two positions in closed form,
    max(d + A, k + P, h + Q, R) (6 operations), R for each pair of orders (4)
    and its four E terms, and the reduction (7 per pair of orders: min, max,
    32-bit add, 64-bit add, two compares): 376 per 24 orders.  Otherwise the
    last m = min(T, 4) positions walked step by step (64 / 15 / 4 / 1 steps
    for m! = 24 / 6 / 2 / 1 orders) plus the same reduction (4 for a single
    order).  The head positions recomputed between blocks are not counted.
    With four workers a fraction 1 - `full` of the 24-order tails take the
    closed form where the HtD engine's path ends all 24 (tm_chain_tail_counts):
    every tail first costs the test (six differences, six compares, four
    ands: 16); a closed one then takes its minimum and maximum (2 adds, 2
    compares), 24 h + the table's sum (2) and the 64-bit sum (2): 8."""
    if T == 4:
        return (16 + full * (6 * 16 + 4 + 12 * 4 + 24 * 6 + 12 * 7) + (1.0 - full) * 8) / 24
    m = min(T, 4)
    steps = {4: 64, 3: 15, 2: 4, 1: 1}[m]
    red = {4: 12 * 7, 3: 3 * 7, 2: 7, 1: 4}[m]
    return (6 * steps + red) / math.factorial(m)


def chain_leg(args, log, groups: int = CHAIN_GROUPS, steps: int = 20) -> dict:
    """Orders/s of the chained-task search (Sec. 6.1 experiment setup):
    4096 groups of 4 workers x 4 dependent tasks, (4!)^4 = 331,776 orders
    each, one tm_exhaustive_chain_batch_dev call per step, L2 flushed."""
    import torch
    from paper_1806_10113_gb300 import tm
    dev = torch.device("cuda")
    b = inputs.chained_groups(groups, CHAIN_WORKERS, CHAIN_ROUNDS, seed=7)
    w = b.meta["workers"]
    G = b.G
    n_orders = G * math.factorial(CHAIN_WORKERS) ** CHAIN_ROUNDS
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    d_tasks, d_off, d_w, d_dma = d(b.tasks), d(b.offsets), d(w), d(b.dma)
    d_stats = torch.zeros(G * tm.STATS_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    d_status = torch.zeros(G, dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    step = lambda: tm.tm_exhaustive_chain_batch_dev(d_tasks, d_off, b.offsets, d_w, w, d_dma,
                                                    d_stats, d_status)
    for _ in range(args.warmup):
        step()
    ms, clocks = timed_steps(step, steps, flush=flush.zero_)
    torch.cuda.synchronize()
    if (d_status.cpu().numpy() != 0).any():
        raise RuntimeError("chained workload: device status errors")
    step_s = statistics.mean(ms) / 1000.0
    tails, closed = tm.tm_chain_tail_counts()   # of the last timed step
    full = 1.0 - closed / tails if tails else 1.0
    ops = chain_ops_per_order(CHAIN_WORKERS, full)
    achieved = ops * n_orders / step_s / 1e12
    log(f"chain: {n_orders / step_s:.3e} orders/s")
    return {"workload": (f"{G} chained groups: {CHAIN_WORKERS} workers x {CHAIN_ROUNDS} dependent "
                         f"tasks, each DK or DT (p=1/2), log-uniform [1e4,1e7] ns, seed 7, DMA "
                         f"engines alternating 2/1: exhaustive (T!)^N orders per group"),
            "value": n_orders / step_s, "unit": UNIT, "ms_per_step": 1000 * step_s, "steps": steps,
            "orders_per_step": n_orders,
            "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MiB write)",
            "roofline": {"bound": "alu", "achieved": achieved, "peak": INT32_PEAK_TOPS,
                         "unit": "Tops/s (int32)", "frac": achieved / INT32_PEAK_TOPS,
                         "kernel": "chain prep + enumeration + finalize (whole call)",
                         "ops_per_order": round(ops, 3),
                         "ops_basis": (f"{closed} of {tails} 24-order tails ({100 * (1 - full):.1f}%) "
                                       "in the closed form of the HtD engine's path, the rest "
                                       "order by order (see chain_ops_per_order)"),
                         "traffic": None},
            "clocks": clocks}


def run_chain(args):
    """The chained-task search alone (its own line; the default run carries
    the same measurement as the `chain` key)."""
    import torch
    torch.cuda.set_device(0)
    log = lambda m: print(m, file=sys.stderr, flush=True)
    leg = chain_leg(args, log, groups=args.groups or CHAIN_GROUPS, steps=min(args.steps, 50))
    out = {"metric": "orderings evaluated/s (exact model, chained tasks)", "n_gpus": 1,
           "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "int32", "data": "synthetic",
           "config": {"workload": leg.pop("workload"), "l2": leg.pop("l2")},
           "gpu_launches": 3 * leg["steps"], **leg}
    print(json.dumps(out))
    return 0


def run_tm(args):
    import torch
    from paper_1806_10113_gb300 import tm

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = dist_init("nccl")
    stream = torch.cuda.current_stream()

    b = workload(rank, args.workload)
    G, T = b.G, int(b.tasks.shape[0])
    n_orders = orders_per_step(b)
    d_tasks = torch.from_numpy(b.tasks).to(dev)
    d_offsets = torch.from_numpy(b.offsets).to(dev)
    d_dma = torch.from_numpy(b.dma).to(dev)
    d_stats = torch.zeros(G * tm.STATS_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    d_status = torch.zeros(G, dtype=torch.int32, device=dev)
    d_orders = torch.zeros(T, dtype=torch.int32, device=dev)
    d_ms = torch.zeros(G, dtype=torch.int32, device=dev)
    from paper_1806_10113_gb300 import autotune
    if args.tuning:
        vals = [int(x) for x in args.tuning.split(",")] + [0, 0, 0]
        tuning = dict(zip(("pdmax", "fuse_finalize", "blocks_per_sm", "item_cost",
                           "chunks_per_thread", "unroll"), vals[:6]))
    else:
        tuning = autotune.tune(b.tasks, b.offsets, b.dma, cache_path=None, reps=10)
    tm.tm_set_default_tuning(**tuning)          # also for the host-pointer (e2e) calls
    plan = tm.Plan(b.offsets, **tuning)
    launches_per_step = plan.launches()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    ek_capture = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    for e in ek_capture:
        e.record(stream)

    def step():
        tm.tm_schedule_batch_dev(plan, d_tasks, d_dma, d_stats, d_orders, d_ms, d_status, stream)

    if args.graph:
        # one CUDA-graph launch per step; the enumeration's timing events are
        # recorded inside the graph and swapped per step
        plan.set_timing(*ek_capture)
        plan.capture(d_tasks, d_dma, d_stats, d_orders, d_ms, d_status)
        plan.set_timing(None, None)

        def step():
            plan.graph_launch(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    status = d_status.cpu().numpy()
    if (status != 0).any():
        raise RuntimeError(f"device status errors: {status}")

    K = args.steps
    # the enumeration kernel's own time (roofline) comes from KE further
    # steps with the plan's timing hook; the value steps run without it, so
    # that the pass's launches follow each other directly (programmatic
    # dependent launch); a captured graph carries its events in every step
    KE = K if args.graph else min(K, 200)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(K)]
    ek = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(KE)]
    for a, c in ek:          # torch creates an event on its first record
        a.record(stream)
        c.record(stream)
    sampler = ClockSampler(bus_id_of(local))
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.2)
    wall0 = time.perf_counter()
    for k in range(K):
        flush.zero_()                        # evict L2 between timed steps
        if args.graph:
            plan.graph_set_timing(*ek[k])
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if dist is not None:
        dist.barrier()
    clocks = sampler.stop()
    if not args.graph:
        for k in range(KE):
            flush.zero_()
            plan.set_timing(*ek[k])
            step()
        torch.cuda.synchronize()
    plan.set_timing(None, None)
    step_ms = [a.elapsed_time(c) for a, c in ev]
    enum_ms = [a.elapsed_time(c) for a, c in ek]
    total_s = sum(step_ms) / 1000.0
    total_s = max_over_ranks(dist, total_s, dev)
    all_orders = sum_over_ranks(dist, float(n_orders * K), dev)
    value = all_orders / total_s

    # end to end through the host-pointer ABI: inputs from pinned host memory,
    # results read back every step
    h_tasks = torch.from_numpy(b.tasks).pin_memory().numpy()
    h_offsets = torch.from_numpy(b.offsets).pin_memory().numpy()
    h_dma = torch.from_numpy(b.dma).pin_memory().numpy()
    e2e_steps = max(3, min(K, 50))
    for _ in range(2):
        tm.tm_schedule_batch(h_tasks, h_offsets, h_dma)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        st, ho, hms = tm.tm_schedule_batch(h_tasks, h_offsets, h_dma)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e_s = max_over_ranks(dist, e2e_s, dev)
    # per call: tasks and device models in; stats, status, orders, makespans out
    h2d = h_tasks.nbytes + h_dma.nbytes
    d2h = st.nbytes + 4 * G + ho.nbytes + hms.nbytes

    ws_total = ws
    result = None
    full, basis = walk_basis(plan, tuning)
    if rank == 0:
        enum_avg_s = statistics.mean(enum_ms) / 1000.0
        ops_order = ops_per_order(b, full)
        alg_ops = ops_order * n_orders
        achieved = alg_ops / enum_avg_s / 1e12
        maxplus_achieved = ops_per_order(b) * n_orders / enum_avg_s / 1e12
        stepwise_achieved = STEPWISE_OPS_PER_ORDER * n_orders / enum_avg_s / 1e12
        traffic = profiled_traffic()
        rates = tm.tm_measure_int32_rates()
        result = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws_total, "steps": K,
            "warmup": args.warmup, "ms_per_step": 1000.0 * total_s / K,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload], "groups": G,
                       "orders_per_step": n_orders, "tuning": tuning,
                       "launch": "cuda graph" if args.graph else "stream",
                       "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MiB write)",
                       "parallelism": f"replicas x{ws_total}, no collective on the data path"},
            "groups_per_s": G * K * ws_total / total_s,
            "e2e": {"value": n_orders * ws_total / e2e_s, "unit": UNIT,
                    "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                    "ms_per_step": 1000 * e2e_s},
            "gpu_launches": launches_per_step * K,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": INT32_PEAK_TOPS,
                         "unit": "Tops/s (int32)", "frac": achieved / INT32_PEAK_TOPS,
                         "traffic": traffic,
                         "kernel": "enum_kernel (exhaustive enumeration)",
                         "kernel_ms": 1000 * enum_avg_s,
                         "ops_per_order": round(ops_order, 3),
                         "ops_basis": basis,
                         "maxplus_ops_per_order": round(ops_per_order(b), 3),
                         "maxplus_frac": maxplus_achieved / INT32_PEAK_TOPS,
                         "stepwise_ops_per_order": round(STEPWISE_OPS_PER_ORDER, 3),
                         "stepwise_frac": stepwise_achieved / INT32_PEAK_TOPS,
                         "peak_basis": "152 SMs x 128 int32 lanes/clk x 2070 MHz (derived)",
                         "measured_int32_tops": {k: v / 1e12 for k, v in rates.items()},
                         "measured_basis": "independent int32 max / add / max-then-add chains "
                                           "on every SM (tm_measure_int32_rates), after the "
                                           "timed region"},
            "clocks": clocks,
            "wall_s_timed": wall,
        }
        if ws_total == 1 and not args.no_cpu_baseline:
            result["cpu_baseline"] = cpu_baseline(b, 1 if args.workload == "dkdt32x12" else 2)
        if ws_total == 1 and args.workload == "dkdt64x10" and not args.no_secondary:
            log = lambda m: print(m, file=sys.stderr, flush=True)
            result["n12"] = n12_leg(args, log)
            result["learned"] = learned_leg(args, log)
            result["chain"] = chain_leg(args, log)
        print(json.dumps(result))
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    plan.close()
    return 0


# ---- learned beam and serving (secondary workloads) --------------------------------

FLOPS_PER_RANKER_ROW = 2 * (32 * 128 + 128 * 128 + 128 * 128 + 128)


def trained_ranker(args, log):
    from paper_1806_10113_gb300 import learn, tm
    ranker = tm.Ranker(seed=5)
    if args.ranker:
        ranker.set_params(np.load(args.ranker))
        return ranker, {"loaded": args.ranker}
    info = learn.train(ranker, groups=args.train_groups, epochs=3, seed=5, lr=2e-3, log=log)
    if args.ranker_out:
        np.save(args.ranker_out, ranker.get_params())
    return ranker, {k: info[k] for k in ("groups", "epochs", "losses", "label_s", "train_s")}


def run_beam12(args):
    import torch
    from paper_1806_10113_gb300 import learn, tm
    torch.cuda.set_device(0)
    log = lambda m: print(m, file=sys.stderr)
    ranker, train_info = trained_ranker(args, log)
    test = inputs.half_dk_half_dt(args.groups or 2048, 12, seed=3, models=(2, 1))
    G, T = test.G, int(test.tasks.shape[0])
    dev = learn.to_device(test)
    d_tasks, d_offsets, d_devs = dev
    # the exhaustive optimum, timed (one pass over all groups after a warm-up on a few)
    plan_small = tm.Plan(test.offsets[:9])
    d_stats = torch.zeros(G * 72, dtype=torch.uint8, device="cuda")
    tm.tm_exhaustive_batch_dev(plan_small, d_tasks, d_devs, d_stats)
    plan = tm.Plan(test.offsets, pdmax=5)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    tm.tm_exhaustive_batch_dev(plan, d_tasks, d_devs, d_stats)
    e1.record()
    torch.cuda.synchronize()
    ex_s = e0.elapsed_time(e1) / 1000.0
    best = learn.stats_host(d_stats, G)["best"].astype(np.int64)
    plan.close()
    # the beam search, device-timed over K steps
    d_orders = torch.zeros(T, dtype=torch.int32, device="cuda")
    d_ms = torch.zeros(G, dtype=torch.int32, device="cuda")
    d_won = torch.zeros(G, dtype=torch.int32, device="cuda")
    step = lambda: tm.tm_beam_batch_dev(ranker, d_tasks, d_offsets, test.offsets, d_devs,
                                        BEAM_WIDTH, d_orders, d_ms, d_beam_won=d_won,
                                        refine_starts=REFINE_STARTS)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    K = min(args.steps, 50)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(K)]
    sampler = ClockSampler(bus_id_of(0))
    sampler.start()
    time.sleep(0.2)
    for k in range(K):
        ev[k][0].record()
        step()
        ev[k][1].record()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    beam_s = statistics.mean(a.elapsed_time(c) for a, c in ev) / 1000.0
    ms = d_ms.cpu().numpy().astype(np.int64)
    gap = (ms - best) / best
    # e2e: inputs from pinned host memory, orders and makespans read back
    h_tasks = torch.from_numpy(test.tasks).pin_memory()
    h_off = torch.from_numpy(test.offsets).pin_memory()
    h_dma = torch.from_numpy(test.dma).pin_memory()
    o_orders = torch.empty(T, dtype=torch.int32).pin_memory()
    o_ms = torch.empty(G, dtype=torch.int32).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(5):
        d_tasks.copy_(h_tasks, non_blocking=True)
        d_offsets.copy_(h_off, non_blocking=True)
        d_devs.copy_(h_dma, non_blocking=True)
        step()
        o_orders.copy_(d_orders, non_blocking=True)
        o_ms.copy_(d_ms, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / 5
    # the ranker's forward kernel alone on the beam's row count, for its roofline
    chunk = 1 << 22   # 4M rows, a launch of the size the beam's chunks reach at width 16
    X = torch.zeros(chunk * 32, dtype=torch.int16, device="cuda")
    lg = torch.zeros(chunk, dtype=torch.float32, device="cuda")
    for _ in range(3):
        ranker.forward_dev(X, chunk, lg)
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record()
    for _ in range(10):
        ranker.forward_dev(X, chunk, lg)
    f1.record()
    torch.cuda.synchronize()
    fwd_s = f0.elapsed_time(f1) / 1000.0 / 10
    tflops = FLOPS_PER_RANKER_ROW * chunk / fwd_s / 1e12
    peak = measured_peak("bf16_tflops") or 1900.0
    out = {
        "metric": "task groups scheduled/s at <=1% gap (learned beam, n=12)",
        "value": G / beam_s, "unit": "groups/s", "n_gpus": 1, "steps": K,
        "warmup": args.warmup, "ms_per_step": 1000 * beam_s, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16 ranker, int32 model",
        "data": "synthetic",
        "config": {"workload": WORKLOADS["beam12"], "groups": G, "beam": BEAM_WIDTH,
                   "refine_starts": REFINE_STARTS,
                   "l2": "inputs < L2; no flush (ranker weights stay resident by design)"},
        "gap_mean": float(gap.mean()), "gap_p99": float(np.quantile(gap, 0.99)),
        "gap_max": float(gap.max()),
        "within_1pct": float((gap <= 0.01).mean()), "optimal": float((gap == 0).mean()),
        "beam_won": float(d_won.float().mean()),
        "exhaustive_groups_per_s": G / ex_s,
        "speedup_vs_exhaustive": (G / beam_s) / (G / ex_s),
        "e2e": {"value": G / e2e_s, "unit": "groups/s",
                "h2d_bytes_per_step": int(test.tasks.nbytes + test.offsets.nbytes + test.dma.nbytes),
                "d2h_bytes_per_step": int(4 * T + 4 * G)},
        "gpu_launches": 2 + 12 * 3 + 1,
        "roofline": {"bound": "tensor", "kernel": "forward_tc_kernel (ranker MLP, tcgen05 bf16, TMEM accumulator)",
                     "achieved": tflops, "peak": peak, "unit": "TFLOP/s",
                     "frac": tflops / peak, "traffic": None,
                     "basis": f"{FLOPS_PER_RANKER_ROW} FLOP per row, {chunk} rows per launch, "
                              "timed alone"},
        "clocks": clocks,
        "train": train_info,
    }
    print(json.dumps(out))
    return 0


def run_serve(args):
    import torch
    from paper_1806_10113_gb300 import tm
    torch.cuda.set_device(0)
    log = lambda m: print(m, file=sys.stderr)
    ranker, train_info = trained_ranker(args, log)
    rate, seconds = 20000.0, args.serve_seconds
    G = int(rate * seconds)
    b = inputs.training_groups(G, 4, 16, seed=4)
    rng = np.random.default_rng(4)
    arrivals = np.cumsum(rng.exponential(1e9 / rate, G)).astype(np.int64)
    srv = tm.Server(exact_max_n=args.exact_max_n, beam_width=BEAM_WIDTH, ranker=ranker, lanes=4,
                    lane_groups=1024, lane_subsets=1024 * 64, refine_starts=REFINE_STARTS)
    warm = min(G, 2000)
    srv.replay(b.tasks[:b.offsets[warm]], b.offsets[:warm + 1], b.dma[:warm],
               arrivals[:warm] - arrivals[0])
    sampler = ClockSampler(bus_id_of(0))
    sampler.start()
    time.sleep(0.2)
    t0 = time.perf_counter()
    res = srv.replay(b.tasks, b.offsets, b.dma, arrivals)
    wall = time.perf_counter() - t0
    clocks = sampler.stop()
    counters = srv.counters()
    srv.close()
    if (res["status"] != 0).any():
        raise RuntimeError("server reported errors")
    lat_ms = res["latency_ns"] / 1e6
    done_ns = arrivals + res["latency_ns"]
    span_s = (done_ns.max() - arrivals.min()) / 1e9
    meth = res["method"]
    sizes = b.sizes()
    _, h_ms = tm.tm_heuristic_batch(b.tasks, b.offsets, b.dma)
    gain = (h_ms.astype(np.int64) - res["makespan"]) / h_ms
    out = {
        "metric": "decision latency p99 at Poisson 20k groups/s (n~U{4..16})",
        "value": float(np.quantile(lat_ms, 0.99)), "unit": "ms", "n_gpus": 1,
        "steps": 1, "warmup": 1, "ms_per_step": 1000 * wall, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32 model, bf16 ranker",
        "data": "synthetic",
        "config": {"workload": WORKLOADS["serve20k"], "groups": G,
                   "exact_max_n": args.exact_max_n, "lanes": 4, "lane_groups": 1024,
                   "beam": BEAM_WIDTH, "refine_starts": REFINE_STARTS},
        "p50_ms": float(np.quantile(lat_ms, 0.5)), "p90_ms": float(np.quantile(lat_ms, 0.9)),
        "p99_ms": float(np.quantile(lat_ms, 0.99)), "max_ms": float(lat_ms.max()),
        "groups_per_s": G / span_s, "offered_groups_per_s": rate,
        "batches": counters["batches"], "mean_batch_groups": G / max(1, counters["batches"] - 1),
        "max_batch_groups": counters["max_batch_groups"],
        "methods": {"exhaustive": int((meth == 0).sum()), "beam": int((meth == 1).sum()),
                    "heuristic": int((meth == 2).sum())},
        "latency_by_size_ms": {
            str(n): {"p50": float(np.quantile(lat_ms[sizes == n], 0.5)),
                     "p99": float(np.quantile(lat_ms[sizes == n], 0.99))}
            for n in range(4, 17) if (sizes == n).any()},
        "gain_over_heuristic_mean": float(gain.mean()),
        "gain_over_heuristic_large_mean": float(gain[sizes > args.exact_max_n].mean()),
        "e2e": {"value": G / span_s, "unit": "groups/s",
                "h2d_bytes_per_step": int(b.tasks.nbytes + b.dma.nbytes),
                "d2h_bytes_per_step": int(res.nbytes)},
        "gpu_launches": None,
        "clocks": clocks,
        "train": train_info,
    }
    print(json.dumps(out))
    return 0


# Integer operations per event of the partial-overlap loop, counted from its
# body: readiness checks and starts (8), the speed choice (3), two exact
# ceiling divisions by an invariant rate (2 x 13), three candidate ends and
# their minimum (12), progress of three engines (15).  An order of n tasks
# has at most 3n events.
OVERLAP_OPS_PER_EVENT = 8 + 3 + 26 + 12 + 15
OVERLAP_RUN = 64            # consecutive ranks per enumeration thread
# One DtH of the closed-form tail: the kernels up to it (an add each, about
# one per DtH), the max with the DtH engine and the add of its duration, and
# the position bookkeeping (2).
OVERLAP_OPS_PER_TAIL = 1 + 2 + 2


def overlap_loop_events(t, order, num, den):
    """Events of the partial-overlap loop for one order until the last HtD
    ends (after that the kernel finishes in closed form), the event count
    reached when the HtD queue turns to each position (the enumeration
    kernel's resume points), the number of DtH left to the closed-form tail,
    and the makespan the same steps give (two DMA engines).  For counting:
    the bench's makespans come from the kernels."""
    n = len(order)
    ih = ik = idd = 0
    hb = kb = db = False
    hl = kl = dl = 0
    T = 0
    events, at = 0, [0] * n
    while ih < n:
        if not hb:
            at[ih] = events
            hb, hl = True, int(t[order[ih]][0]) * den
        if not kb and ik < ih:
            kb, kl = True, int(t[order[ik]][1])
        if not db and idd < ik:
            db, dl = True, int(t[order[idd]][2]) * den
        events += 1
        rate = num if db else den
        ends = [T + -(-hl // rate)]
        if kb:
            ends.append(T + kl)
        if db:
            ends.append(T + -(-dl // rate))
        nxt = min(ends)
        dt, T = nxt - T, nxt
        hl -= rate * dt
        if hl <= 0:
            hb, ih = False, ih + 1
        if kb:
            kl -= dt
            if kl <= 0:
                kb, ik = False, ik + 1
        if db:
            dl -= rate * dt
            if dl <= 0:
                db, idd = False, idd + 1
    # the tail: every HtD has ended by T, nothing overlaps any more
    kfree = T + kl if kb else T
    kp = ik + 1 if kb else ik
    dfree = T + -(-dl // den) if db else T
    tail = 0
    for p in range(idd + 1 if db else idd, n):
        ke = T
        if p == ik and kb:
            ke = kfree
        elif p >= ik:
            while kp <= p:
                kfree += int(t[order[kp]][1])
                kp += 1
            ke = kfree
        dfree = max(dfree, ke) + int(t[order[p]][2])
        tail += 1
    return events, at, tail, max(dfree, kfree)


def overlap_ops_per_order(b, num, den, runs_per_group=16):
    """Average integer operations the enumeration kernel executes per order:
    each thread simulates the first order of its run of OVERLAP_RUN ranks in
    full and resumes every later one at the first position where it differs
    from the one before; events cost OVERLAP_OPS_PER_EVENT, each DtH of the
    closed-form tail OVERLAP_OPS_PER_TAIL.  Measured on runs spread over each
    group's rank space.  Returns (ops, events, tail steps) per order."""
    ev_total = tail_total = orders = 0
    for g in range(b.G):
        t = b.group(g)
        n = t.shape[0]
        nf = math.factorial(n)
        for r in range(runs_per_group):
            start = (nf // runs_per_group * r) // OVERLAP_RUN * OVERLAP_RUN
            rest, rank, order = list(range(n)), start, []
            for i in range(n):
                f = math.factorial(n - 1 - i)
                order.append(rest.pop(rank // f))
                rank %= f
            prev = None
            for _ in range(OVERLAP_RUN):
                ev, at, tail, _ = overlap_loop_events(t, order, num, den)
                q = 0 if prev is None else next(i for i in range(n) if order[i] != prev[i])
                ev_total += ev - at[q]
                tail_total += tail
                orders += 1
                prev = list(order)
                # lexicographic successor
                i = n - 2
                while i >= 0 and order[i] > order[i + 1]:
                    i -= 1
                if i < 0:
                    break
                j = n - 1
                while order[j] < order[i]:
                    j -= 1
                order[i], order[j] = order[j], order[i]
                order[i + 1:] = reversed(order[i + 1:])
    ev, tail = ev_total / orders, tail_total / orders
    return OVERLAP_OPS_PER_EVENT * ev + OVERLAP_OPS_PER_TAIL * tail, ev, tail


def run_overlap(args):
    import torch
    from paper_1806_10113_gb300 import tm
    torch.cuda.set_device(0)
    import oracle
    num, den = 2, 3
    b = inputs.dk_dt_groups(16, 10, seed=1, models=(2,))
    G = b.G
    n_orders = G * math.factorial(10)
    dev = torch.device("cuda", 0)
    d_tasks = torch.from_numpy(b.tasks).to(dev)
    d_off = torch.from_numpy(b.offsets).to(dev)
    d_dma = torch.from_numpy(b.dma).to(dev)
    d_stats = torch.zeros(G * 72, dtype=torch.uint8, device=dev)
    d_status = torch.zeros(G, dtype=torch.int32, device=dev)
    step = lambda: tm.tm_exhaustive_overlap_batch_dev(d_tasks, d_off, b.offsets, d_dma, num, den,
                                                      d_stats, d_status)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if (d_status.cpu().numpy() != 0).any():
        raise RuntimeError("device status errors")
    K = min(args.steps, 20)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(K)]
    sampler = ClockSampler(bus_id_of(0))
    sampler.start()
    time.sleep(0.2)
    for k in range(K):
        ev[k][0].record()
        step()
        ev[k][1].record()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    step_s = statistics.mean(a.elapsed_time(c) for a, c in ev) / 1000.0
    value = n_orders / step_s
    # e2e through the host-pointer call (copies in and out inside the timing)
    t0 = time.perf_counter()
    for _ in range(3):
        st = tm.tm_exhaustive_overlap_batch(b.tasks, b.offsets, b.dma, num, den)
    e2e_s = (time.perf_counter() - t0) / 3
    # the oracle on one host core: random orders of the same groups
    rng = np.random.default_rng(0)
    sample = 20000
    picks = [(int(rng.integers(G)), rng.permutation(10)) for _ in range(sample)]
    t0 = time.perf_counter()
    for g, o in picks:
        oracle.predict_overlap(b.group(g), o, 2, num, den)
    cpu_s = time.perf_counter() - t0
    ops_order, events, tail = overlap_ops_per_order(b, num, den)
    achieved = ops_order * value / 1e12
    out = {
        "metric": "orderings evaluated/s (partial-overlap model, N=10, exhaustive)",
        "value": value, "unit": "orders/s", "n_gpus": 1, "steps": K, "warmup": args.warmup,
        "ms_per_step": 1000 * step_s, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": WORKLOADS["overlap10"], "groups": G, "orders_per_step": n_orders,
                   "rate": f"{num}/{den}", "l2": "inputs < L2 (compute-bound; no flush)"},
        "e2e": {"value": n_orders / e2e_s, "unit": "orders/s",
                "h2d_bytes_per_step": int(b.tasks.nbytes + b.offsets.nbytes + b.dma.nbytes),
                "d2h_bytes_per_step": int(st.nbytes + 4 * G)},
        "gpu_launches": 3 * K,
        "roofline": {"bound": "alu", "kernel": "ovl_enum_kernel (event loop per order)",
                     "achieved": achieved, "peak": INT32_PEAK_TOPS, "unit": "Tops/s (int32)",
                     "frac": achieved / INT32_PEAK_TOPS, "traffic": None,
                     "ops_per_order": round(ops_order, 1),
                     "events_per_order": round(events, 2),
                     "tail_steps_per_order": round(tail, 2),
                     "ops_basis": "what the kernel executes per order (runs of 64 ranks, each "
                                  "order resumed at its first changed position, closed-form tail "
                                  "after the last HtD; counted on 16 runs per group): events x "
                                  "ops per event of the loop body + tail DtH x ops per tail step",
                     "peak_basis": "152 SMs x 128 int32 lanes/clk x 2070 MHz (derived)"},
        "cpu_baseline": {"value": sample / cpu_s, "unit": "orders/s", "cores": 1,
                         "kind": "oracle",
                         "sample": f"{sample} random orders of the same groups, one "
                                   f"oracle.predict_overlap call each ({cpu_s:.2f} s)"},
        "clocks": clocks,
    }
    print(json.dumps(out))
    return 0


def run_heuristic(args):
    import torch
    from paper_1806_10113_gb300 import tm
    import oracle
    torch.cuda.set_device(0)
    b = inputs.training_groups(1 << 20, 4, 16, seed=6)
    G, T = b.G, int(b.tasks.shape[0])
    dev = torch.device("cuda", 0)
    d_tasks = torch.from_numpy(b.tasks).to(dev)
    d_off = torch.from_numpy(b.offsets).to(dev)
    d_dma = torch.from_numpy(b.dma).to(dev)
    d_orders = torch.zeros(T, dtype=torch.int32, device=dev)
    d_ms = torch.zeros(G, dtype=torch.int32, device=dev)
    d_status = torch.zeros(G, dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    step = lambda: tm.tm_heuristic_batch_dev(d_tasks, d_off, G, d_dma, d_orders, d_ms, d_status)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if (d_status.cpu().numpy() != 0).any():
        raise RuntimeError("device status errors")
    K = min(args.steps, 200)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(K)]
    sampler = ClockSampler(bus_id_of(0))
    sampler.start()
    time.sleep(0.2)
    for k in range(K):
        flush.zero_()
        ev[k][0].record()
        step()
        ev[k][1].record()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    step_s = statistics.mean(a.elapsed_time(c) for a, c in ev) / 1000.0
    # parity on a sample against the oracle
    idx = np.random.default_rng(0).integers(0, G, 2000)
    orders = d_orders.cpu().numpy()
    ms = d_ms.cpu().numpy()
    for g in idx:
        o, m = oracle.heuristic(b.group(int(g)), int(b.dma[g]))
        if list(orders[b.offsets[g]:b.offsets[g + 1]]) != o or int(ms[g]) != m:
            raise RuntimeError(f"heuristic mismatch on group {g}")
    t0 = time.perf_counter()
    for _ in range(3):
        tm.tm_heuristic_batch(b.tasks, b.offsets, b.dma)
    e2e_s = (time.perf_counter() - t0) / 3
    sample = 1 << 17
    cores = oracle.hardware_threads()
    t0 = time.perf_counter()
    oracle.heuristic_batch(b.tasks[:b.offsets[sample]], b.offsets[:sample + 1], b.dma[:sample])
    cpu_s = time.perf_counter() - t0
    out = {
        "metric": "task groups scheduled/s (reordering heuristic, Algorithm 1)",
        "value": G / step_s, "unit": "groups/s", "n_gpus": 1, "steps": K, "warmup": args.warmup,
        "ms_per_step": 1000 * step_s, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": WORKLOADS["heuristic1m"], "groups": G,
                   "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MiB write)"},
        "e2e": {"value": G / e2e_s, "unit": "groups/s",
                "h2d_bytes_per_step": int(b.tasks.nbytes + b.offsets.nbytes + b.dma.nbytes),
                "d2h_bytes_per_step": int(4 * T + 4 * G)},
        "gpu_launches": K,
        "roofline": {"bound": "hbm", "kernel": "heuristic_kernel (one warp per group)",
                     "achieved": (b.tasks.nbytes + b.offsets.nbytes + b.dma.nbytes + 4 * T + 4 * G)
                     / step_s / 1e9,
                     "peak": measured_peak("hbm_gbs") or 6800.0, "unit": "GB/s",
                     "frac": (b.tasks.nbytes + b.offsets.nbytes + b.dma.nbytes + 4 * T + 4 * G)
                     / step_s / 1e9 / (measured_peak("hbm_gbs") or 6800.0),
                     "traffic": None,
                     "note": "bytes = tasks, offsets, models in; orders, makespans out; the "
                             "kernel is latency-bound (n dependent warp reductions per group)"},
        "parity_sample": "2000 groups equal to the oracle's orders and makespans",
        "cpu_baseline": {"value": sample / cpu_s, "unit": "groups/s", "cores": cores,
                         "kind": "oracle",
                         "sample": f"the first {sample} groups, oracle heuristic on {cores} "
                                   f"threads ({cpu_s:.2f} s)"},
        "clocks": clocks,
    }
    print(json.dumps(out))
    return 0


def run_single(args):
    """Latency of one small group through the host-pointer calls (the
    paper's own use: one group, scheduled when it is submitted)."""
    import torch
    from paper_1806_10113_gb300 import tm
    import oracle
    torch.cuda.set_device(0)
    b = inputs.single_group_uniform(n=6, seed=0)
    # both searches in one call (the host-pointer tm_schedule_batch)
    for _ in range(max(args.warmup, 10)):
        tm.tm_schedule_batch(b.tasks, b.offsets, b.dma)
    K = min(args.steps, 2000)
    lat = []
    for _ in range(K):
        t0 = time.perf_counter()
        st, order, ms = tm.tm_schedule_batch(b.tasks, b.offsets, b.dma)
        lat.append(time.perf_counter() - t0)
    ref = oracle.exhaustive(b.tasks, 2)
    if int(st[0]["best"]) != ref["best"] or ([int(x) for x in order], int(ms[0])) != \
            oracle.heuristic(b.tasks, 2):
        raise RuntimeError("mismatch with the oracle")
    t0 = time.perf_counter()
    for _ in range(200):
        oracle.exhaustive(b.tasks, 2)
        oracle.heuristic(b.tasks, 2)
    cpu_s = (time.perf_counter() - t0) / 200
    lat_us = np.asarray(lat) * 1e6
    out = {
        "metric": "schedule latency of one 6-task group (exhaustive 720 orders + heuristic)",
        "value": float(np.median(lat_us)), "unit": "us", "n_gpus": 1, "steps": K,
        "warmup": args.warmup, "ms_per_step": float(np.median(lat_us)) / 1000,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic", "config": {"workload": WORKLOADS["single6"]},
        "p99_us": float(np.quantile(lat_us, 0.99)),
        "e2e": {"value": float(np.median(lat_us)), "unit": "us",
                "h2d_bytes_per_step": int(2 * b.tasks.nbytes + 8),
                "d2h_bytes_per_step": int(72 + 4 * 6 + 8)},
        "gpu_launches": 3,
        "cpu_baseline": {"value": cpu_s * 1e6, "unit": "us", "cores": 1, "kind": "oracle",
                         "sample": "the same group, oracle exhaustive + heuristic, 200 calls"},
    }
    print(json.dumps(out))
    return 0


def measured_peak(key: str):
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            v = json.load(f).get(key)
        return float(v) if v else None
    except (OSError, ValueError, TypeError):
        return None


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["tm", "reference"], default="tm")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true",
                    help="default workload: skip the 12-task, learned-path and chained legs")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="dkdt64x10")
    ap.add_argument("--graph", action="store_true", help="replay each step as one CUDA graph")
    ap.add_argument("--tuning", default="",
                    help="pdmax,fuse_finalize,blocks_per_sm[,item_cost[,chunks_per_thread[,unroll]]] "
                         "(skips the autotuner)")
    ap.add_argument("--groups", type=int, default=0, help="beam12: test groups (default 2048)")
    ap.add_argument("--train-groups", type=int, default=2_000_000)
    ap.add_argument("--ranker", default="", help="load ranker parameters (.npy) instead of training")
    ap.add_argument("--ranker-out", default="", help="save the trained ranker parameters (.npy)")
    ap.add_argument("--serve-seconds", type=float, default=5.0)
    ap.add_argument("--exact-max-n", type=int, default=12)
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "beam12":
        return run_beam12(args)
    if args.workload == "serve20k":
        return run_serve(args)
    if args.workload == "overlap10":
        return run_overlap(args)
    if args.workload == "heuristic1m":
        return run_heuristic(args)
    if args.workload == "single6":
        return run_single(args)
    if args.workload == "chain4x4":
        return run_chain(args)
    return run_tm(args)


if __name__ == "__main__":
    sys.exit(main())

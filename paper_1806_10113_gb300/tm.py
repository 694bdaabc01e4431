"""ctypes binding of libtm.so (declared in include/tm.h), same names as the C ABI.

Argument marshalling only: every step of the model runs in the library's CUDA
kernels.  There is no fallback; if libtm.so is missing or a call fails, the
call raises.

Host-pointer calls take array-likes (tasks as int32 [T, 3]: HtD, K, DtH in
ns) and return numpy arrays.  ``*_dev`` calls take CUDA tensors (anything
with ``data_ptr()``; PyTorch is the intended provider) and an optional
stream (a ``torch.cuda.Stream``, a raw handle, or None for the current
PyTorch stream if torch is loaded, else the legacy default stream).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libtm.so")

TM_MAX_TASKS = 16
TM_MAX_EXHAUSTIVE = 12
TM_NOALLOC_MAX_GROUPS = 64
TM_NOALLOC_MAX_TASKS = 768
TM_NOALLOC_MAX_SUBSETS = 4800
TM_RANKER_FEATURES = 32
TM_RANKER_PARAMS = 37377
TM_BEAM_MAX_WIDTH = 64
TM_BEAM_MAX_REFINE_STARTS = 8
TM_CHAIN_MAX_WORKERS = 8

STATS_DTYPE = np.dtype([
    ("best", "<i4"), ("worst", "<i4"), ("sum", "<i8"), ("mean", "<f8"),
    ("best_rank", "<u8"), ("worst_rank", "<u8"),
    ("best_order", "u1", (16,)), ("worst_order", "u1", (16,)),
], align=True)
assert STATS_DTYPE.itemsize == 72

_lock = threading.Lock()
_lib = None


class TMError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} ({code})")


class _Task(ctypes.Structure):
    _fields_ = [("htd", ctypes.c_int32), ("k", ctypes.c_int32), ("dth", ctypes.c_int32)]


class _Device(ctypes.Structure):
    _fields_ = [("dma_engines", ctypes.c_int32)]


_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_SIGS = {
    "tm_predict": [_vp, ctypes.c_int, _vp, _vp, _vp],
    "tm_exhaustive": [_vp, ctypes.c_int, _vp, _vp, _vp],
    "tm_heuristic": [_vp, ctypes.c_int, _vp, _vp, _vp],
    "tm_predict_batch": [_vp, _vp, ctypes.c_int, _vp, _vp, _vp],
    "tm_exhaustive_batch": [_vp, _vp, ctypes.c_int, _vp, _vp],
    "tm_heuristic_batch": [_vp, _vp, ctypes.c_int, _vp, _vp, _vp],
    "tm_predict_batch_dev": [_vp, _vp, ctypes.c_int, _vp, _vp, _vp, _vp, _vp],
    "tm_heuristic_batch_dev": [_vp, _vp, ctypes.c_int, _vp, _vp, _vp, _vp, _vp],
    "tm_plan_create": [_vp, ctypes.c_int, ctypes.POINTER(_vp)],
    "tm_plan_create_tuned": [_vp, ctypes.c_int, _vp, ctypes.POINTER(_vp)],
    "tm_set_default_tuning": [_vp],
    "tm_plan_destroy": [_vp],
    "tm_plan_launches": [_vp],
    "tm_plan_set_timing": [_vp, _vp, _vp],
    "tm_plan_walk_counts": [_vp, ctypes.POINTER(ctypes.c_ulonglong),
                            ctypes.POINTER(ctypes.c_ulonglong)],
    "tm_plan_capture": [_vp, _vp, _vp, _vp, _vp, _vp, _vp],
    "tm_plan_graph_launch": [_vp, _vp],
    "tm_plan_graph_set_timing": [_vp, _vp, _vp],
    "tm_exhaustive_batch_dev": [_vp, _vp, _vp, _vp, _vp, _vp],
    "tm_exhaustive_batch_noalloc": [_vp, _vp, ctypes.c_int, _vp, _vp, _vp, _vp],
    "tm_schedule_batch_dev": [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp],
    "tm_schedule_batch": [_vp, _vp, ctypes.c_int, _vp, _vp, _vp, _vp],
    "tm_ranker_create": [ctypes.c_uint64, ctypes.POINTER(_vp)],
    "tm_ranker_destroy": [_vp],
    "tm_ranker_get_params": [_vp, _vp],
    "tm_ranker_set_params": [_vp, _vp],
    "tm_ranker_errors": [_vp, ctypes.POINTER(ctypes.c_int32)],
    "tm_ranker_rows_count": [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                             ctypes.POINTER(ctypes.c_int32)],
    "tm_ranker_rows_dev": [_vp, _vp, _vp, ctypes.c_int, _vp, _vp, _vp, ctypes.c_int64,
                           ctypes.c_int32, _vp, _vp, _vp, _vp, _vp],
    "tm_ranker_forward_dev": [_vp, _vp, ctypes.c_int64, _vp, _vp],
    "tm_ranker_forward_keep_dev": [_vp, _vp, ctypes.c_int64, _vp, _vp, ctypes.c_int, _vp],
    "tm_ranker_grad_dev": [_vp, _vp, ctypes.c_int64, _vp, _vp, ctypes.c_int32, _vp, _vp, _vp],
    "tm_ranker_adam_dev": [_vp, ctypes.c_float, _vp],
    "tm_beam_batch_dev": [_vp, _vp, _vp, _vp, ctypes.c_int, _vp, ctypes.c_int, ctypes.c_int, _vp,
                          _vp, _vp, _vp, _vp],
    "tm_refine_batch_dev": [_vp, _vp, ctypes.c_int, _vp, _vp, _vp, _vp, _vp],
    "tm_predict_chain": [_vp, ctypes.c_int, ctypes.c_int, _vp, _vp, ctypes.POINTER(ctypes.c_int32)],
    "tm_exhaustive_chain": [_vp, ctypes.c_int, ctypes.c_int, _vp, _vp],
    "tm_exhaustive_chain_batch": [_vp, _vp, _vp, ctypes.c_int, _vp, _vp],
    "tm_exhaustive_chain_batch_dev": [_vp, _vp, _vp, _vp, _vp, ctypes.c_int, _vp, _vp, _vp, _vp],
    "tm_chain_tail_counts": [ctypes.POINTER(ctypes.c_ulonglong), ctypes.POINTER(ctypes.c_ulonglong)],
    "tm_predict_chain_batch_dev": [_vp, _vp, _vp, ctypes.c_int, _vp, _vp, _vp, _vp, _vp],
    "tm_server_create": [_vp, _vp, ctypes.POINTER(_vp)],
    "tm_server_submit": [_vp, _vp, ctypes.c_int, _vp, ctypes.POINTER(ctypes.c_uint64)],
    "tm_server_poll": [_vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int)],
    "tm_server_replay": [_vp, _vp, _vp, ctypes.c_int, _vp, _vp, _vp],
    "tm_server_counters": [_vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                           ctypes.POINTER(ctypes.c_int64)],
    "tm_server_destroy": [_vp],
    "tm_predict_overlap": [_vp, ctypes.c_int, _vp, _vp, _i32, _i32, _vp],
    "tm_predict_overlap_batch": [_vp, _vp, ctypes.c_int, _vp, _vp, _i32, _i32, _vp],
    "tm_predict_overlap_batch_dev": [_vp, _vp, ctypes.c_int, _vp, _vp, _i32, _i32, _vp, _vp, _vp],
    "tm_exhaustive_overlap_batch": [_vp, _vp, ctypes.c_int, _vp, _i32, _i32, _vp],
    "tm_exhaustive_overlap_batch_dev": [_vp, _vp, _vp, ctypes.c_int, _vp, _i32, _i32, _vp, _vp,
                                        _vp],
    "tm_measure_int32_rates": [_vp, _vp, _vp],
    "tm_strerror": [ctypes.c_int],
    "tm_version": [],
}
_RESTYPE = {"tm_plan_destroy": None, "tm_ranker_destroy": None, "tm_server_destroy": None, "tm_strerror": ctypes.c_char_p,
            "tm_version": ctypes.c_char_p}


def lib():
    """Loads libtm.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                                   "`python -m paper_1806_10113_gb300.build`")
            h = ctypes.CDLL(LIB_PATH)
            for name, args in _SIGS.items():
                f = getattr(h, name)
                f.argtypes = args
                f.restype = _RESTYPE.get(name, ctypes.c_int)
            _lib = h
    return _lib


def strerror(code: int) -> str:
    return lib().tm_strerror(int(code)).decode()


def version() -> str:
    return lib().tm_version().decode()


def tm_measure_int32_rates() -> dict:
    """Measured int32 max, add and max-then-add issue rates (operations/s)."""
    v = [ctypes.c_double() for _ in range(3)]
    _check(lib().tm_measure_int32_rates(*[ctypes.byref(x) for x in v]), "tm_measure_int32_rates")
    return {"max": v[0].value, "add": v[1].value, "max_add": v[2].value}


def _check(rc: int, where: str):
    if rc != 0:
        raise TMError(rc, where)


# ---- marshalling helpers ------------------------------------------------------

def _tasks(tasks) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(tasks, dtype=np.int32).reshape(-1, 3))
    return a


def _devs(dma, G: int) -> np.ndarray:
    return np.ascontiguousarray(np.broadcast_to(np.asarray(dma, dtype=np.int32), (G,)))


def _p(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _dptr(t):
    return None if t is None else ctypes.c_void_p(int(t.data_ptr()))


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available() and torch.cuda.is_initialized():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def stats_to_dicts(stats: np.ndarray, sizes) -> list:
    out = []
    for s, n in zip(stats, sizes):
        n = int(n)
        out.append({
            "best": int(s["best"]), "worst": int(s["worst"]), "sum": int(s["sum"]),
            "mean": float(s["mean"]), "best_rank": int(s["best_rank"]),
            "worst_rank": int(s["worst_rank"]),
            "best_order": [int(x) for x in s["best_order"][:n]],
            "worst_order": [int(x) for x in s["worst_order"][:n]],
        })
    return out


# ---- single group, host pointers ---------------------------------------------

def tm_predict(tasks, order, dma_engines: int) -> int:
    t = _tasks(tasks)
    o = np.ascontiguousarray(np.asarray(order, dtype=np.int32))
    dev = np.asarray([dma_engines], dtype=np.int32)
    out = np.zeros(1, dtype=np.int32)
    _check(lib().tm_predict(_p(t), t.shape[0], _p(o), _p(dev), _p(out)), "tm_predict")
    return int(out[0])


def tm_exhaustive(tasks, dma_engines: int) -> dict:
    t = _tasks(tasks)
    dev = np.asarray([dma_engines], dtype=np.int32)
    st = np.zeros(1, dtype=STATS_DTYPE)
    mean = ctypes.c_double(0.0)
    _check(lib().tm_exhaustive(_p(t), t.shape[0], _p(dev), _p(st), ctypes.byref(mean)),
           "tm_exhaustive")
    d = stats_to_dicts(st, [t.shape[0]])[0]
    assert d["mean"] == mean.value
    return d


def tm_heuristic(tasks, dma_engines: int):
    t = _tasks(tasks)
    dev = np.asarray([dma_engines], dtype=np.int32)
    order = np.zeros(max(t.shape[0], 1), dtype=np.int32)
    ms = np.zeros(1, dtype=np.int32)
    _check(lib().tm_heuristic(_p(t), t.shape[0], _p(dev), _p(order), _p(ms)), "tm_heuristic")
    return [int(x) for x in order[:t.shape[0]]], int(ms[0])


# ---- ragged batches, host pointers --------------------------------------------

def tm_predict_batch(tasks, offsets, orders, dma) -> np.ndarray:
    t = _tasks(tasks)
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32))
    G = off.shape[0] - 1
    o = np.ascontiguousarray(np.asarray(orders, dtype=np.int32).reshape(-1))
    dev = _devs(dma, G)
    out = np.zeros(max(G, 1), dtype=np.int32)
    _check(lib().tm_predict_batch(_p(t), _p(off), G, _p(o), _p(dev), _p(out)),
           "tm_predict_batch")
    return out[:G]


def tm_exhaustive_batch(tasks, offsets, dma) -> np.ndarray:
    """Returns a structured array of STATS_DTYPE, one row per group."""
    t = _tasks(tasks)
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32))
    G = off.shape[0] - 1
    dev = _devs(dma, G)
    st = np.zeros(max(G, 1), dtype=STATS_DTYPE)
    _check(lib().tm_exhaustive_batch(_p(t), _p(off), G, _p(dev), _p(st)),
           "tm_exhaustive_batch")
    return st[:G]


def tm_heuristic_batch(tasks, offsets, dma):
    t = _tasks(tasks)
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32))
    G = off.shape[0] - 1
    dev = _devs(dma, G)
    orders = np.zeros(max(t.shape[0], 1), dtype=np.int32)
    ms = np.zeros(max(G, 1), dtype=np.int32)
    _check(lib().tm_heuristic_batch(_p(t), _p(off), G, _p(dev), _p(orders), _p(ms)),
           "tm_heuristic_batch")
    return orders[:t.shape[0]], ms[:G]


def tm_schedule_batch(tasks, offsets, dma):
    """Exhaustive search and heuristic of every group in one call.

    Returns (stats structured array, heuristic orders, heuristic makespans)."""
    t = _tasks(tasks)
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32))
    G = off.shape[0] - 1
    dev = _devs(dma, G)
    st = np.zeros(max(G, 1), dtype=STATS_DTYPE)
    orders = np.zeros(max(t.shape[0], 1), dtype=np.int32)
    ms = np.zeros(max(G, 1), dtype=np.int32)
    _check(lib().tm_schedule_batch(_p(t), _p(off), G, _p(dev), _p(st), _p(orders), _p(ms)),
           "tm_schedule_batch")
    return st[:G], orders[:t.shape[0]], ms[:G]


# ---- ragged batches, device pointers, stream-ordered ---------------------------

def tm_predict_batch_dev(d_tasks, d_offsets, G: int, d_orders, d_devs, d_makespans,
                         d_status=None, stream=None):
    _check(lib().tm_predict_batch_dev(_dptr(d_tasks), _dptr(d_offsets), int(G), _dptr(d_orders),
                                      _dptr(d_devs), _dptr(d_makespans), _dptr(d_status),
                                      _stream(stream)), "tm_predict_batch_dev")


def tm_heuristic_batch_dev(d_tasks, d_offsets, G: int, d_devs, d_orders_out,
                           d_makespans_out=None, d_status=None, stream=None):
    _check(lib().tm_heuristic_batch_dev(_dptr(d_tasks), _dptr(d_offsets), int(G), _dptr(d_devs),
                                        _dptr(d_orders_out), _dptr(d_makespans_out),
                                        _dptr(d_status), _stream(stream)),
           "tm_heuristic_batch_dev")


class Tuning(ctypes.Structure):
    """tm_tuning: pdmax (3..5), fuse_finalize (1 fused, 2 separate), blocks_per_sm,
    item_cost, chunks_per_thread (1 static split, 2..64 dynamic), unroll (1
    straight-line walk level, 2 loop, 3 straight-line with the per-order
    additions on the FMA pipe, 4 as 3 at four blocks per SM, 5 as 3 with the closed
    form for prefixes whose completions one engine's path ends, 6 as 5 with the
    suffix constants in shared memory at four blocks per SM, 7 as 6 with the vote and
    the closed forms in one pass and a rolled quad loop, 8 as 6 with that loop);
    0 = default."""
    _fields_ = [("pdmax", ctypes.c_int32), ("fuse_finalize", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("item_cost", ctypes.c_int32),
                ("chunks_per_thread", ctypes.c_int32), ("unroll", ctypes.c_int32)]


def tm_set_default_tuning(pdmax: int = 0, fuse_finalize: int = 0, blocks_per_sm: int = 0,
                          item_cost: int = 0, chunks_per_thread: int = 0, unroll: int = 0):
    """Tuning for plans made by tm_plan_create and the host-pointer calls."""
    t = Tuning(pdmax, fuse_finalize, blocks_per_sm, item_cost, chunks_per_thread, unroll)
    _check(lib().tm_set_default_tuning(ctypes.byref(t)), "tm_set_default_tuning")


class Plan:
    """Owns a tm_plan (exhaustive search over a fixed set of group sizes)."""

    def __init__(self, offsets, pdmax: int = 0, fuse_finalize: int = 0, blocks_per_sm: int = 0,
                 item_cost: int = 0, chunks_per_thread: int = 0, unroll: int = 0):
        off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32))
        self.G = off.shape[0] - 1
        self.offsets = off
        self.tuning = Tuning(pdmax, fuse_finalize, blocks_per_sm, item_cost, chunks_per_thread,
                             unroll)
        h = ctypes.c_void_p()
        _check(lib().tm_plan_create_tuned(_p(off), self.G, ctypes.byref(self.tuning),
                                          ctypes.byref(h)), "tm_plan_create_tuned")
        self._h = h

    @property
    def handle(self):
        return self._h

    def launches(self) -> int:
        return int(lib().tm_plan_launches(self._h))

    def walk_counts(self):
        """(prefixes walked per run, prefixes of the last run whose 24
        completions were evaluated one by one): tm_plan_walk_counts; call it
        after the run has finished."""
        pre, full = ctypes.c_ulonglong(0), ctypes.c_ulonglong(0)
        _check(lib().tm_plan_walk_counts(self._h, ctypes.byref(pre), ctypes.byref(full)),
               "tm_plan_walk_counts")
        return int(pre.value), int(full.value)

    def set_timing(self, event_before=None, event_after=None):
        """Records two CUDA events (e.g. torch.cuda.Event(enable_timing=True))
        around the enumeration kernel of every later launch; None turns it off."""
        h = lambda e: None if e is None else ctypes.c_void_p(int(getattr(e, "cuda_event", e)))
        _check(lib().tm_plan_set_timing(self._h, h(event_before), h(event_after)),
               "tm_plan_set_timing")

    def capture(self, d_tasks, d_devs, d_stats, d_orders_out, d_makespans_out=None,
                d_status=None):
        """Records one tm_schedule_batch_dev pass over these buffers as a CUDA graph."""
        _check(lib().tm_plan_capture(self._h, _dptr(d_tasks), _dptr(d_devs), _dptr(d_stats),
                                     _dptr(d_orders_out), _dptr(d_makespans_out),
                                     _dptr(d_status)), "tm_plan_capture")

    def graph_launch(self, stream=None):
        """Replays the captured pass on a stream."""
        _check(lib().tm_plan_graph_launch(self._h, _stream(stream)), "tm_plan_graph_launch")

    def graph_set_timing(self, event_before, event_after):
        """Swaps the timing events recorded by the captured graph."""
        h = lambda e: ctypes.c_void_p(int(getattr(e, "cuda_event", e)))
        _check(lib().tm_plan_graph_set_timing(self._h, h(event_before), h(event_after)),
               "tm_plan_graph_set_timing")

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().tm_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tm_schedule_batch_dev(plan: Plan, d_tasks, d_devs, d_stats, d_orders_out,
                          d_makespans_out=None, d_status=None, stream=None):
    """Exhaustive search and heuristic of every group of the plan, two launches."""
    _check(lib().tm_schedule_batch_dev(plan.handle, _dptr(d_tasks), _dptr(d_devs), _dptr(d_stats),
                                       _dptr(d_orders_out), _dptr(d_makespans_out),
                                       _dptr(d_status), _stream(stream)),
           "tm_schedule_batch_dev")


def tm_exhaustive_batch_dev(plan: Plan, d_tasks, d_devs, d_stats, d_status=None, stream=None):
    """d_stats: a device buffer of plan.G * 72 bytes (STATS_DTYPE rows)."""
    _check(lib().tm_exhaustive_batch_dev(plan.handle, _dptr(d_tasks), _dptr(d_devs),
                                         _dptr(d_stats), _dptr(d_status), _stream(stream)),
           "tm_exhaustive_batch_dev")


def tm_exhaustive_batch_noalloc(d_tasks, offsets, d_devs, d_stats, d_status=None, stream=None):
    """Exhaustive search with no allocation, for callers that cannot allocate
    device memory (their GPU memory is owned by another allocator, or they
    cannot pay for cudaMalloc / cudaFree where they run).

    Same results as tm_exhaustive_batch_dev.  ``offsets`` is a HOST array;
    the other buffers are device tensors.  The library's fixed 1 MiB working
    array caps a batch at TM_NOALLOC_MAX_GROUPS groups, TM_NOALLOC_MAX_TASKS
    tasks and TM_NOALLOC_MAX_SUBSETS 4-task subsets (TMError code -8 beyond).  All calls share that array, so
    calls that could overlap on the GPU must be serialised."""
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32))
    G = off.shape[0] - 1
    _check(lib().tm_exhaustive_batch_noalloc(_dptr(d_tasks), _p(off), G, _dptr(d_devs),
                                             _dptr(d_stats), _dptr(d_status), _stream(stream)),
           "tm_exhaustive_batch_noalloc")


# ---- learned order ranker and beam search --------------------------------------

def tm_ranker_rows_count(offsets):
    """(rows, states) of the training rows of a batch with these host offsets."""
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32))
    rows, states = ctypes.c_int64(0), ctypes.c_int32(0)
    _check(lib().tm_ranker_rows_count(_p(off), off.shape[0] - 1, ctypes.byref(rows),
                                      ctypes.byref(states)), "tm_ranker_rows_count")
    return int(rows.value), int(states.value)


class Ranker:
    """Owns a tm_ranker: the learned order ranker (4-layer bfloat16 MLP) whose
    proposals feed tm_beam_batch_dev.  Lives on the CUDA device current at
    creation."""

    def __init__(self, seed: int = 0):
        h = ctypes.c_void_p()
        _check(lib().tm_ranker_create(ctypes.c_uint64(seed & ((1 << 64) - 1)), ctypes.byref(h)),
               "tm_ranker_create")
        self._h = h

    @property
    def handle(self):
        return self._h

    def get_params(self) -> np.ndarray:
        out = np.zeros(TM_RANKER_PARAMS, dtype=np.float32)
        _check(lib().tm_ranker_get_params(self._h, _p(out)), "tm_ranker_get_params")
        return out

    def set_params(self, params):
        a = np.ascontiguousarray(np.asarray(params, dtype=np.float32).reshape(-1))
        if a.shape[0] != TM_RANKER_PARAMS:
            raise ValueError(f"expected {TM_RANKER_PARAMS} parameters, got {a.shape[0]}")
        _check(lib().tm_ranker_set_params(self._h, _p(a)), "tm_ranker_set_params")

    def errors(self) -> int:
        """1 if a bounded wait of the tensor-core scoring kernel ever expired."""
        c = ctypes.c_int32(0)
        _check(lib().tm_ranker_errors(self._h, ctypes.byref(c)), "tm_ranker_errors")
        return int(c.value)

    def rows_dev(self, d_tasks, d_offsets, G: int, d_devs, rows: int, states: int, d_X,
                 d_state_off, d_target, d_orders=None, d_stats=None, d_status=None,
                 stream=None):
        """Training rows along d_orders (or d_stats' best orders)."""
        _check(lib().tm_ranker_rows_dev(self._h, _dptr(d_tasks), _dptr(d_offsets), int(G),
                                        _dptr(d_devs), _dptr(d_orders), _dptr(d_stats),
                                        int(rows), int(states), _dptr(d_X), _dptr(d_state_off),
                                        _dptr(d_target), _dptr(d_status), _stream(stream)),
               "tm_ranker_rows_dev")

    def forward_dev(self, d_X, rows: int, d_logits, stream=None):
        _check(lib().tm_ranker_forward_dev(self._h, _dptr(d_X), int(rows), _dptr(d_logits),
                                           _stream(stream)), "tm_ranker_forward_dev")

    def forward_keep_dev(self, d_X, rows: int, d_logits, d_acts, path: int = 0, stream=None):
        """Logits and the hidden layers' bfloat16 activations [3 x rows x 128];
        path 0 the tensor-core scoring kernel, 1 the training forward."""
        _check(lib().tm_ranker_forward_keep_dev(self.handle, _dptr(d_X), int(rows),
                                                _dptr(d_logits), _dptr(d_acts), int(path),
                                                _stream(stream)), "tm_ranker_forward_keep_dev")

    def grad_dev(self, d_X, rows: int, d_state_off, d_target, states: int, d_grad=None,
                 d_loss=None, stream=None):
        _check(lib().tm_ranker_grad_dev(self._h, _dptr(d_X), int(rows), _dptr(d_state_off),
                                        _dptr(d_target), int(states), _dptr(d_grad),
                                        _dptr(d_loss), _stream(stream)), "tm_ranker_grad_dev")

    def adam_dev(self, lr: float, stream=None):
        _check(lib().tm_ranker_adam_dev(self._h, ctypes.c_float(lr), _stream(stream)),
               "tm_ranker_adam_dev")

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().tm_ranker_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tm_beam_batch_dev(ranker: Ranker, d_tasks, d_offsets, offsets, d_devs, beam_width: int,
                      d_orders_out, d_makespans_out=None, d_status=None, d_beam_won=None,
                      stream=None, refine_starts: int = 0):
    """Beam search of every group with the ranker's proposals; never worse than
    the heuristic.  ``offsets`` is the HOST copy of d_offsets.  With
    refine_starts = K > 0 the K best finished beams and the heuristic's order
    each start the exact-model descent (tm_refine_batch_dev)."""
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32))
    _check(lib().tm_beam_batch_dev(ranker.handle, _dptr(d_tasks), _dptr(d_offsets), _p(off),
                                   off.shape[0] - 1, _dptr(d_devs), int(beam_width),
                                   int(refine_starts), _dptr(d_orders_out),
                                   _dptr(d_makespans_out), _dptr(d_status), _dptr(d_beam_won),
                                   _stream(stream)), "tm_beam_batch_dev")


def tm_refine_batch_dev(d_tasks, d_offsets, G: int, d_devs, d_orders, d_makespans=None,
                        d_status=None, stream=None):
    """Exact-model descent (swaps and moves of one task) from the orders in
    d_orders, which receive the results."""
    _check(lib().tm_refine_batch_dev(_dptr(d_tasks), _dptr(d_offsets), int(G), _dptr(d_devs),
                                     _dptr(d_orders), _dptr(d_makespans), _dptr(d_status),
                                     _stream(stream)), "tm_refine_batch_dev")


# ---- serving -------------------------------------------------------------------

TM_METHOD_EXHAUSTIVE, TM_METHOD_BEAM, TM_METHOD_HEURISTIC = 0, 1, 2

RESULT_DTYPE = np.dtype([
    ("ticket", "<u8"), ("status", "<i4"), ("n", "<i4"), ("makespan", "<i4"), ("method", "<i4"),
    ("latency_ns", "<i8"), ("order", "<i4", (16,)),
], align=True)
assert RESULT_DTYPE.itemsize == 96


class ServerConfig(ctypes.Structure):
    """tm_server_config (0 = default for the sizes)."""
    _fields_ = [("lanes", ctypes.c_int32), ("lane_groups", ctypes.c_int32),
                ("lane_tasks", ctypes.c_int32), ("lane_subsets", ctypes.c_int32),
                ("exact_max_n", ctypes.c_int32), ("beam_width", ctypes.c_int32),
                ("tuning", Tuning), ("refine_starts", ctypes.c_int32)]


class Server:
    """Owns a tm_server: continuous batching of task groups that arrive one at
    a time (exhaustive optimum up to exact_max_n tasks, beam search with
    `ranker` or the heuristic above)."""

    def __init__(self, exact_max_n: int = 12, beam_width: int = 0, ranker: Ranker = None,
                 lanes: int = 0, lane_groups: int = 0, lane_tasks: int = 0,
                 lane_subsets: int = 0, tuning: Tuning = None, refine_starts: int = 0):
        self.config = ServerConfig(lanes, lane_groups, lane_tasks, lane_subsets, exact_max_n,
                                   beam_width, tuning if tuning is not None else Tuning(),
                                   refine_starts)
        self._ranker = ranker          # keeps the ranker alive while the server runs
        h = ctypes.c_void_p()
        _check(lib().tm_server_create(ctypes.byref(self.config),
                                      ranker.handle if ranker is not None else None,
                                      ctypes.byref(h)), "tm_server_create")
        self._h = h

    def submit(self, tasks, dma_engines: int) -> int:
        t = _tasks(tasks)
        dev = np.asarray([dma_engines], dtype=np.int32)
        ticket = ctypes.c_uint64(0)
        _check(lib().tm_server_submit(self._h, _p(t), t.shape[0], _p(dev), ctypes.byref(ticket)),
               "tm_server_submit")
        return int(ticket.value)

    def poll(self, max_results: int = 1024, wait_us: int = 0) -> np.ndarray:
        out = np.zeros(max(max_results, 1), dtype=RESULT_DTYPE)
        k = ctypes.c_int(0)
        _check(lib().tm_server_poll(self._h, _p(out), int(max_results), int(wait_us),
                                    ctypes.byref(k)), "tm_server_poll")
        return out[:k.value]

    def replay(self, tasks, offsets, dma, arrival_ns) -> np.ndarray:
        """Open-loop load from the calling thread; results in group order."""
        t = _tasks(tasks)
        off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32))
        G = off.shape[0] - 1
        dev = _devs(dma, G)
        arr = np.ascontiguousarray(np.asarray(arrival_ns, dtype=np.int64))
        out = np.zeros(max(G, 1), dtype=RESULT_DTYPE)
        _check(lib().tm_server_replay(self._h, _p(t), _p(off), G, _p(dev), _p(arr), _p(out)),
               "tm_server_replay")
        return out[:G]

    def counters(self) -> dict:
        b, c, m = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int64(0)
        _check(lib().tm_server_counters(self._h, ctypes.byref(b), ctypes.byref(c),
                                        ctypes.byref(m)), "tm_server_counters")
        return {"batches": b.value, "completed": c.value, "max_batch_groups": m.value}

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().tm_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- partial-overlap variant ------------------------------------------------------

def tm_predict_overlap(tasks, order, dma_engines: int, rate_num: int, rate_den: int) -> int:
    """Makespan of one order when concurrent HtD and DtH transfers each run at
    rate_num / rate_den of full speed (see include/tm.h)."""
    t = _tasks(tasks)
    o = np.ascontiguousarray(np.asarray(order, dtype=np.int32))
    dev = np.asarray([dma_engines], dtype=np.int32)
    out = np.zeros(1, dtype=np.int32)
    _check(lib().tm_predict_overlap(_p(t), t.shape[0], _p(o), _p(dev), int(rate_num),
                                    int(rate_den), _p(out)), "tm_predict_overlap")
    return int(out[0])


def tm_predict_overlap_batch(tasks, offsets, orders, dma, rate_num: int, rate_den: int):
    t = _tasks(tasks)
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32))
    G = off.shape[0] - 1
    o = np.ascontiguousarray(np.asarray(orders, dtype=np.int32).reshape(-1))
    dev = _devs(dma, G)
    out = np.zeros(max(G, 1), dtype=np.int32)
    _check(lib().tm_predict_overlap_batch(_p(t), _p(off), G, _p(o), _p(dev), int(rate_num),
                                          int(rate_den), _p(out)), "tm_predict_overlap_batch")
    return out[:G]


def tm_predict_overlap_batch_dev(d_tasks, d_offsets, G: int, d_orders, d_devs, rate_num: int,
                                 rate_den: int, d_makespans, d_status=None, stream=None):
    _check(lib().tm_predict_overlap_batch_dev(_dptr(d_tasks), _dptr(d_offsets), int(G),
                                              _dptr(d_orders), _dptr(d_devs), int(rate_num),
                                              int(rate_den), _dptr(d_makespans), _dptr(d_status),
                                              _stream(stream)), "tm_predict_overlap_batch_dev")


def tm_exhaustive_overlap_batch(tasks, offsets, dma, rate_num: int, rate_den: int) -> np.ndarray:
    t = _tasks(tasks)
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32))
    G = off.shape[0] - 1
    dev = _devs(dma, G)
    st = np.zeros(max(G, 1), dtype=STATS_DTYPE)
    _check(lib().tm_exhaustive_overlap_batch(_p(t), _p(off), G, _p(dev), int(rate_num),
                                             int(rate_den), _p(st)), "tm_exhaustive_overlap_batch")
    return st[:G]


def tm_exhaustive_overlap_batch_dev(d_tasks, d_offsets, offsets, d_devs, rate_num: int,
                                    rate_den: int, d_stats, d_status=None, stream=None):
    """``offsets`` is the HOST copy of d_offsets."""
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32))
    _check(lib().tm_exhaustive_overlap_batch_dev(_dptr(d_tasks), _dptr(d_offsets), _p(off),
                                                 off.shape[0] - 1, _dptr(d_devs), int(rate_num),
                                                 int(rate_den), _dptr(d_stats), _dptr(d_status),
                                                 _stream(stream)),
           "tm_exhaustive_overlap_batch_dev")


# ---- chained tasks ---------------------------------------------------------------

def _workers(workers, G: int) -> np.ndarray:
    return np.ascontiguousarray(np.broadcast_to(np.asarray(workers, dtype=np.int32), (G,)))


def tm_predict_chain(tasks, workers: int, order, dma_engines: int) -> int:
    """Makespan of one order of a chained group: tasks[r * workers + w] is
    worker w's round-r task; `order` lists task indices round by round."""
    t = _tasks(tasks)
    n = t.shape[0]
    if workers < 1 or n % workers:
        raise TMError(-1, "tm_predict_chain")
    o = np.ascontiguousarray(np.asarray(order, dtype=np.int32))
    dev = np.asarray([dma_engines], dtype=np.int32)
    ms = ctypes.c_int32(0)
    _check(lib().tm_predict_chain(_p(t), int(workers), n // int(workers), _p(o), _p(dev),
                                  ctypes.byref(ms)), "tm_predict_chain")
    return int(ms.value)


def tm_exhaustive_chain(tasks, workers: int, dma_engines: int) -> dict:
    """All (workers!)^rounds orders of one chained group."""
    t = _tasks(tasks)
    n = t.shape[0]
    if workers < 1 or n % workers:
        raise TMError(-1, "tm_exhaustive_chain")
    dev = np.asarray([dma_engines], dtype=np.int32)
    st = np.zeros(1, dtype=STATS_DTYPE)
    _check(lib().tm_exhaustive_chain(_p(t), int(workers), n // int(workers), _p(dev), _p(st)),
           "tm_exhaustive_chain")
    return stats_to_dicts(st, [n])[0]


def tm_exhaustive_chain_batch(tasks, offsets, workers, dma) -> np.ndarray:
    """tm_stats of every chained group of a ragged batch (workers[g] each)."""
    t = _tasks(tasks)
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32))
    G = off.shape[0] - 1
    st = np.zeros(max(G, 1), dtype=STATS_DTYPE)
    _check(lib().tm_exhaustive_chain_batch(_p(t), _p(off), _p(_workers(workers, G)), G,
                                           _p(_devs(dma, G)), _p(st)), "tm_exhaustive_chain_batch")
    return st[:G]


def tm_exhaustive_chain_batch_dev(d_tasks, d_offsets, offsets, d_workers, workers, d_devs,
                                  d_stats, d_status=None, stream=None):
    """Device-pointer form; ``offsets`` and ``workers`` are the HOST copies."""
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32))
    G = off.shape[0] - 1
    w = _workers(workers, G)
    _check(lib().tm_exhaustive_chain_batch_dev(_dptr(d_tasks), _dptr(d_offsets), _p(off),
                                               _dptr(d_workers), _p(w), G, _dptr(d_devs),
                                               _dptr(d_stats), _dptr(d_status), _stream(stream)),
           "tm_exhaustive_chain_batch_dev")


def tm_chain_tail_counts():
    """(tail blocks walked, tail blocks in closed form) of this host thread's
    last exhaustive chained search; call it once the search has finished."""
    tails, closed = ctypes.c_ulonglong(0), ctypes.c_ulonglong(0)
    _check(lib().tm_chain_tail_counts(ctypes.byref(tails), ctypes.byref(closed)),
           "tm_chain_tail_counts")
    return int(tails.value), int(closed.value)


def tm_predict_chain_batch_dev(d_tasks, d_offsets, d_workers, G: int, d_orders, d_devs,
                               d_makespans, d_status=None, stream=None):
    _check(lib().tm_predict_chain_batch_dev(_dptr(d_tasks), _dptr(d_offsets), _dptr(d_workers),
                                            int(G), _dptr(d_orders), _dptr(d_devs),
                                            _dptr(d_makespans), _dptr(d_status), _stream(stream)),
           "tm_predict_chain_batch_dev")

"""CPU oracle for the temporal execution model, its exhaustive search and the
reordering heuristic of Lazaro-Munoz et al. (arXiv 1806.10113).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA library
never calls it and shares no code with it.

The arithmetic lives in ``tm_oracle.cpp`` (plain C++, int64): a literal
event-driven FIFO simulation of Sec. 4.1 (Figs. 4 and 6), a
``std::next_permutation`` enumeration of all n! orders, and Algorithm 1 of
Sec. 5.1.  This module only builds that file with g++ and marshals arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tm_oracle.cpp")
_HDR = os.path.join(_HERE, "tm_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


class OrcTask(ctypes.Structure):
    _fields_ = [("htd", ctypes.c_int32), ("k", ctypes.c_int32), ("dth", ctypes.c_int32)]


class OrcStats(ctypes.Structure):
    _fields_ = [
        ("best", ctypes.c_int64),
        ("worst", ctypes.c_int64),
        ("sum", ctypes.c_int64),
        ("mean", ctypes.c_double),
        ("best_rank", ctypes.c_uint64),
        ("worst_rank", ctypes.c_uint64),
        ("best_order", ctypes.c_int32 * 16),
        ("worst_order", ctypes.c_int32 * 16),
    ]


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` next to its source (plain g++, no -march)."""
    with _lock:
        newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
        if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
            return _LIB
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["g++", "-O3", "-std=c++17", "-shared", "-fPIC", "-pthread",
               "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is None:
        # TM_ORACLE_LIB lets the mutation test load a deliberately broken copy.
        path = os.environ.get("TM_ORACLE_LIB") or build()
        lib = ctypes.CDLL(path)
        P = ctypes.POINTER
        lib.orc_predict.argtypes = [P(OrcTask), ctypes.c_int, P(ctypes.c_int32), ctypes.c_int,
                                    P(ctypes.c_int64), P(ctypes.c_int64)]
        lib.orc_exhaustive.argtypes = [P(OrcTask), ctypes.c_int, ctypes.c_int, P(OrcStats)]
        lib.orc_exhaustive_batch.argtypes = [P(OrcTask), P(ctypes.c_int32), ctypes.c_int,
                                             P(ctypes.c_int32), ctypes.c_int, P(OrcStats)]
        lib.orc_heuristic.argtypes = [P(OrcTask), ctypes.c_int, ctypes.c_int, P(ctypes.c_int32),
                                      P(ctypes.c_int64)]
        lib.orc_heuristic_batch.argtypes = [P(OrcTask), P(ctypes.c_int32), ctypes.c_int,
                                            P(ctypes.c_int32), ctypes.c_int, P(ctypes.c_int32),
                                            P(ctypes.c_int64)]
        lib.orc_exhaustive_prefixes.argtypes = [P(OrcTask), P(ctypes.c_int32), P(ctypes.c_int32),
                                                P(ctypes.c_int32), P(ctypes.c_int32), ctypes.c_int,
                                                ctypes.c_int, ctypes.c_int, P(OrcStats)]
        lib.orc_predict_overlap.argtypes = [P(OrcTask), ctypes.c_int, P(ctypes.c_int32),
                                            ctypes.c_int, ctypes.c_int32, ctypes.c_int32,
                                            P(ctypes.c_int64), P(ctypes.c_int64)]
        lib.orc_exhaustive_overlap.argtypes = [P(OrcTask), ctypes.c_int, ctypes.c_int,
                                               ctypes.c_int32, ctypes.c_int32, P(OrcStats)]
        lib.orc_predict_chain.argtypes = [P(OrcTask), ctypes.c_int, ctypes.c_int,
                                          P(ctypes.c_int32), ctypes.c_int, P(ctypes.c_int64),
                                          P(ctypes.c_int64)]
        lib.orc_exhaustive_chain.argtypes = [P(OrcTask), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             P(OrcStats)]
        lib.orc_exhaustive_chain_batch.argtypes = [P(OrcTask), P(ctypes.c_int32),
                                                   P(ctypes.c_int32), ctypes.c_int,
                                                   P(ctypes.c_int32), ctypes.c_int, P(OrcStats)]
        lib.orc_hardware_threads.argtypes = []
        for f in ("orc_predict", "orc_exhaustive", "orc_exhaustive_batch", "orc_heuristic",
                  "orc_heuristic_batch", "orc_hardware_threads", "orc_exhaustive_prefixes",
                  "orc_predict_overlap", "orc_exhaustive_overlap", "orc_predict_chain",
                  "orc_exhaustive_chain", "orc_exhaustive_chain_batch"):
            getattr(lib, f).restype = ctypes.c_int
        _lib = lib
    return _lib


def _tasks(tasks) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(tasks, dtype=np.int32).reshape(-1, 3))
    return a


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"oracle {what}: invalid arguments (rc={rc})")


def hardware_threads() -> int:
    return _load().orc_hardware_threads()


def predict(tasks, order, dma_engines: int, timeline: bool = False):
    """Total time of one order (event-driven simulation, Sec. 4.1).

    With ``timeline=True`` also returns an (n, 3, 2) int64 array of
    {start, end} for the HtD, K and DtH command of the task at each position.
    """
    t = _tasks(tasks)
    o = np.ascontiguousarray(np.asarray(order, dtype=np.int32))
    n = t.shape[0]
    ms = ctypes.c_int64(0)
    tl = np.zeros(6 * n, dtype=np.int64)
    rc = _load().orc_predict(_ptr(t, OrcTask), n, _ptr(o, ctypes.c_int32), int(dma_engines),
                             ctypes.byref(ms), _ptr(tl, ctypes.c_int64))
    _check(rc, "predict")
    if timeline:
        return int(ms.value), tl.reshape(n, 3, 2)
    return int(ms.value)


def predict_overlap(tasks, order, dma_engines: int, rate_num: int, rate_den: int,
                    timeline: bool = False):
    """Total time of one order under the partial-overlap variant: concurrent
    HtD and DtH transfers each run at rate_num / rate_den of full speed, end
    times re-estimated on every change, rounded up to whole ns (Sec. 4.2.1;
    parity unpinned by the paper).  Same conventions as `predict`."""
    t = _tasks(tasks)
    o = np.ascontiguousarray(np.asarray(order, dtype=np.int32))
    n = t.shape[0]
    ms = ctypes.c_int64(0)
    tl = np.zeros(6 * n, dtype=np.int64)
    rc = _load().orc_predict_overlap(_ptr(t, OrcTask), n, _ptr(o, ctypes.c_int32),
                                     int(dma_engines), int(rate_num), int(rate_den),
                                     ctypes.byref(ms), _ptr(tl, ctypes.c_int64))
    _check(rc, "predict_overlap")
    if timeline:
        return int(ms.value), tl.reshape(n, 3, 2)
    return int(ms.value)


def exhaustive_overlap(tasks, dma_engines: int, rate_num: int, rate_den: int) -> dict:
    """Best / worst / sum / mean over all n! orders under the partial-overlap
    variant (n <= 12)."""
    t = _tasks(tasks)
    s = OrcStats()
    rc = _load().orc_exhaustive_overlap(_ptr(t, OrcTask), t.shape[0], int(dma_engines),
                                        int(rate_num), int(rate_den), ctypes.byref(s))
    _check(rc, "exhaustive_overlap")
    return _stats_dict(s, t.shape[0])


def _stats_dict(s: OrcStats, n: int) -> dict:
    return {
        "best": int(s.best), "worst": int(s.worst), "sum": int(s.sum), "mean": float(s.mean),
        "best_rank": int(s.best_rank), "worst_rank": int(s.worst_rank),
        "best_order": [int(x) for x in s.best_order[:n]],
        "worst_order": [int(x) for x in s.worst_order[:n]],
    }


def exhaustive(tasks, dma_engines: int) -> dict:
    """Best / worst / sum / mean over all n! orders (n <= 12)."""
    t = _tasks(tasks)
    s = OrcStats()
    rc = _load().orc_exhaustive(_ptr(t, OrcTask), t.shape[0], int(dma_engines), ctypes.byref(s))
    _check(rc, "exhaustive")
    return _stats_dict(s, t.shape[0])


def exhaustive_batch(tasks, offsets, dma_engines, nthreads: int = 0) -> list:
    """Per-group exhaustive statistics of a ragged batch, on host threads."""
    t = _tasks(tasks)
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32))
    G = off.shape[0] - 1
    dma = np.ascontiguousarray(np.broadcast_to(np.asarray(dma_engines, dtype=np.int32), (G,)))
    out = (OrcStats * max(G, 1))()
    rc = _load().orc_exhaustive_batch(_ptr(t, OrcTask), _ptr(off, ctypes.c_int32), G,
                                      _ptr(dma, ctypes.c_int32), int(nthreads), out)
    _check(rc, "exhaustive_batch")
    return [_stats_dict(out[g], int(off[g + 1] - off[g])) for g in range(G)]


def exhaustive_prefixes(tasks, offsets, dma_engines, item_group, item_prefix,
                        nthreads: int = 0) -> list:
    """Statistics of the orders under fixed prefixes (bounded timing samples).

    item_group[i] is a group index; item_prefix[i] the first positions of
    every order enumerated for item i (all items share one prefix length)."""
    t = _tasks(tasks)
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32))
    G = off.shape[0] - 1
    dma = np.ascontiguousarray(np.broadcast_to(np.asarray(dma_engines, dtype=np.int32), (G,)))
    grp = np.ascontiguousarray(np.asarray(item_group, dtype=np.int32))
    pre = np.ascontiguousarray(np.asarray(item_prefix, dtype=np.int32).reshape(grp.shape[0], -1))
    plen = pre.shape[1]
    out = (OrcStats * max(grp.shape[0], 1))()
    rc = _load().orc_exhaustive_prefixes(_ptr(t, OrcTask), _ptr(off, ctypes.c_int32),
                                         _ptr(dma, ctypes.c_int32), _ptr(grp, ctypes.c_int32),
                                         _ptr(pre, ctypes.c_int32), plen, grp.shape[0],
                                         int(nthreads), out)
    _check(rc, "exhaustive_prefixes")
    return [_stats_dict(out[i], int(off[grp[i] + 1] - off[grp[i]])) for i in range(grp.shape[0])]


def heuristic(tasks, dma_engines: int):
    """Order chosen by Algorithm 1 (readings H1-H5) and its total time."""
    t = _tasks(tasks)
    n = t.shape[0]
    order = np.zeros(n, dtype=np.int32)
    ms = ctypes.c_int64(0)
    rc = _load().orc_heuristic(_ptr(t, OrcTask), n, int(dma_engines), _ptr(order, ctypes.c_int32),
                               ctypes.byref(ms))
    _check(rc, "heuristic")
    return [int(x) for x in order], int(ms.value)


def heuristic_batch(tasks, offsets, dma_engines, nthreads: int = 0):
    """Heuristic orders (concatenated like the tasks) and makespans per group."""
    t = _tasks(tasks)
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32))
    G = off.shape[0] - 1
    dma = np.ascontiguousarray(np.broadcast_to(np.asarray(dma_engines, dtype=np.int32), (G,)))
    orders = np.zeros(max(t.shape[0], 1), dtype=np.int32)
    ms = np.zeros(max(G, 1), dtype=np.int64)
    rc = _load().orc_heuristic_batch(_ptr(t, OrcTask), _ptr(off, ctypes.c_int32), G,
                                     _ptr(dma, ctypes.c_int32), int(nthreads),
                                     _ptr(orders, ctypes.c_int32), _ptr(ms, ctypes.c_int64))
    _check(rc, "heuristic_batch")
    return orders[: t.shape[0]], ms[:G]


# ---- chained tasks ---------------------------------------------------------------

def predict_chain(tasks, workers: int, order, dma_engines: int, timeline: bool = False):
    """Total time of one order of a chained group (Sec. 6.1 experiment setup):
    tasks[r * workers + w] is worker w's task of round r; `order` lists the
    task indices round by round.  With ``timeline=True`` also returns the
    (n, 3, 2) {start, end} array of every position's HtD, K and DtH."""
    t = _tasks(tasks)
    o = np.ascontiguousarray(np.asarray(order, dtype=np.int32))
    n = t.shape[0]
    if int(workers) < 1 or n % int(workers):
        raise ValueError("predict_chain: the task count must be a multiple of workers")
    rounds = n // int(workers)
    ms = ctypes.c_int64(0)
    tl = np.zeros(6 * max(n, 1), dtype=np.int64)
    rc = _load().orc_predict_chain(_ptr(t, OrcTask), int(workers), rounds,
                                   _ptr(o, ctypes.c_int32), int(dma_engines), ctypes.byref(ms),
                                   _ptr(tl, ctypes.c_int64))
    _check(rc, "predict_chain")
    if timeline:
        return int(ms.value), tl[:6 * n].reshape(n, 3, 2)
    return int(ms.value)


def exhaustive_chain(tasks, workers: int, dma_engines: int) -> dict:
    """All (workers!)^rounds orders of one chained group."""
    t = _tasks(tasks)
    n = t.shape[0]
    if int(workers) < 1 or n % int(workers):
        raise ValueError("exhaustive_chain: the task count must be a multiple of workers")
    out = OrcStats()
    rc = _load().orc_exhaustive_chain(_ptr(t, OrcTask), int(workers), n // int(workers),
                                      int(dma_engines), ctypes.byref(out))
    _check(rc, "exhaustive_chain")
    return _stats_dict(out, n)


def exhaustive_chain_batch(tasks, offsets, workers, dma_engines, nthreads: int = 0) -> list:
    """exhaustive_chain of every group of a ragged batch (workers[g] per group)."""
    t = _tasks(tasks)
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32))
    G = off.shape[0] - 1
    w = np.ascontiguousarray(np.broadcast_to(np.asarray(workers, dtype=np.int32), (G,)))
    dma = np.ascontiguousarray(np.broadcast_to(np.asarray(dma_engines, dtype=np.int32), (G,)))
    out = (OrcStats * max(G, 1))()
    rc = _load().orc_exhaustive_chain_batch(_ptr(t, OrcTask), _ptr(off, ctypes.c_int32),
                                            _ptr(w, ctypes.c_int32), G, _ptr(dma, ctypes.c_int32),
                                            int(nthreads), out)
    _check(rc, "exhaustive_chain_batch")
    return [_stats_dict(out[g], int(off[g + 1] - off[g])) for g in range(G)]

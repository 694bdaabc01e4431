"""The C-ABI library builds, loads and exports every function tm.h declares.

These run without a GPU: besides symbol checks they only exercise argument
checks that the library performs on the host before any CUDA call.
"""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1806_10113_gb300 import build as tmbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def tm():
    tmbuild.build()
    from paper_1806_10113_gb300 import tm as tmmod
    return tmmod


def declared_functions():
    src = open(os.path.join(ROOT, "include", "tm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tm_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ["tm_predict", "tm_exhaustive", "tm_heuristic", "tm_predict_batch",
              "tm_exhaustive_batch", "tm_heuristic_batch", "tm_predict_batch_dev",
              "tm_heuristic_batch_dev", "tm_exhaustive_batch_dev", "tm_plan_create",
              "tm_plan_destroy", "tm_strerror"]:
        assert f in names


def test_library_exports_every_declared_symbol(tm):
    h = ctypes.CDLL(tm.LIB_PATH)
    for name in declared_functions():
        assert hasattr(h, name), name


def test_binding_names_match_header(tm):
    for name in declared_functions():
        if name.startswith("tm_plan_") or name in ("tm_strerror", "tm_version"):
            continue
        for prefix, cls in (("tm_ranker_", tm.Ranker), ("tm_server_", tm.Server)):
            if name.startswith(prefix) and not hasattr(tm, name):
                # methods of the class (create / destroy are its constructor / close)
                method = name[len(prefix):]
                assert method in ("create", "destroy") or hasattr(cls, method), name
                break
        else:
            assert hasattr(tm, name), name


def test_ranker_rows_count(tm):
    sizes = [1, 2, 3, 16, 7, 10]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
    rows, states = tm.tm_ranker_rows_count(off)
    assert rows == sum(n * (n + 1) // 2 - 1 for n in sizes if n >= 2)
    assert states == sum(n - 1 for n in sizes)
    assert tm.tm_ranker_rows_count([0]) == (0, 0)
    for bad in ([0, 17], [1, 3], [0, 2, 2]):                # n > 16, offsets[0] != 0, n = 0
        with pytest.raises(tm.TMError) as e:
            tm.tm_ranker_rows_count(bad)
        assert e.value.code == -1


def test_strerror_and_version(tm):
    assert tm.strerror(0) == "ok"
    assert "negative" in tm.strerror(-2)
    assert tm.version().startswith("tm ")


def test_tm_stats_layout_matches_numpy_dtype(tm):
    assert tm.STATS_DTYPE.itemsize == 72
    assert tm.STATS_DTYPE.fields["best_order"][1] == 40


@pytest.mark.parametrize("bad,code", [
    ([[1, -1, 0]], -2),                                  # negative duration
    ([[2**30, 2**30, 0]], -3),                           # duration sum above INT32_MAX
])
def test_host_side_rejections(tm, bad, code):
    with pytest.raises(tm.TMError) as e:
        tm.tm_predict(bad, [0], 2)
    assert e.value.code == code
    with pytest.raises(tm.TMError) as e:
        tm.tm_heuristic(bad, 2)
    assert e.value.code == code


def test_host_side_rejections_shape_and_model(tm):
    t = [[1, 2, 3], [4, 5, 6]]
    for call, code in [
        (lambda: tm.tm_predict(t, [0, 0], 2), -1),          # not a permutation
        (lambda: tm.tm_predict(t, [0, 1], 3), -1),          # bad DMA engine count
        (lambda: tm.tm_exhaustive(np.ones((13, 3)), 2), -4),  # n > 12
        (lambda: tm.tm_heuristic(np.ones((17, 3)), 2), -1),  # n > 16
        (lambda: tm.tm_predict_batch(t, [0, 2, 2], [0, 1], 2), -1),  # empty group
        (lambda: tm.tm_exhaustive_batch(t, [1, 2], 2), -1),  # offsets[0] != 0
    ]:
        with pytest.raises(tm.TMError) as e:
            call()
        assert e.value.code == code


def test_plan_rejects_sizes_without_gpu(tm):
    with pytest.raises(tm.TMError) as e:
        tm.Plan([0, 13])
    assert e.value.code == -4


def test_tuning_layout_and_rejection_on_host(tm):
    import ctypes
    assert ctypes.sizeof(tm.Tuning) == 24
    for kw in ({"pdmax": 6}, {"pdmax": 2}, {"fuse_finalize": 3}, {"chunks_per_thread": 65},
               {"fuse_finalize": 1, "chunks_per_thread": 2}, {"unroll": 9}, {"unroll": -1},
               {"item_cost": (1 << 20) + 1}):
        with pytest.raises(tm.TMError) as e:
            tm.tm_set_default_tuning(**kw)
        assert e.value.code == -1, kw
    tm.tm_set_default_tuning(fuse_finalize=1)   # chunks_per_thread 0 means 1: allowed
    tm.tm_set_default_tuning()            # back to the library's defaults


def test_server_config_rejected_on_host(tm):
    # argument checks run before any CUDA call
    for kw in ({"exact_max_n": 13}, {"exact_max_n": -1}, {"lanes": 9},
               {"beam_width": 65}, {"beam_width": 8}, {"lane_tasks": 8}):
        with pytest.raises(tm.TMError) as e:
            tm.Server(**kw)
        assert e.value.code == -1, kw


def test_result_layout(tm):
    assert tm.RESULT_DTYPE.itemsize == 96
    assert tm.RESULT_DTYPE.fields["order"][1] == 32


def test_overlap_rate_and_bound_rejected_on_host(tm):
    t = [[1, 2, 3], [4, 5, 6]]
    for num, den in ((0, 1), (3, 2), (1, 1025), (-1, 4)):
        with pytest.raises(tm.TMError) as e:
            tm.tm_predict_overlap(t, [0, 1], 2, num, den)
        assert e.value.code == -1, (num, den)
    # transfers stretched 4x pass INT32_MAX although the plain sum does not
    big = [[2**28, 1, 2**28], [2**28, 1, 2**28]]
    with pytest.raises(tm.TMError) as e:
        tm.tm_predict_overlap(big, [0, 1], 2, 1, 4)
    assert e.value.code == -3
    with pytest.raises(tm.TMError) as e:
        tm.tm_exhaustive_overlap_batch(big, [0, 2], [2], 1, 4)
    assert e.value.code == -3

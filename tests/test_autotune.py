"""Host logic of the autotuner, with the device timing replaced by a fake:
shape keys, the choice of the fastest candidate, the bit-identity check of
the candidates' results and the per-shape cache."""
import json

import pytest

from paper_1806_10113_gb300 import autotune


def test_shape_key_is_the_size_histogram():
    assert autotune.shape_key([0, 10, 20, 30]) == "n10x3"
    assert autotune.shape_key([0, 4, 9, 13, 22]) == "n4x2,n5x1,n9x1"


def _fake(times, outputs=None):
    calls = []

    def time_tuning(tasks, offsets, dma, tuning, reps=20, warmup=3, with_heuristic=True):
        key = tuple(sorted(tuning.items()))
        calls.append(key)
        out = outputs(tuning) if outputs else b"same"
        return times(tuning), out
    return time_tuning, calls


def test_picks_the_fastest_and_caches_it(tmp_path, monkeypatch):
    cands = {"pdmax": (3, 4, 5), "fuse_finalize": (2,), "blocks_per_sm": (0,),
             "item_cost": (4096,), "chunks_per_thread": (1, 3), "unroll": (1, 2)}
    fake, calls = _fake(lambda t: 1.0 + abs(t["pdmax"] - 4) + 0.1 * t["unroll"]
                        + 0.01 * t["chunks_per_thread"])
    monkeypatch.setattr(autotune, "time_tuning", fake)
    cache = str(tmp_path / "cache.json")
    best = autotune.tune(None, [0, 10, 20], [2, 1], cache_path=cache, candidates=cands)
    assert best == {"pdmax": 4, "fuse_finalize": 2, "blocks_per_sm": 0, "item_cost": 4096,
                    "chunks_per_thread": 1, "unroll": 1}
    assert len(calls) == 12
    data = json.load(open(cache))
    assert data["n10x2"]["tuning"] == best and len(data["n10x2"]["timed"]) == 12
    # a second call for the same shape reads the cache and times nothing
    calls.clear()
    assert autotune.tune(None, [0, 10, 20], [1, 1], cache_path=cache, candidates=cands) == best
    assert calls == []


def test_rejects_candidates_that_change_results(monkeypatch):
    cands = {"pdmax": (4, 5)}
    fake, _ = _fake(lambda t: 1.0, outputs=lambda t: bytes([t["pdmax"]]))
    monkeypatch.setattr(autotune, "time_tuning", fake)
    with pytest.raises(RuntimeError):
        autotune.tune(None, [0, 10], [2], cache_path=None, candidates=cands)

"""bench.py's reference arm (the oracle timed on the host cores) keeps the
JSON contract: one line, the workload's own metric and unit, `impl`,
`cpu_baseline` and a zero-copy `e2e`; the serving workload, which the
oracle cannot serve, says so in an `unavailable` line."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*extra):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3", *extra],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    return json.loads(lines[0])


@pytest.mark.parametrize("workload,unit,higher", [("dkdt64x10", "orders/s", True),
                                                   ("single6", "us", False)])
def test_reference_line(workload, unit, higher):
    d = _run("--workload", workload)
    assert d["impl"] == "reference" and d["unit"] == unit and d["higher_is_better"] is higher
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": unit, "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_default_reference_matches_the_bench_metric():
    sys.path.insert(0, ROOT)
    import bench
    d = _run()
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT


def test_serving_reference_is_unavailable():
    d = _run("--workload", "serve20k")
    assert set(d) == {"impl", "unavailable"} and d["impl"] == "reference"

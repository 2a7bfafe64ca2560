"""bench.py's reference arm (the oracle on the host cores) for every
workload: it needs no GPU, prints one JSON line with impl "reference" on
the metric, unit and config of our arm, and describes its CPU baseline."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*extra):
    cmd = [sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"] + list(extra)
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    return json.loads(lines[0])


@pytest.mark.parametrize("workload,extra,metric_key,unit", [
    ("product", ["--n", "512"], "PRODUCT_METRIC", "products/s"),
    ("serving", ["--requests", "30", "--ref-rotations", "2000"], "SERVING_METRIC", "solves/s"),
    ("batched", [], "BATCHED_METRIC", "solves/s"),
    ("cfg2", ["--ref-rotations", "3000"], "METRIC", "solves/s"),
])
def test_reference_arm_line(workload, extra, metric_key, unit):
    sys.path.insert(0, ROOT)
    import bench
    d = _run("--workload", workload, *extra)
    assert d["impl"] == "reference" and d["metric"] == getattr(bench, metric_key) and d["unit"] == unit
    assert d["value"] > 0 and d["higher_is_better"] is True and d["n_gpus"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    if workload == "serving":
        assert d["latency_ms"]["p99"] >= d["latency_ms"]["p50"] > 0


def test_reference_and_cpu_baseline_share_one_rule():
    """Both oracle legs extrapolate a timed sample to the same rotation count
    (the oracle's own count for the workload and preconditioner)."""
    sys.path.insert(0, ROOT)
    import bench
    d = _run("--workload", "cfg2", "--ref-rotations", "3000")
    need = bench.ORACLE_SOLVE_ROTATIONS[("cfg2", 1024, 3)]
    assert ("extrapolated to %d rotations" % need) in d["cpu_baseline"]["sample"]
    assert "refinement" in d["config"]["preconditioner"]

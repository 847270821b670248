"""bench.py's reference arm on CPU: the oracle timed on this host for the
workload and metric the CUDA arm reports, as one JSON line from rank 0; other
ranks exit without work or output."""
from __future__ import annotations

import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = {"impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
        "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"}


def _run(args, **env):
    e = dict(os.environ, **env)
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", *args], cwd=ROOT, env=e,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return [ln for ln in r.stdout.splitlines() if ln.strip()]


@pytest.mark.parametrize("workload,metric,unit", [
    ("er", "input edges/s to maximal matching", "edges/s"),
    ("paper_sweep", "speedup of lm_match over the sequential local max (max over the sweep)", "x"),
])
def test_reference_line(workload, metric, unit):
    import bench
    lines = _run(["--workload", workload, "--steps", "2", "--warmup", "1"])
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert KEYS <= d.keys()
    assert d["impl"] == "reference" and d["config"]["workload"] == workload
    assert d["metric"] == metric and d["unit"] == unit and d["higher_is_better"] is True
    assert metric in (bench.METRIC, bench.METRIC_SWEEP)
    assert d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_sample_is_the_named_workload():
    # ER is small enough for the oracle to take whole: the line says so
    d = json.loads(_run(["--workload", "er", "--steps", "1", "--warmup", "0"])[0])
    assert d["config"]["sample"].startswith("the whole workload: Erdos-Renyi n=10000 m=50000")


def test_other_ranks_print_nothing():
    assert _run(["--workload", "er", "--steps", "1"], RANK="1", LOCAL_RANK="1", WORLD_SIZE="2") == []

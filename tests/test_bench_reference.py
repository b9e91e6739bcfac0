"""The benchmark's reference arm (the oracle on the host cores) keeps the JSON
contract: one line with the metric, value, unit, steps, timing, the oracle as
cpu_baseline and an e2e object, for the default and the parametric workloads'
metric names (run here on small samples; no GPU)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = {"impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
        "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"}


def run(args):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *args],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    return json.loads(lines[0])


def test_reference_arm_small():
    d = run(["--workload", "small", "--steps", "1", "--warmup", "0"])
    assert KEYS <= set(d)
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "queries/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["higher_is_better"] is True and d["vs_baseline"] is None


def test_reference_arm_parametric():
    pytest.importorskip("scipy")
    d = run(["--workload", "param", "--steps", "1", "--warmup", "0"])
    assert KEYS <= set(d)
    assert d["value"] > 0 and "Algorithm 2" in d["metric"]

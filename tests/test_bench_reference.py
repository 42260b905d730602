"""The CPU reference arm of bench.py (the C oracle on the headline workload), on the CPU.

`bench.py --impl reference` must print one JSON line with the benchmark contract's keys,
measured (not extrapolated) step times, the host thread count, and the same workload
description as the GPU arm; a small mesh keeps it fast here.
"""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_a_measured_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "32",
                          "--steps", "4", "--warmup", "2"], capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert out.returncode == 0, out.stderr
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 4 and d["warmup"] == 2
    assert d["unit"] == "solves/s" and d["value"] > 0 and d["higher_is_better"] is True
    # one step is one solve, so the rate and the step time agree
    assert abs(d["value"] * d["ms_per_step"] / 1000.0 - 1.0) < 1e-9
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    cfg = d["config"]
    assert cfg["n"] == 32 and cfg["sources"] == 10 and cfg["tol"] == 1e-6 and cfg["levels"] == 4
    assert "warm-started sequence of 10 GRF sources" in cfg["workload"]
    assert 4.0 <= d["cycles_per_solve"] <= 8.0

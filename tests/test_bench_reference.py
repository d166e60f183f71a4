"""The benchmark's reference arm (the float64 oracle on host cores) on the CPU:
one JSON line with the measured rate, the cpu_baseline and e2e objects, and an
`unavailable` line for workloads the arm does not cover."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run(*args):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, capture_output=True,
                         text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout
    return json.loads(lines[0])


def test_reference_arm_line():
    d = run("--impl", "reference", "--workload", "pair2k", "--steps", "1", "--warmup", "1")
    assert d["impl"] == "reference" and d["unit"] == "GCUPS" and d["value"] > 0
    assert d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 1
    assert d["config"]["cells_per_step"] == 2000 * 1500
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "GCUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_unavailable_for_uncovered_workload():
    d = run("--impl", "reference", "--workload", "serve")
    assert d["impl"] == "reference" and "serve" in d["unavailable"]


def test_reference_arm_default_is_the_ragged_batch():
    """With no --workload the arm times the same workload as the default
    line (the 65,536-pair ragged int32 batch) and states the host's cores."""
    d = run("--impl", "reference", "--steps", "1", "--warmup", "1")
    assert d["impl"] == "reference" and d["dtype"] == "int64"
    assert d["config"]["n_pairs"] == 65536 and "ragged batch" in d["config"]["workload"]
    cb = d["cpu_baseline"]
    assert cb["host_cores"] == os.cpu_count() and 1 <= cb["cores"] <= cb["host_cores"]

"""bench.py's reference arm (the FP64 oracle timed on the host cores) on a
small workload: one JSON line with the contract's keys, the warm-up steps it
was asked for, and its unavailable line where the oracle arm does not apply."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", *args], cwd=ROOT,
                         capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, out.stdout
    return json.loads(lines[0])


def test_reference_arm_line():
    d = _run("--workload", "imag3d", "--steps", "2", "--warmup", "3")
    assert d["impl"] == "reference"
    assert d["value"] > 0 and d["unit"] == "site-updates/s"
    assert d["steps"] == 2 and d["warmup"] == 3
    assert d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert "32^3" in d["config"]["workload"]
    # the same config dict the GPU arm prints for the workload (one GPU, FP64 line)
    sys.path.insert(0, ROOT)
    import bench
    assert d["config"] == bench.workload_config(bench.WORKLOADS["imag3d"], "fp64", 1)


def test_reference_arm_unavailable_for_the_batched_sweep():
    d = _run("--workload", "batched2d", "--steps", "1", "--warmup", "3")
    assert d["impl"] == "reference" and "unavailable" in d

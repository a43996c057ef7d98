"""The benchmark's reference arm (the FP64 oracle timed on all host cores,
one whole-field forward + adjoint application per step) runs without a GPU: its one JSON line carries the keys of the benchmark contract
with the same metric and configuration as the GPU arm, and the GPU arm's
helpers compute the workload and the algorithmic bytes the roofline uses."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = {"impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
        "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
        "cpu_baseline", "e2e"}


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0", "--cpu-seconds", "0.3"],
                         cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert KEYS <= set(d)
    assert d["impl"] == "reference" and d["unit"] == "Gpts/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    # the oracle runs on every core the process may use (OpenMP over slices)
    assert d["cpu_baseline"]["cores"] == len(os.sched_getaffinity(0))
    assert "whole field" in d["cpu_baseline"]["sample"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["nx"] == 1024 and d["config"]["ny"] == 384 and d["config"]["nz"] == 72
    assert d["config"]["nvar"] == 2


def test_algorithmic_bytes_of_the_regional_workload():
    """The roofline's algorithmic bytes per application of the regional
    workload (1024 x 384, 72 levels, T and S): 56,623,104 points x 8 B plus
    393,216 horizontal points x 33 B = 465,960,960 B."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.algorithmic_bytes(1024, 384, 72, 2) == 465_960_960
    assert bench.workload_name(72).startswith("regional basin 1024x384x72")

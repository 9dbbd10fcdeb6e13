"""The benchmark's reference arm (the FP64 oracle on the host cores) prints one valid JSON line with
the contract's keys; run here on the smallest workload."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--workload", "tiny_o4_v8", "--cpu-sample", "1"],
                       capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "cpu_baseline", "e2e"):
        assert key in d
    assert d["impl"] == "reference" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_spectrum_peak_count_on_known_poles():
    """The bench counts peaks of -A (A = -(1/pi) sum Im G_pp is negative at poles with the -i eta sign):
    three Lorentzians of different weights on a grid give three peaks at their positions."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    grid = np.linspace(-1.0, -0.2, 5000)
    poles, wts, eta = [-0.9, -0.55, -0.31], [1.0, 0.3, 0.05], 0.01
    G = sum(w / (grid - p - 1j * eta) for p, w in zip(poles, wts))
    A = -G.imag / np.pi
    pk = bench.spectrum_peaks(A, grid)
    assert pk["count"] == 3
    assert np.allclose(pk["positions_ha"], poles, atol=2e-4)

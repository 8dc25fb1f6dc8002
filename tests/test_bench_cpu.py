"""bench.py's host-side pieces on CPU: the reference arm's JSON line (the oracle timed on
bounded samples) and the accuracy helpers of the batched and serving legs."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
                          "--cpu-seconds", "0.3"], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["value"] > 0.0 and d["unit"] == "GB/s" and d["higher_is_better"] is True
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def test_accuracy_helpers():
    sys.path.insert(0, ROOT)
    import bench

    rng = np.random.default_rng(3)
    X = rng.standard_normal((40, 5))
    R = bench.lapack_r(X)
    assert np.all(np.diag(R) >= 0.0) and np.allclose(np.tril(R, -1), 0.0)
    assert np.linalg.norm(R.T @ R - X.T @ X) <= 1e-13 * np.linalg.norm(X) ** 2
    assert bench.rel_err(R, R) == 0.0
    assert bench.rel_err(2.0 * R, R) == pytest.approx(1.0)
    assert bench.tolerance(8, 1e4) == pytest.approx(8e-9)
    assert bench.tolerance(8, 0.5) == pytest.approx(8e-13)  # kappa below 1 counts as 1

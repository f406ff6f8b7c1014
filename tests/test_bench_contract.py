"""The benchmark's output contract, checked on CPU through its reference arm
(the oracle on the host cores), and the product path's refusal to run
without its compiled library."""

import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                          "--warmup", "3", "--oracle-seconds", "0.5"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["unit"] == "frames/s" and d["value"] > 0
    assert d["steps"] == 1 and d["warmup"] == 3 and d["higher_is_better"] is True
    assert d["config"]["workload"].startswith("(3,6) PEG LDPC n=1008")
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_binding_fails_loudly_without_the_library(monkeypatch):
    from paper_0902_0657_gb300 import build as B
    from paper_0902_0657_gb300 import lpdec as L
    monkeypatch.setattr(B, "LIB", os.path.join(ROOT, "no_such_dir", "liblpdec.so"))
    monkeypatch.setattr(L, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        L.lpdec_default_params()


def test_serving_latency_summary_counts_unserved_frames_as_slowest():
    """Serving latencies: frames still running at a level's end (NaN) rank
    above every served frame; a percentile that falls on them is None."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    lat = np.array([0.1] * 98 + [np.nan, np.nan])   # 98 served in 100 ms, 2 cut off
    s = bench.latency_summary(lat, 100)
    assert s["p50_ms"] == pytest.approx(100.0) and s["max_served_ms"] == pytest.approx(100.0)
    assert s["p99_ms"] is None and s["p99.9_ms"] is None
    s = bench.latency_summary(np.linspace(0.001, 1.0, 1000), 1000)
    assert s["p50_ms"] == pytest.approx(501.0, rel=1e-3) and s["p99.9_ms"] == pytest.approx(1000.0)

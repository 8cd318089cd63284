"""Host-side checks of bench.py: the reference arm's JSON line (the FP64
oracle timed on the host cores) on a small R-MAT graph, and the replica
throughput aggregation."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _reference_line(*extra):
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--scale", "12", "--edges", "30000",
                          "--steps", "2", "--warmup", "1", *extra], cwd=ROOT, capture_output=True, text=True,
                         timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    return json.loads(lines[0])


def test_reference_line_counts_the_edges_it_visits():
    d = _reference_line()
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1 and d["higher_is_better"] is True
    assert d["config"]["workload"].startswith("rmat12-30000e-k3")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"]
    assert cb["host"]["nproc"] >= 1 and cb["host"]["cpu"]
    assert "60000 of 60000 directed edges" in cb["sample"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    # one step is one sampled epoch: every directed edge of this small graph, (1 + k) pair updates each
    updates = 60000 * (1 + 3)
    assert d["value"] * d["ms_per_step"] / 1e3 == pytest.approx(updates, rel=1e-6)
    # one FP64 core: far below a billion pair updates per second
    assert 1e5 < d["value"] < 1e9
    assert d["s_per_layout_extrapolated"] == pytest.approx(60000 * 4 * 30 / d["value"], rel=1e-9)


def test_replica_throughput_without_a_process_group():
    sys.path.insert(0, ROOT)
    import bench
    ups, ms = bench.replica_throughput(250.0, 1e9)
    assert ms == 250.0 and ups == pytest.approx(4e9)

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


def test_rooflines_follow_their_definitions():
    """HBM term: 4 B per directed edge + 8 B per vertex; L2 term: 64 (k+1) B per
    directed edge against the streaming-read probe; operation terms: (k+1)
    loads and (k+1) atomic adds per directed edge against the probes; the
    binding roofline is the term with the larger time."""
    import bench
    nnz, n, k, ms = 68_000_000, 4_194_304, 3, 3.5
    probes = {"l2_read_bytes_per_s": 14e12, "random_loads_per_s": 300e9, "random_atomic_adds_per_s": 200e9,
              "random_load_atomic_pairs_per_s": 80e9}
    r = bench.rooflines(nnz, n, k, ms, probes, 6689.1, "measured", 663e6, "kernel")
    hbm_bytes = 4 * nnz + 8 * (n + 1)
    assert r["hbm"]["algorithmic_bytes_per_launch"] == hbm_bytes
    assert abs(r["hbm"]["frac"] - hbm_bytes / (ms / 1e3) / 1e9 / 6689.1) < 1e-12
    assert abs(r["hbm"]["traffic_over_algorithmic"] - 663e6 / hbm_bytes) < 1e-12
    l2_bytes = 64 * (k + 1) * nnz
    assert r["l2"]["algorithmic_bytes_per_launch"] == l2_bytes
    assert abs(r["l2"]["frac"] - l2_bytes / (ms / 1e3) / 14e12) < 1e-12
    ops = (k + 1) * nnz
    assert abs(r["ops"]["bound_ms"] - 1e3 * max(ops / 300e9, ops / 200e9)) < 1e-9
    assert r["ops"]["binding"] == "atomic adds"
    assert abs(r["ops"]["mixed_frac"] - ops / 80e9 / (ms / 1e3)) < 1e-12
    assert r["binding"] is r["l2"]        # 17.4 GB at 14 TB/s outlasts 0.3 GB at 6.7 TB/s
    # without probes only the HBM term is reported, and it binds
    r = bench.rooflines(nnz, n, k, ms, None, 6689.1, "measured", None, "kernel")
    assert r["l2"] is None and r["ops"] is None and r["binding"] is r["hbm"]
    # the synchronous mode writes two 8-byte integer atomics per update
    r = bench.rooflines(nnz, n, k, ms, probes, 6689.1, "measured", None, "kernel", sync=True)
    assert r["l2"]["algorithmic_bytes_per_launch"] == 96 * (k + 1) * nnz
    assert r["ops"]["atomic_adds_per_launch"] == 2 * ops and "mixed_frac" not in r["ops"]
    # ... and its mix is one load and two integer atomics per term (probe op 4)
    probes["random_load_int64_atomic_triples_per_s"] = 50e9
    r = bench.rooflines(nnz, n, k, ms, probes, 6689.1, "measured", None, "kernel", sync=True)
    assert abs(r["ops"]["mixed_frac"] - ops / 50e9 / (ms / 1e3)) < 1e-12


def test_recorded_traffic_only_for_its_workload_and_source():
    """The DRAM bytes recorded by an ncu capture apply only to the workload,
    sampler and kernel source they were taken on."""
    import json
    import os
    import bench
    rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    e = rec["hogwild_red_k3"]
    got = bench.recorded_traffic("hogwild_red", 3, e["workload"], e["sampler"])
    if e["source_hash"] == bench.kernel_source_hash():
        assert got == float(e["dram_bytes_per_launch"])
    else:
        assert got is None
    assert bench.recorded_traffic("hogwild_red", 3, "rmat21-17000000e-k3-30ep-bfs", e["sampler"]) is None
    assert bench.recorded_traffic("hogwild_red", 3, e["workload"], "degree") is None
    assert bench.recorded_traffic("hogwild_red", 5, e["workload"], e["sampler"]) is None

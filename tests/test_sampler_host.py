"""The weighted samplers' alias tables (host side, no GPU): the library's
construction must give bit for bit the table of the oracle's independent
construction, since both sides draw negatives from it."""
import numpy as np
import pytest

import oracle
import paper_2608_01907_gb300 as snap
from synth import rmat_graph, sbm_graph, tiny_graph


@pytest.fixture(scope="module")
def lib():
    snap.build()        # cross-compiles here without a GPU; a no-op when up to date
    return snap


@pytest.mark.parametrize("name", ["sbm", "tiny", "rmat", "star"])
def test_degree_table_matches_oracle(lib, name):
    if name == "sbm":
        g = sbm_graph(seed=3)
    elif name == "tiny":
        g = tiny_graph(700, 2500, seed=5)          # isolated vertices: zero weight
    elif name == "rmat":
        g = rmat_graph(14, 60_000, seed=2)
    else:
        n = 50
        from synth import edges_to_csr
        g_rp, g_ci = edges_to_csr(n, np.zeros(n - 1, np.int64), np.arange(1, n))
        thr, al = lib.snap_sampler_table(lib.SAMPLER_DEGREE, g_rp)
        ref = oracle.Sampler.degree(g_rp)
        assert np.array_equal(thr, ref.prob) and np.array_equal(al, ref.alias)
        return
    thr, al = lib.snap_sampler_table(lib.SAMPLER_DEGREE, g.row_ptr)
    ref = oracle.Sampler.degree(g.row_ptr)
    assert np.array_equal(thr, ref.prob)
    assert np.array_equal(al, ref.alias)


@pytest.mark.parametrize("seed", range(5))
def test_weight_table_matches_oracle(lib, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 5000))
    w = (rng.pareto(1.1, n) * rng.choice([1e-6, 1.0, 1e6])).astype(np.float32)
    w[rng.random(n) < 0.2] = 0.0
    if not np.any(w > 0):
        w[0] = 1.0
    thr, al = lib.snap_sampler_table(lib.SAMPLER_WEIGHTS, node_weights=w)
    ref = oracle.Sampler.weights(w)
    assert np.array_equal(thr, ref.prob)
    assert np.array_equal(al, ref.alias)


def test_table_errors(lib):
    for bad in ([1.0, -2.0], [0.0, 0.0], [np.nan, 1.0], [np.inf, 1.0]):
        with pytest.raises(lib.SnapError) as ei:
            lib.snap_sampler_table(lib.SAMPLER_WEIGHTS, node_weights=np.array(bad, np.float32))
        assert ei.value.status == 1
    with pytest.raises(lib.SnapError):
        lib.snap_sampler_table(lib.SAMPLER_UNIFORM, np.array([0, 1, 2], np.int64))
    with pytest.raises(lib.SnapError):
        lib.snap_sampler_table(lib.SAMPLER_DEGREE, np.array([0, 0, 0], np.int64))   # no edges


def test_create_rejects_bad_sampler_options_before_device_work(lib):
    g = tiny_graph(20, 40, seed=1)
    with pytest.raises(lib.SnapError) as ei:      # WEIGHTS without weights
        lib.snap_layout_create(g.row_ptr, g.col_idx, opts=lib.make_options(sampler=lib.SAMPLER_WEIGHTS), stream=0)
    assert ei.value.status == 1
    w = np.ones(g.n, np.float32)
    w[3] = -1.0
    with pytest.raises(lib.SnapError) as ei:
        lib.snap_layout_create(g.row_ptr, g.col_idx, stream=0,
                               opts=lib.make_options(sampler=lib.SAMPLER_WEIGHTS, node_weights=w))
    assert ei.value.status == 1
    with pytest.raises(lib.SnapError) as ei:
        lib.snap_layout_create(g.row_ptr, g.col_idx, opts=lib.make_options(sampler=7), stream=0)
    assert ei.value.status == 1

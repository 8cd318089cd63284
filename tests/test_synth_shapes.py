"""The seeded input generators against the workload recipes they stand in
for: each returns a valid symmetric CSR (rows strictly ascending, no loops)
with the sizes, densities, degree skew and community mixing its recipe
states.  Nothing here touches the method's arithmetic."""
import numpy as np

from synth import (batch_sbm_graphs, initial_positions, lfr_graph, rmat_graph, sbm_graph,
                   serving_graph_pool)


def _check_csr(g):
    rp, ci = g.row_ptr, g.col_idx
    assert rp.dtype == np.int64 and ci.dtype == np.int32
    assert rp.size == g.n + 1 and rp[0] == 0 and rp[-1] == ci.size and np.all(np.diff(rp) >= 0)
    rows = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(rp))
    if ci.size:
        assert ci.min() >= 0 and ci.max() < g.n and not np.any(ci == rows)
        same_row = rows[1:] == rows[:-1]
        assert np.all(np.diff(ci.astype(np.int64))[same_row] > 0)
        fwd = rows * g.n + ci
        rev = ci.astype(np.int64) * g.n + rows
        assert np.array_equal(np.sort(fwd), np.sort(rev))
    return rows


def _mixing(g, rows):
    return float(np.mean(g.labels[rows] != g.labels[g.col_idx]))


def test_sbm_2000_recipe():
    g = sbm_graph(seed=1)
    rows = _check_csr(g)
    assert g.n == 2000 and np.array_equal(np.bincount(g.labels), [250] * 8)
    same = g.labels[rows] == g.labels[g.col_idx]
    pairs_in = 8 * 250 * 249 // 2
    pairs_out = 2000 * 1999 // 2 - pairs_in
    for edges, p, pairs in ((same.sum() // 2, 0.08, pairs_in), ((~same).sum() // 2, 0.0015, pairs_out)):
        assert abs(edges - pairs * p) < 5 * np.sqrt(pairs * p * (1 - p))
    assert g.row_ptr[-1] // 2 == 22_557          # seed 1


def test_lfr_260k_recipe():
    g = lfr_graph(seed=1)
    rows = _check_csr(g)
    assert g.n == 260_000
    assert g.row_ptr[-1] // 2 == 6_885_031       # seed 1; target 6.9M
    sizes = np.bincount(g.labels)
    assert sizes.size == 87 and sizes.sum() == g.n and sizes.min() >= 800 and sizes.max() <= 20_000
    # a share mu = 0.1 of the stubs crosses communities (de-duplication removes
    # a few more of the dense intra-community pairs)
    assert 0.09 < _mixing(g, rows) < 0.12
    deg = np.diff(g.row_ptr)
    assert abs(deg.mean() - 2 * 6.9e6 / 260_000) < 1.0
    # maximum-likelihood tail exponent above degree 60: the power law of
    # exponent 2.3, steepened slightly by the truncation at the community size
    tail = deg[deg >= 60].astype(np.float64)
    alpha = 1 + tail.size / np.log(tail / 59.5).sum()
    assert 2.2 < alpha < 2.6


def test_rmat_exact_count_and_skew():
    g = rmat_graph(16, 500_000, seed=2)
    _check_csr(g)
    assert g.n == 1 << 16 and g.row_ptr[-1] == 1_000_000
    deg = np.diff(g.row_ptr)
    assert deg.max() > 30 * deg.mean()           # a = 0.57: heavy hubs
    assert (deg == 0).mean() > 0.1               # isolated vertices stay in the graph


def test_batch_of_planted_partitions_recipe():
    graphs = batch_sbm_graphs(count=48, seed=3)
    cross = total = 0
    for g in graphs:
        rows = _check_csr(g)
        assert 100 <= g.n <= 20_000
        c = int(g.labels.max()) + 1
        assert 4 <= c <= 32
        mean_deg = g.row_ptr[-1] / g.n
        assert 5.0 < mean_deg <= 20.0
        mix = _mixing(g, rows)
        cross += mix * rows.size
        total += rows.size
        # where a community can hold its vertices' intra-community edges
        # (size >= 4x the mean degree) the realised mixing is about mu; in a
        # community of a few vertices the draws repeat pairs, de-duplication
        # removes them and the share of cross edges rises (up to ~0.23)
        if g.n / c >= 4 * mean_deg:
            assert mix < 0.12
    assert 0.08 < cross / total < 0.11
    ns = np.array([g.n for g in graphs])
    # log-uniform sizes: both ends of [100, 20000] are reached in 48 draws
    assert ns.min() < 400 and ns.max() > 5_000


def test_serving_pool_recipe():
    pool = serving_graph_pool(count=6, emax=200_000, seed=4)
    for q, g in enumerate(pool):
        _check_csr(g)
        e = g.row_ptr[-1] // 2
        assert 500 <= e <= 200_000
        if q % 2 == 0:                           # R-MAT, n = 2^ceil(log2(|E|/4))
            assert g.n & (g.n - 1) == 0 and g.n >= e // 4
        else:                                    # 8-community planted partition, n = |E|/5
            assert int(g.labels.max()) + 1 == 8
            assert 4.0 < 2 * e / g.n <= 10.0


def test_initial_positions_are_seeded_uniform_float32():
    a = initial_positions(100_000, 7)
    assert a.dtype == np.float32 and a.shape == (100_000, 2)
    assert np.array_equal(a, initial_positions(100_000, 7)) and not np.array_equal(a, initial_positions(100_000, 8))
    assert a.min() >= -1.0 and a.max() < 1.0
    assert abs(a.mean()) < 0.01 and abs(a.var() - 1 / 3) < 0.01

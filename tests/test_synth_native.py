"""The native R-MAT generator (synth/rmat_native.c) used for graphs too large
for numpy: a valid symmetric CSR with exactly the requested edges, the same
graph for any thread count, and the degree statistics of the numpy generator
(same model and rules, different random stream)."""
import numpy as np
import pytest

from synth import rmat_graph, rmat_graph_native


def _check_csr(g, m):
    rp, ci = g.row_ptr, g.col_idx
    assert rp[0] == 0 and rp[-1] == 2 * m and np.all(np.diff(rp) >= 0)
    rows = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(rp))
    assert np.all(rows != ci)                                  # no self-loops
    key = rows * g.n + ci
    assert np.all(np.diff(key) > 0)                            # rows sorted, no duplicates
    assert np.array_equal(np.sort(ci.astype(np.int64) * g.n + rows), key)   # symmetric


@pytest.mark.parametrize("scale,m", [(8, 2_000), (14, 100_000), (17, 1_000_000)])
def test_native_rmat_is_a_valid_graph_with_exact_edges(scale, m):
    _check_csr(rmat_graph_native(scale, m, seed=5), m)


def test_native_rmat_does_not_depend_on_threads():
    a = rmat_graph_native(15, 200_000, seed=7, threads=1)
    b = rmat_graph_native(15, 200_000, seed=7, threads=4)
    assert np.array_equal(a.row_ptr, b.row_ptr) and np.array_equal(a.col_idx, b.col_idx)
    c = rmat_graph_native(15, 200_000, seed=8, threads=4)
    assert not np.array_equal(a.col_idx, c.col_idx)


def test_native_rmat_matches_numpy_generator_statistics():
    nat = np.diff(rmat_graph_native(17, 1_000_000, seed=1).row_ptr)
    ref = np.diff(rmat_graph(17, 1_000_000, seed=1).row_ptr)
    assert abs((nat == 0).mean() - (ref == 0).mean()) < 0.01            # isolated share
    assert 0.8 < nat.max() / ref.max() < 1.25                           # hub size
    for q in (50, 90, 99, 99.9):
        assert abs(np.percentile(nat, q) - np.percentile(ref, q)) <= max(1.0, 0.1 * np.percentile(ref, q))

"""Pins of the oracle's weighted negative sampler (degree or caller weights):
the alias table (Walker's method, Vose's construction), the draw with
rejection of the source, and the objective whose gradient the weighted
draws follow in expectation -- Section 3.3's derivation with the sampler's
P(s|i) in place of 1/(|V|-1); Section 6 names non-uniform negatives as
future work.  Each pin checks a property fixed by the mathematics, not a
second copy of the code."""
import math
from fractions import Fraction

import numpy as np
import pytest
from scipy import stats

import oracle
from synth import tiny_graph

FULL = 0xFFFFFFFF


# --------------------------------------------------------------------------
# Alias table
# --------------------------------------------------------------------------
def test_alias_two_nodes_by_hand():
    # q = (1, 3): columns hold Q = 4, nodes bring n*q = (2, 6).  Node 0 is
    # small: it keeps 2 of column 0 and node 1 fills the other 2; node 1 is
    # left with 4 = Q and fills its own column.
    prob, alias = oracle.alias_build([1, 3])
    assert prob.tolist() == [1 << 31, FULL]
    assert alias.tolist() == [1, 1]


def test_alias_three_nodes_by_hand():
    # q = (1, 1, 2): Q = 4, n*q = (3, 3, 6).  Small queue (0, 1), large stack
    # (2).  Column 0: 3 of node 0, alias 2 (node 2 keeps 5); column 1: 3 of
    # node 1, alias 2 (node 2 keeps 4 = Q, full).
    prob, alias = oracle.alias_build([1, 1, 2])
    assert prob.tolist() == [3 << 30, 3 << 30, FULL]
    assert alias.tolist() == [2, 2, 2]


def _table_distribution(prob, alias):
    """Exact probability of each node under the table (col uniform, then
    accept col with probability prob/2^32, else its alias)."""
    n = prob.size
    p = [Fraction(0)] * n
    for c in range(n):
        keep = Fraction(int(prob[c]), 1 << 32)
        if int(alias[c]) == c:
            keep = Fraction(1)
        p[c] += keep / n
        p[int(alias[c])] += (1 - keep) / n
    return p


@pytest.mark.parametrize("case", range(6))
def test_alias_table_realises_the_weights(case):
    rng = np.random.default_rng(case)
    n = int(rng.integers(2, 60))
    if case == 0:
        q = rng.integers(0, 5, n)
    elif case == 1:
        q = rng.integers(1, 1 << 32, n, dtype=np.uint64)
    elif case == 2:
        q = np.zeros(n, np.int64)
        q[rng.integers(0, n)] = 7           # one node takes everything
    elif case == 3:
        q = (rng.pareto(1.2, n) * 100).astype(np.int64) + 1
    else:
        q = rng.integers(0, 1000, n)
    q = np.asarray(q, dtype=np.uint64)
    if q.sum() == 0:
        q[0] = 1
    prob, alias = oracle.alias_build(q)
    assert np.all((alias >= 0) & (alias < n))
    Q = int(q.sum())
    got = _table_distribution(prob, alias)
    refs = np.bincount(alias, minlength=n)
    for s in range(n):
        # each column's threshold is floor(mass * 2^32 / Q): off by < 2^-32
        bound = Fraction(1 + int(refs[s]), n << 32)
        assert abs(got[s] - Fraction(int(q[s]), Q)) <= bound, s
    # zero-weight nodes appear only in columns that never pick them
    for s in np.nonzero(q == 0)[0]:
        assert got[s] == 0


def test_alias_equal_weights_gives_full_columns():
    prob, alias = oracle.alias_build([5] * 17)
    assert np.all(prob == FULL) and np.array_equal(alias, np.arange(17))


def test_alias_rejects_zero_total():
    with pytest.raises(ValueError):
        oracle.alias_build([0, 0, 0])


def test_quantize_weights():
    q = oracle.quantize_weights(np.array([4.0, 2.0, 0.0, 1.0, 3e-10], np.float32))
    assert q.tolist()[:4] == [1 << 32, 1 << 31, 0, 1 << 30]
    w = float(np.float32(3e-10))
    assert int(q[4]) == round(w / 4.0 * 2 ** 32)
    for bad in ([1.0, -1.0], [0.0, 0.0], [1.0, np.inf], [np.nan, 1.0]):
        with pytest.raises(ValueError):
            oracle.quantize_weights(np.array(bad, np.float32))


# --------------------------------------------------------------------------
# The draw: rejection of the source, fallback after 16 rejections
# --------------------------------------------------------------------------
def _p_cond(q, i, s):
    q = [int(x) for x in q]
    Q, n = sum(q), len(q)
    rho = q[i] / Q
    r16 = rho ** 16
    rest = Q - q[i]
    return (1 - r16) * q[s] / rest + r16 / (n - 1)


def test_weighted_draw_matches_conditional_distribution():
    q = [36, 3, 1, 0]     # rho_0 = 0.9: the fallback term 0.9^16 / 3 is visible
    sam = oracle.Sampler(q)
    n, i, M = 4, 0, 60000
    draws = np.array([oracle.edge_negatives(e, 0, 5, i, n, 1, sam)[0][0] for e in range(M)])
    assert not np.any(draws == i)
    obs = np.bincount(draws, minlength=n)[1:]
    exp = np.array([_p_cond(q, i, s) for s in (1, 2, 3)]) * M
    assert exp.sum() == pytest.approx(M)
    chi2 = ((obs - exp) ** 2 / exp).sum()
    assert chi2 < stats.chi2.ppf(0.9999, df=2), (obs, exp)
    # without the fallback term node 3 would never be drawn
    assert obs[2] > 0.5 * exp[2]


def test_weighted_draw_falls_back_to_uniform_after_16_rejections():
    q = np.array([1 << 32, 0, 0, 1], np.uint64)   # the source holds all but 2^-32 of the weight
    sam = oracle.Sampler(q)
    for e in range(40):
        s, used = oracle.edge_negatives(e, 3, 9, 0, 4, 1, sam)
        assert used == 33                            # 16 attempts x 2 words + 1
        assert s[0] == oracle.uniform_negative(oracle.edge_word(e, 3, 32, 9), 0, 4)


def test_uniform_sampler_uses_one_word_per_negative():
    for e in range(20):
        s, used = oracle.edge_negatives(e, 1, 4, 3, 50, 5)
        assert used == 5
        assert s.tolist() == [oracle.uniform_negative(oracle.edge_word(e, 1, m, 4), 3, 50) for m in range(5)]


def test_weighted_negatives_consume_words_in_order():
    g = tiny_graph(30, 60, seed=2)
    sam = oracle.Sampler.degree(g.row_ptr)
    for e in range(10):
        i = int(np.searchsorted(g.row_ptr, e, side="right") - 1)
        full, used = oracle.edge_negatives(e, 2, 7, i, g.n, 6, sam)
        first, used3 = oracle.edge_negatives(e, 2, 7, i, g.n, 3, sam)
        assert full[:3].tolist() == first.tolist() and used >= used3 >= 6


# --------------------------------------------------------------------------
# The objective the weighted draws follow
# --------------------------------------------------------------------------
def test_equal_weights_objective_is_the_uniform_objective():
    g = tiny_graph(40, 90, seed=7)
    Y = np.random.default_rng(1).uniform(-2, 2, size=(g.n, 2))
    a = oracle.objective(g.row_ptr, g.col_idx, g.n, Y, 3)
    b = oracle.objective(g.row_ptr, g.col_idx, g.n, Y, 3, sampler=oracle.Sampler([3] * g.n))
    assert b["attr"] == a["attr"]
    assert b["rep"] == pytest.approx(a["rep"], rel=1e-12)


def test_weighted_gradient_matches_finite_differences():
    g = tiny_graph(9, 12, seed=3)
    Y = np.random.default_rng(2).uniform(-1.5, 1.5, size=(g.n, 2))
    sam = oracle.Sampler.degree(g.row_ptr)
    G = oracle.exact_gradient(g.row_ptr, g.col_idx, g.n, Y, 3, sampler=sam)
    h = 1e-6
    for i in range(g.n):
        for c in range(2):
            Yp, Ym = Y.copy(), Y.copy()
            Yp[i, c] += h
            Ym[i, c] -= h
            fd = (oracle.objective(g.row_ptr, g.col_idx, g.n, Yp, 3, sampler=sam)["total"]
                  - oracle.objective(g.row_ptr, g.col_idx, g.n, Ym, 3, sampler=sam)["total"]) / (2 * h)
            assert abs(fd - G[i, c]) < 1e-7 * max(1.0, abs(G[i, c]))


def test_weighted_objective_sampled_estimates_exact():
    g = tiny_graph(200, 600, seed=4)
    Y = np.random.default_rng(3).uniform(-2, 2, size=(g.n, 2))
    sam = oracle.Sampler.degree(g.row_ptr)
    ex = oracle.objective(g.row_ptr, g.col_idx, g.n, Y, 3, sampler=sam)
    sa = oracle.objective_sampled(g.row_ptr, g.col_idx, g.n, Y, 3, 2_000_000, 77, sampler=sam)
    assert sa["attr"] == pytest.approx(ex["attr"], rel=1e-12)
    assert sa["rep"] == pytest.approx(ex["rep"], rel=2e-2)


@pytest.mark.parametrize("kind", ["degree", "weights"])
def test_weighted_displacement_converges_to_its_gradient(kind):
    g = tiny_graph(8, 10, seed=5)
    rng = np.random.default_rng(6)
    Y = rng.uniform(-1.5, 1.5, size=(g.n, 2))
    if kind == "degree":
        sam = oracle.Sampler.degree(g.row_ptr)
    else:
        sam = oracle.Sampler.weights(rng.uniform(0.1, 3.0, g.n).astype(np.float32))
    k, M = 3, 20000
    Ds = np.stack([oracle.epoch_displacement(g.row_ptr, g.col_idx, g.n, Y, 0, k, seed, sampler=sam)
                   for seed in range(1, M + 1)])
    mean, se = Ds.mean(0), Ds.std(0, ddof=1) / math.sqrt(M)
    target = -2.0 * oracle.exact_gradient(g.row_ptr, g.col_idx, g.n, Y, k, sampler=sam)
    z = np.abs(mean - target) / np.maximum(se, 1e-15)
    assert z.max() < 5.0, z.max()
    # the same test rejects the uniform sampler's coefficient
    uni = -2.0 * oracle.exact_gradient(g.row_ptr, g.col_idx, g.n, Y, k)
    assert (np.abs(mean - uni) / np.maximum(se, 1e-15)).max() > 10.0

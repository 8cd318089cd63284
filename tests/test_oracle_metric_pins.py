"""Pins of the oracle's cluster metrics (Section 4.1: SI and CQ = ARI of the
ground truth against k-means of the layout), used to evaluate layouts of
graphs with planted communities."""
import math

import numpy as np
import pytest

import oracle


def test_silhouette_four_points_by_hand():
    # clusters {(0,0),(0,1)} and {(10,0),(10,1)}: for every point a = 1 and
    # b = (10 + sqrt(101)) / 2, so SI = 1 - 1/b
    Y = np.array([[0, 0], [0, 1], [10, 0], [10, 1]], float)
    b = (10 + math.sqrt(101)) / 2
    assert oracle.silhouette(Y, [0, 0, 1, 1]) == pytest.approx(1 - 1 / b, rel=1e-14)
    assert oracle.silhouette(Y, [1, 1, 0, 0]) == pytest.approx(1 - 1 / b, rel=1e-14)   # label names do not matter


def test_silhouette_limits_and_sampling():
    rng = np.random.default_rng(1)
    lab = np.repeat(np.arange(3), 50)
    far = rng.normal(size=(150, 2)) * 1e-3 + np.repeat(np.array([[0, 0], [100, 0], [0, 100]]), 50, axis=0)
    assert oracle.silhouette(far, lab) > 0.999
    mixed = rng.normal(size=(150, 2))
    assert abs(oracle.silhouette(mixed, rng.permutation(lab))) < 0.1
    # a sample of nodes averages the same per-node values
    nodes = np.arange(0, 150, 3)
    full = oracle.silhouette(far, lab)
    assert oracle.silhouette(far, lab, nodes) == pytest.approx(full, abs=1e-4)
    # singleton clusters contribute 0
    Y = np.array([[0, 0], [5, 5], [5, 6]], float)
    got = oracle.silhouette(Y, [0, 1, 1])
    b1, b2 = math.hypot(5, 5), math.hypot(5, 6)
    assert got == pytest.approx(((b1 - 1) / b1 + (b2 - 1) / b2) / 3, rel=1e-14)


def test_adjusted_rand_by_hand():
    # contingency {(0,0): 2, (0,1): 1, (1,1): 1, (1,2): 2}: I = 2, row pairs 6,
    # column pairs 3, C(6,2) = 15 -> E = 1.2, M = 4.5, ARI = 0.8 / 3.3
    assert oracle.adjusted_rand([0, 0, 0, 1, 1, 1], [0, 0, 1, 1, 2, 2]) == pytest.approx(0.8 / 3.3, rel=1e-14)
    lab = np.random.default_rng(2).integers(0, 7, 500)
    assert oracle.adjusted_rand(lab, lab) == pytest.approx(1.0)
    assert oracle.adjusted_rand(lab, (lab + 3) % 7) == pytest.approx(1.0)             # renamed clusters
    other = np.random.default_rng(3).integers(0, 7, 500)
    assert abs(oracle.adjusted_rand(lab, other)) < 0.02


def test_kmeans_recovers_separated_blobs_and_cq():
    rng = np.random.default_rng(4)
    centres = rng.uniform(-100, 100, size=(6, 2))
    lab = np.repeat(np.arange(6), 80)
    Y = centres[lab] + rng.normal(size=(480, 2))
    pred, inertia = oracle.kmeans(Y, 6, seed=3)
    assert oracle.adjusted_rand(lab, pred) == pytest.approx(1.0)
    assert inertia == pytest.approx(((Y - centres[lab]) ** 2).sum(), rel=0.05)
    assert oracle.cluster_quality(Y, lab) == pytest.approx(1.0)
    assert abs(oracle.cluster_quality(rng.normal(size=(480, 2)), lab)) < 0.05

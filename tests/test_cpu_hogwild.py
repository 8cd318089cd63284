"""The CPU throughput baseline (oracle/cpu_hogwild.c: FP32, OpenMP, the
lock-free bundle scheme of Section 3.4) lays out like Algorithm 1: on the SBM
graph its 30-epoch layouts reach the oracle's objective (Eq. 4) and NP
(Section 4.1) within 2% over 5 seeds, with one thread and with several; with
one thread and a fixed bundle order it is deterministic."""
import numpy as np
import pytest

import oracle
from synth import initial_positions, sbm_graph

SCHED = dict(kind=0, eta0=1.0, eta_min=1e-3, total_epochs=30)


@pytest.fixture(scope="module")
def sbm():
    return sbm_graph(seed=1)


@pytest.fixture(scope="module")
def oracle_scores(sbm):
    g = sbm
    out = []
    for seed in range(1, 6):
        Y = oracle.seq(g.row_ptr, g.col_idx, g.n, initial_positions(g.n, seed), 30, 3, SCHED, seed=seed)
        out.append((oracle.objective(g.row_ptr, g.col_idx, g.n, Y, 3)["total"],
                    oracle.neighborhood_preservation(g.row_ptr, g.col_idx, g.n, Y)))
    return np.array(out)


@pytest.mark.parametrize("threads", [1, 4])
def test_cpu_hogwild_quality_within_two_percent(sbm, oracle_scores, threads):
    g = sbm
    out = []
    for seed in range(1, 6):
        Y, used = oracle.cpu_hogwild(g.row_ptr, g.col_idx, g.n, initial_positions(g.n, seed), 30, 3, SCHED,
                                     seed=seed, threads=threads, order_seed=seed)
        assert used == threads and np.all(np.isfinite(Y))
        out.append((oracle.objective(g.row_ptr, g.col_idx, g.n, Y, 3)["total"],
                    oracle.neighborhood_preservation(g.row_ptr, g.col_idx, g.n, Y)))
    m, o = np.array(out).mean(0), oracle_scores.mean(0)
    print(f"cpu hogwild {threads} threads: objective {m[0]:.1f} vs {o[0]:.1f}, NP {m[1]:.4f} vs {o[1]:.4f}")
    assert abs(m[0] / o[0] - 1) < 0.02 and abs(m[1] / o[1] - 1) < 0.02


def test_cpu_hogwild_one_thread_is_deterministic(sbm):
    g = sbm
    a, _ = oracle.cpu_hogwild(g.row_ptr, g.col_idx, g.n, initial_positions(g.n, 2), 3, 3, SCHED, seed=4, threads=1)
    b, _ = oracle.cpu_hogwild(g.row_ptr, g.col_idx, g.n, initial_positions(g.n, 2), 3, 3, SCHED, seed=4, threads=1)
    assert np.array_equal(a, b)

"""Worker functions for the oracle process pools of the quality tests (they
must be importable by spawned processes)."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

SCHED = dict(kind=0, eta0=1.0, eta_min=1e-3, total_epochs=30)


def lfr_oracle_layout(seed):
    """Algorithm 1 (shuffled order), 30 epochs, k = 3, on the LFR-style graph."""
    import oracle
    from synth import initial_positions, lfr_graph
    g = lfr_graph(seed=1)
    return oracle.seq(g.row_ptr, g.col_idx, g.n, initial_positions(g.n, seed), 30, 3, SCHED, seed=seed)


def lfr_score(Y):
    """Objective (exact edge sum + 20M sampled pairs) and NP on 2,048 vertices."""
    import oracle
    from synth import lfr_graph
    g = lfr_graph(seed=1)
    nodes = np.sort(np.random.default_rng(5).choice(g.n, 2048, replace=False)).astype(np.int32)
    ob = oracle.objective_sampled(g.row_ptr, g.col_idx, g.n, Y, 3, 20_000_000, 99)["total"]
    return ob, oracle.neighborhood_preservation(g.row_ptr, g.col_idx, g.n, Y, nodes)

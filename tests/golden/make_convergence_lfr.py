"""Writes tests/golden/convergence_lfr.txt: the FP64 oracle's layouts of the
LFR-style community graph (260,000 vertices, ~6.9M edges, seed 1) after T = 10
and T = 30 epochs, scored -- the stored side of the convergence test against
T (Section 4.2, Fig. 5a; tests/test_gpu_convergence_lfr.py).

Each layout is Algorithm 1 in the oracle (FP64, edge list shuffled once),
k = 3, linear step decay from eta0 = 1 over T epochs (floor 1e-3 eta0),
initial positions and random words from seed 1.  Scores, by the oracle:
silhouette index SI (Section 4.1) of the planted communities on 2,000
vertices drawn without replacement (numpy PCG64 seed 11), and neighbourhood
preservation NP (r = 2) on 1,000 non-isolated vertices drawn from the same
generator after them.

Calls only oracle/ and synth/.  About 3 minutes of one core for T = 30; the
two runs go to a spawned process pool:

    python tests/golden/make_convergence_lfr.py
"""
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "convergence_lfr.txt")
TS = (10, 30)
K, SEED = 3, 1


def graph():
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from gpu_helpers import lfr260k
    return lfr260k()


def samples(g):
    rng = np.random.default_rng(11)
    si_nodes = np.sort(rng.choice(g.n, 2000, replace=False)).astype(np.int32)
    np_nodes = np.sort(rng.choice(np.nonzero(np.diff(g.row_ptr))[0], 1000, replace=False)).astype(np.int32)
    return si_nodes, np_nodes


def score(g, Y):
    import oracle
    si_nodes, np_nodes = samples(g)
    return (oracle.silhouette(Y, g.labels, si_nodes),
            oracle.neighborhood_preservation(g.row_ptr, g.col_idx, g.n, Y, np_nodes))


def job(T):
    import oracle
    from synth import initial_positions
    g = graph()
    t = time.time()
    Y = oracle.seq(g.row_ptr, g.col_idx, g.n, initial_positions(g.n, SEED), T, K,
                   dict(kind=0, eta0=1.0, eta_min=1e-3, total_epochs=T), seed=SEED)
    secs = time.time() - t
    si, npv = score(g, Y)
    return T, si, npv, secs


def main():
    import oracle
    oracle.build()
    assert graph().labels is not None
    with mp.get_context("spawn").Pool(len(TS)) as pool:
        rows = sorted(pool.map(job, TS))
    with open(OUT, "w") as f:
        f.write("# FP64 oracle layouts (Algorithm 1) of the LFR-style graph (260,000 vertices, seed 1), k = 3,\n"
                "# eta0 = 1 linear decay over T epochs, seed 1; SI (Section 4.1) of the planted communities on\n"
                "# 2,000 vertices and NP (r = 2) on 1,000 non-isolated vertices (PCG64 seed 11).\n"
                "# Written by tests/golden/make_convergence_lfr.py.\n"
                "# T si np oracle_seconds\n")
        for T, si, npv, secs in rows:
            f.write(f"{T} {float(si)!r} {float(npv)!r} {secs:.0f}\n")
    print(open(OUT).read())


if __name__ == "__main__":
    main()

"""Writes tests/golden/quality_rmat22_k3.txt: the FP64 oracle's layouts of the
bench's workload graph, scored -- the stored side of the full-size Hogwild
quality gate (tests/test_gpu_quality_rmat22.py).

Workload: R-MAT 2^22 nodes / 34,000,000 undirected edges (a, b, c = .57, .19,
.19, seed 1), BFS locality relabelling, k = 3 negatives, 30 epochs, linear
step decay from eta0 = 1 (floor 1e-3 eta0), seeds 1..5 (initial positions and
random words).  Each layout is Algorithm 1 in the oracle (FP64, the directed
edge list shuffled once), scored by the oracle: the objective of Eq. 4 (exact
edge sum plus 20,000,000 sampled vertex pairs, sample seed 99), the
neighbourhood preservation of Section 4.1 (r = 2) on 1,024 vertices drawn
without replacement from the non-isolated ones (numpy PCG64 seed 2024), and
where the 64 highest-degree vertices sit relative to their neighbours (hub
offset, below).

Calls only oracle/ and synth/.  About 15 minutes of one core per seed; the
seeds run in a spawned process pool:

    python tests/golden/make_quality_rmat22.py [--processes 5]
"""
import argparse
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "quality_rmat22_k3.txt")
SEEDS = (1, 2, 3, 4, 5)
K, EPOCHS = 3, 30
SCHED = dict(kind=0, eta0=1.0, eta_min=1e-3, total_epochs=EPOCHS)
PAIRS, PAIR_SEED = 20_000_000, 99
NP_NODES, NP_SEED = 1024, 2024


def graph():
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from gpu_helpers import rmat22_bfs
    return rmat22_bfs()


def np_sample(row_ptr):
    deg = np.diff(row_ptr)
    cand = np.nonzero(deg > 0)[0]
    return np.sort(np.random.default_rng(NP_SEED).choice(cand, NP_NODES, replace=False)).astype(np.int32)


def hub_offset(g, Y, hubs=64):
    """Where the highest-degree vertices end up relative to their neighbours:
    for each of the `hubs` vertices of highest degree, the distance from its
    position to the centroid of its neighbours' positions, divided by the
    neighbours' rms distance to that centroid; the mean over those vertices."""
    deg = np.diff(g.row_ptr)
    top = np.argsort(-deg, kind="stable")[:hubs]
    out = []
    for h in top:
        nb = Y[g.col_idx[g.row_ptr[h]:g.row_ptr[h + 1]]]
        c = nb.mean(axis=0)
        spread = np.sqrt(((nb - c) ** 2).sum(axis=1).mean())
        out.append(np.linalg.norm(Y[h] - c) / spread)
    return float(np.mean(out))


def score(g, Y):
    """(objective of Eq. 4, NP, hub offset) of a layout, by the oracle."""
    import oracle
    ob = oracle.objective_sampled(g.row_ptr, g.col_idx, g.n, Y, K, PAIRS, PAIR_SEED)["total"]
    return ob, oracle.neighborhood_preservation(g.row_ptr, g.col_idx, g.n, Y, np_sample(g.row_ptr)), \
        hub_offset(g, np.asarray(Y, dtype=np.float64))


def job(seed):
    import oracle
    from synth import initial_positions
    g = graph()
    t = time.time()
    Y = oracle.seq(g.row_ptr, g.col_idx, g.n, initial_positions(g.n, seed), EPOCHS, K, SCHED, seed=seed)
    secs = time.time() - t
    ob, npv, hub = score(g, Y)
    return seed, ob, npv, hub, secs


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--processes", type=int, default=len(SEEDS))
    args = ap.parse_args()
    import oracle
    oracle.build()
    graph()   # generate and cache once before the pool starts
    with mp.get_context("spawn").Pool(args.processes) as pool:
        rows = sorted(pool.map(job, SEEDS))
    with open(OUT, "w") as f:
        f.write("# FP64 oracle layouts (Algorithm 1) of R-MAT 2^22 / 34,000,000 edges, BFS relabelling,\n"
                "# k = 3, 30 epochs, eta0 = 1 linear decay; scored by the oracle: objective of Eq. 4\n"
                "# (exact edges + 20,000,000 sampled pairs, seed 99) and NP (Section 4.1, r = 2) on 1,024\n"
                "# non-isolated vertices (PCG64 seed 2024); hub offset = mean over the 64 highest-degree\n"
                "# vertices of |y_h - centroid of its neighbours| / the neighbours' rms distance to it.\n"
                "# Written by tests/golden/make_quality_rmat22.py.\n"
                "# seed objective np hub_offset oracle_seconds\n")
        for seed, ob, npv, hub, secs in rows:
            f.write(f"{seed} {float(ob)!r} {float(npv)!r} {float(hub)!r} {secs:.0f}\n")
    print(open(OUT).read())


if __name__ == "__main__":
    main()

"""Writes tests/golden/quality_rmat25_k3.txt: the FP64 oracle's layouts of a
graph whose positions do not fit in L2 -- R-MAT 2^25 nodes / 268,435,456
undirected edges (the native generator, seed 1, BFS locality relabelling;
positions 268 MB) -- scored; the stored side of
tests/test_gpu_past_l2.py.

Each layout is Algorithm 1 in the oracle (FP64, edge list shuffled once),
k = 3, 30 epochs, linear step decay from eta0 = 1 (floor 1e-3 eta0), seeds
1..3.  Scores, by the oracle: the objective of Eq. 4 (exact edge sum plus
20,000,000 sampled vertex pairs, sample seed 99) and NP (Section 4.1, r = 2)
on 1,024 non-isolated vertices (PCG64 seed 2024), as in
make_quality_rmat22.py.

Calls only oracle/ and synth/.  About two hours of one core and 9 GB of host
memory per seed; the seeds run in a spawned process pool:

    python tests/golden/make_quality_rmat25.py
"""
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
sys.path.insert(0, HERE)

OUT = os.path.join(HERE, "quality_rmat25_k3.txt")
SEEDS = (1, 2, 3)
K, EPOCHS = 3, 30
SCHED = dict(kind=0, eta0=1.0, eta_min=1e-3, total_epochs=EPOCHS)


def graph():
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from gpu_helpers import rmat25_bfs
    return rmat25_bfs()


def score(g, Y):
    import make_quality_rmat22 as mq
    return mq.score(g, Y)


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
    import oracle
    oracle.build()
    graph()   # generate and cache once before the pool starts
    with mp.get_context("spawn").Pool(len(SEEDS)) as pool:
        rows = sorted(pool.map(job, SEEDS))
    with open(OUT, "w") as f:
        f.write("# FP64 oracle layouts (Algorithm 1) of R-MAT 2^25 / 268,435,456 edges (native generator),\n"
                "# BFS relabelling, k = 3, 30 epochs, eta0 = 1 linear decay; objective of Eq. 4 (exact edges +\n"
                "# 20,000,000 sampled pairs, seed 99), NP (r = 2) on 1,024 non-isolated vertices (seed 2024),\n"
                "# hub offset as in quality_rmat22_k3.txt.  Written by tests/golden/make_quality_rmat25.py.\n"
                "# seed objective np hub_offset oracle_seconds\n")
        for seed, ob, npv, hub, secs in rows:
            f.write(f"{seed} {float(ob)!r} {float(npv)!r} {float(hub)!r} {secs:.0f}\n")
    print(open(OUT).read())


if __name__ == "__main__":
    main()

"""Layout quality against the number of epochs T (Section 4.2, Fig. 5a): the
sequential algorithm (oracle) and the two lock-free GPU modes on the LFR-style
graph (260k vertices, 6.9M edges, planted communities), k = 3, eta0 = 1, the
linear schedule over T epochs, one layout per T and mode from the same
initial positions and seed.

Scored by the oracle on every layout: SI and CQ (Section 4.1) against the
planted communities, on a fixed sample of vertices for SI, and NP (r = 2) on a
fixed sample.  Too slow for the test suite (the oracle runs every T); it runs
as a script on the GPU host:

    python tests/convergence_T.py [--T 5,10,20,30,50,80] [--out FILE]
"""
import argparse
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

CACHE = "/tmp/snap_convergence_lfr.npz"


def load():
    z = np.load(CACHE)
    return int(z["n"]), z["row_ptr"], z["col_idx"], z["labels"]


def oracle_layout(T):
    import oracle
    from synth import initial_positions
    n, rp, ci, _ = load()
    t = time.time()
    Y = oracle.seq(rp, ci, n, initial_positions(n, 1), T, 3, dict(eta0=1.0, total_epochs=T), seed=1)
    path = f"/tmp/snap_conv_oracle_{T}.npy"
    np.save(path, Y)
    return path, time.time() - t


def score(path):
    import oracle
    n, rp, ci, labels = load()
    Y = np.load(path)
    rng = np.random.default_rng(11)
    si_nodes = np.sort(rng.choice(n, 2000, replace=False)).astype(np.int32)
    np_nodes = np.sort(rng.choice(np.nonzero(np.diff(rp))[0], 1000, replace=False)).astype(np.int32)
    return dict(layout=os.path.basename(path), si=oracle.silhouette(Y, labels, si_nodes),
                cq=oracle.cluster_quality(Y, labels), np=oracle.neighborhood_preservation(rp, ci, n, Y, np_nodes))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--T", default="5,10,20,30,50,80")
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    Ts = [int(x) for x in args.T.split(",")]
    ctx = mp.get_context("spawn")
    import oracle
    import paper_2608_01907_gb300 as snap
    from synth import initial_positions, lfr_graph
    oracle.build()
    if not os.path.exists(CACHE):
        g = lfr_graph(seed=1)
        np.savez(CACHE, n=g.n, row_ptr=g.row_ptr, col_idx=g.col_idx, labels=g.labels)
    n, rp, ci, _ = load()
    pool = ctx.Pool(min(len(Ts), os.cpu_count() or 1))
    pending = pool.map_async(oracle_layout, Ts)
    import torch
    paths = []
    for mode, name in ((snap.MODE_HOGWILD_RED, "hogwild_red"), (snap.MODE_HOGWILD, "hogwild")):
        with snap.Layout(rp, ci, opts=snap.make_options(mode=mode)) as L:
            for T in Ts:
                pos = torch.from_numpy(initial_positions(n, 1)).cuda()
                L.epochs(pos, 0, T, 3, snap.linear_schedule(1.0, T), 1)
                L.check()
                p = f"/tmp/snap_conv_{name}_{T}.npy"
                np.save(p, pos.cpu().numpy().astype(np.float64))
                paths.append(p)
    oracle_runs = pending.get()
    pool.close()
    paths += [p for p, _ in oracle_runs]
    with ctx.Pool(min(len(paths), os.cpu_count() or 1)) as p2:
        rows = p2.map(score, paths)
    out = open(args.out, "w") if args.out else sys.stdout
    for r in rows:
        print(json.dumps(r), file=out)
    print(json.dumps({"workload": "lfr-260k-6.9M k=3 eta0=1", "T": Ts,
                      "oracle_seconds": [t for _, t in oracle_runs]}), file=out)
    if args.out:
        out.close()


if __name__ == "__main__":
    main()

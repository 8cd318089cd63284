"""Quality of GPU Hogwild layouts against the FP64 oracle at full size:
R-MAT 2^22 nodes / 34,000,000 undirected edges (degree-sorted BFS
relabelling), k = 3, 30 epochs, eta0 = 1, five seeds.

Too slow for the test suite (each oracle layout is ~8 G pair updates on one
core), so it runs as a script on the GPU host:

    python tests/quality_full_size.py [--seeds 5] [--np-nodes 1024] [--out FILE]

The oracle runs Algorithm 1 (shuffled edge order) for every seed in a
process pool; the GPU runs the same seeds through the C ABI.  Every layout,
GPU or oracle, is scored by the oracle: the objective of Eq. 4 (exact edge
sum, 20M sampled vertex pairs, the same pairs for all layouts) and the
neighbourhood preservation of Section 4.1 (r = 2) on a fixed sample of
vertices.  Prints one JSON line per layout and a summary line.
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

GRAPH_CACHE = "/tmp/snap_quality_rmat22.npz"
SCHED = dict(kind=0, eta0=1.0, eta_min=1e-3, total_epochs=30)


def load_graph():
    z = np.load(GRAPH_CACHE)
    return int(z["n"]), z["row_ptr"], z["col_idx"]


def oracle_layout(seed):
    import oracle
    from synth import initial_positions
    n, rp, ci = load_graph()
    t = time.time()
    Y = oracle.seq(rp, ci, n, initial_positions(n, seed), 30, 3, SCHED, seed=seed)
    np.save(f"/tmp/snap_quality_oracle_{seed}.npy", Y)
    return seed, time.time() - t


def score(args):
    path, nodes_path = args
    import oracle
    n, rp, ci = load_graph()
    Y = np.load(path)
    nodes = np.load(nodes_path)
    ob = oracle.objective_sampled(rp, ci, n, Y, 3, 20_000_000, 99)
    npm = oracle.neighborhood_preservation(rp, ci, n, Y, nodes)
    return path, ob["total"], npm


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--seeds", type=int, default=5)
    ap.add_argument("--np-nodes", type=int, default=1024)
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    ctx = mp.get_context("spawn")
    import oracle
    import paper_2608_01907_gb300 as snap
    from synth import initial_positions, rmat_graph
    oracle.build()
    if not os.path.exists(GRAPH_CACHE):
        g = rmat_graph(22, 34_000_000, seed=1)
        _, rp, ci = snap.snap_graph_reorder(g.row_ptr, g.col_idx, g.n)
        np.savez(GRAPH_CACHE, n=g.n, row_ptr=rp, col_idx=ci)
    n, rp, ci = load_graph()
    seeds = list(range(1, args.seeds + 1))
    pool = ctx.Pool(min(len(seeds), os.cpu_count() or 1))
    pending = pool.map_async(oracle_layout, seeds)

    import torch
    sched = snap.linear_schedule(1.0, 30)
    paths = []
    for mode, name in ((snap.MODE_HOGWILD, "hogwild"), (snap.MODE_HOGWILD_RED, "hogwild_red")):
        with snap.Layout(rp, ci, opts=snap.make_options(mode=mode)) as L:
            for seed in seeds:
                pos = torch.from_numpy(initial_positions(n, seed)).cuda()
                L.epochs(pos, 0, 30, 3, sched, seed)
                L.check()
                p = f"/tmp/snap_quality_{name}_{seed}.npy"
                np.save(p, pos.cpu().numpy().astype(np.float64))
                paths.append(p)
    times = pending.get()
    pool.close()
    paths += [f"/tmp/snap_quality_oracle_{s}.npy" for s in seeds]
    rng = np.random.default_rng(2024)
    deg = np.diff(rp)
    candidates = np.nonzero(deg > 0)[0]
    nodes = np.sort(rng.choice(candidates, args.np_nodes, replace=False)).astype(np.int32)
    nodes_path = "/tmp/snap_quality_np_nodes.npy"
    np.save(nodes_path, nodes)
    with ctx.Pool(min(len(paths), os.cpu_count() or 1)) as p2:
        scores = p2.map(score, [(p, nodes_path) for p in paths])
    res = {}
    lines = []
    for path, ob, npm in scores:
        kind = "hogwild_red" if "hogwild_red" in path else ("hogwild" if "hogwild" in path else "oracle")
        res.setdefault(kind, []).append((ob, npm))
        lines.append({"layout": os.path.basename(path), "objective": ob, "np": npm})
    summary = {"workload": "rmat22-34000000e-bfs k=3 30 epochs eta0=1", "seeds": seeds,
               "np_nodes": args.np_nodes, "oracle_seconds": [t for _, t in times]}
    o = np.array(res["oracle"]).mean(0)
    summary["oracle"] = {"objective": o[0], "np": o[1]}
    for kind in ("hogwild", "hogwild_red"):
        m = np.array(res[kind]).mean(0)
        summary[kind] = {"objective": m[0], "np": m[1], "objective_rel": m[0] / o[0] - 1, "np_rel": m[1] / o[1] - 1}
    out = open(args.out, "w") if args.out else sys.stdout
    for ln in lines:
        print(json.dumps(ln), file=out)
    print(json.dumps(summary), file=out)
    if args.out:
        out.close()
        print(json.dumps(summary))


if __name__ == "__main__":
    main()

"""Helpers shared by the GPU tests: run the CUDA path through the C ABI and
compare with the oracle."""
import numpy as np

import paper_2608_01907_gb300 as snap

# Per-coordinate parity gate of the synchronous mode after one epoch: FP32
# kernel against the FP64 oracle on the same Philox streams.  The error of a
# difference y_i - y_j in FP32 scales with the magnitude of the positions, not
# of the difference, so each coordinate's error is measured relative to
# max(|y|, rms(Y)).
SYNC_RTOL = 1e-4


def parity_error(gpu: np.ndarray, ref: np.ndarray) -> float:
    ref = np.asarray(ref, dtype=np.float64)
    gpu = np.asarray(gpu, dtype=np.float64)
    scale = max(float(np.sqrt((ref ** 2).mean())), 1e-30)
    return float((np.abs(gpu - ref) / np.maximum(np.abs(ref), scale)).max())


def schedule_dict(s: snap.SnapSchedule) -> dict:
    return dict(kind=s.kind, eta0=s.eta0, eta_min=s.eta_min, total_epochs=s.total_epochs)


def _row_position(q: int, L: int) -> int:
    """Stored position of the rank-q entry of an oriented row of length L:
    (a q) mod L, a the odd number from floor(0.618 L) | 1 upwards coprime with L."""
    from math import gcd
    if L <= 2:
        return q
    a = int(0.6180339887498949 * L) | 1
    while gcd(a, L) != 1:
        a += 2
    return (a * q) % L


def oriented_order(g, ascending: bool = False) -> np.ndarray:
    """Visiting order of the directed CSR edges by one Hogwild lane (built
    here from the documented rule, independently of the library): every
    undirected edge in the row of its higher-ranked endpoint (degree, then
    smaller id); a row's entries in ascending partner id, then stored at
    _row_position (or left ascending: the row order SNAP_FLAG_ASCENDING_ROWS
    selects); rows in vertex order; per entry (i, j) then (j, i)."""
    rp, ci = g.row_ptr, g.col_idx
    deg = np.diff(rp)
    order = []
    for i in range(g.n):
        row = []
        for e in range(rp[i], rp[i + 1]):
            j = ci[e]
            if deg[i] > deg[j] or (deg[i] == deg[j] and i < j):
                rev = rp[j] + int(np.searchsorted(ci[rp[j]:rp[j + 1]], i))
                assert ci[rev] == i
                row.append((e, rev))
        placed = [None] * len(row)
        for q, pair in enumerate(row):
            placed[q if ascending else _row_position(q, len(row))] = pair
        for e, rev in placed:
            order += [e, rev]
    assert sorted(order) == list(range(g.nnz))
    return np.array(order, dtype=np.int64)


def gpu_layout(torch, g, Y0, epochs, k, sched, seed, opts=None, epoch_begin=0):
    """Runs epochs on the GPU through the C ABI; returns the float32 positions."""
    pos = torch.from_numpy(np.ascontiguousarray(Y0, dtype=np.float32)).cuda()
    with snap.Layout(g.row_ptr, g.col_idx, opts=opts) as L:
        L.epochs(pos, epoch_begin, epochs, k, sched, seed)
        L.check()
    torch.cuda.synchronize()
    return pos.cpu().numpy()


def cached_graph(name: str, make):
    """A generated input graph, cached on local disk under a key that includes
    the hash of the generator sources (a changed generator never reuses a
    stale graph).  `make()` returns a synth Graph."""
    import os
    import tempfile

    from synth import Graph, source_digest
    d = os.path.join(tempfile.gettempdir(), "snap_test_cache")
    os.makedirs(d, exist_ok=True)
    path = os.path.join(d, f"{name}_{source_digest()}.npz")
    if os.path.exists(path):
        z = np.load(path)
        labels = z["labels"] if "labels" in z.files else None
        return Graph(int(z["n"]), z["row_ptr"], z["col_idx"], labels=labels, name=name)
    g = make()
    tmp = path + f".{os.getpid()}.npz"
    extra = {"labels": g.labels} if g.labels is not None else {}
    np.savez(tmp, n=g.n, row_ptr=g.row_ptr, col_idx=g.col_idx, **extra)
    os.replace(tmp, path)
    return g


def rmat22_bfs():
    """The bench's workload graph: R-MAT 2^22 / 34,000,000 undirected edges,
    BFS locality relabelling."""
    from synth import bfs_relabel, rmat_graph
    return cached_graph("rmat22_34m_bfs", lambda: bfs_relabel(rmat_graph(22, 34_000_000, seed=1)))


def lfr260k():
    """The LFR-style 260k-node / ~6.9M-edge community graph (seed 1)."""
    from synth import lfr_graph
    return cached_graph("lfr260k_s1_labelled", lambda: lfr_graph(seed=1))


def coordinate_error(gpu: np.ndarray, ref: np.ndarray) -> np.ndarray:
    """Per-vertex parity error (max over the two coordinates), each relative
    to max(|y|, rms(Y)) as in parity_error."""
    ref = np.asarray(ref, dtype=np.float64)
    gpu = np.asarray(gpu, dtype=np.float64)
    scale = max(float(np.sqrt((ref ** 2).mean())), 1e-30)
    return (np.abs(gpu - ref) / np.maximum(np.abs(ref), scale)).max(axis=1)


def rmat25_bfs():
    """A graph whose positions exceed L2: R-MAT 2^25 / 268,435,456 undirected
    edges from the native generator (seed 1), BFS locality relabelling."""
    from synth import bfs_relabel, rmat_graph_native
    return cached_graph("rmat25_268m_native_bfs", lambda: bfs_relabel(rmat_graph_native(25, 268_435_456, seed=1)))

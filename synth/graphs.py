"""Synthetic graph generators shaped like the paper's workloads (Section 4.1, Table 2).

The paper's datasets (SNAP com-*, SuiteSparse, the tsNET/DRGraph sets) are not
available here, so seeded generators stand in for their shapes:

* ``sbm_graph``      -- the 8-class graph of Fig. 1 / Fig. 3 (2,000 nodes).
* ``lfr_graph``      -- an LFR-style power-law community graph shaped like the
                        Orkut-communities teaser graph (259,019 / 6,893,156).
* ``rmat_graph``     -- an R-MAT graph shaped like com-lj (3,997,962 / 34,681,189).
* ``batch_sbm_graphs`` -- many small SBM graphs for batched launches.

Every graph comes back as a symmetric CSR (int64 ``row_ptr``, int32 ``col_idx``)
with rows sorted strictly ascending and no self-loops: each undirected edge is
stored as the two directed edges (i, j) and (j, i) (Section 3.3).  Everything is
drawn from numpy's PCG64 stream, which gives the same values on x86 and Arm.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import os

import numpy as np


@dataclass
class Graph:
    n: int
    row_ptr: np.ndarray          # int64, n + 1
    col_idx: np.ndarray          # int32, 2|E|
    labels: np.ndarray | None = None   # int32 community id per node, if any
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    @property
    def num_undirected_edges(self) -> int:
        return self.nnz // 2

    @property
    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr).astype(np.int32)


def _rng(seed: int, tag: int) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence([int(seed), int(tag)]))


def edges_to_csr(n: int, u: np.ndarray, v: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Undirected edge list (duplicates and self-loops allowed) -> symmetric CSR.

    Self-loops are dropped, duplicates merged, and both directions stored.
    Rows come out sorted ascending.
    """
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    keep = u != v
    u, v = u[keep], v[keep]
    rows = np.concatenate([u, v])
    cols = np.concatenate([v, u])
    key = np.sort(rows * n + cols)
    if key.size:
        uniq = np.empty(key.size, dtype=bool)
        uniq[0] = True
        np.not_equal(key[1:], key[:-1], out=uniq[1:])
        key = key[uniq]
    rows = key // n
    cols = (key - rows * n).astype(np.int32)
    counts = np.bincount(rows, minlength=n).astype(np.int64)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return row_ptr, cols


def _canonical_unique(n: int, u: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Sorted unique canonical keys min*n+max of the non-loop undirected edges."""
    keep = u != v
    a = np.minimum(u[keep], v[keep]).astype(np.int64)
    b = np.maximum(u[keep], v[keep]).astype(np.int64)
    key = np.sort(a * n + b)
    if key.size == 0:
        return key
    uniq = np.empty(key.size, dtype=bool)
    uniq[0] = True
    np.not_equal(key[1:], key[:-1], out=uniq[1:])
    return key[uniq]


def tiny_graph(n: int, m: int, seed: int = 0) -> Graph:
    """A small random graph: a random spanning path plus m random extra edges."""
    rng = _rng(seed, 11)
    perm = rng.permutation(n)
    u = [perm[:-1]]
    v = [perm[1:]]
    if m > 0:
        u.append(rng.integers(0, n, m))
        v.append(rng.integers(0, n, m))
    row_ptr, col_idx = edges_to_csr(n, np.concatenate(u), np.concatenate(v))
    return Graph(n, row_ptr, col_idx, name=f"tiny-n{n}-m{m}-s{seed}")


def sbm_graph(n: int = 2000, blocks: int = 8, p_in: float = 0.08, p_out: float = 0.0015,
              seed: int = 1) -> Graph:
    """Stochastic block model with equal blocks and an exact Bernoulli draw per pair.

    Stand-in for the 8-class graph of Fig. 1 and Fig. 3 (Sections 3.1-3.3).
    """
    rng = _rng(seed, 21)
    labels = (np.arange(n) * blocks // n).astype(np.int32)
    iu, ju = np.triu_indices(n, k=1)
    same = labels[iu] == labels[ju]
    prob = np.where(same, p_in, p_out)
    hit = rng.random(iu.size) < prob
    row_ptr, col_idx = edges_to_csr(n, iu[hit], ju[hit])
    return Graph(n, row_ptr, col_idx, labels=labels,
                 name=f"sbm-n{n}-b{blocks}-s{seed}",
                 meta=dict(p_in=p_in, p_out=p_out, blocks=blocks, seed=seed))


def _powerlaw_sample(rng: np.random.Generator, size: int, expo: float, lo: float, hi: float) -> np.ndarray:
    """Continuous truncated power law p(x) ~ x^-expo on [lo, hi] by inverse CDF."""
    u = rng.random(size)
    a = lo ** (1.0 - expo)
    b = hi ** (1.0 - expo)
    return (a - u * (a - b)) ** (1.0 / (1.0 - expo))


def _powerlaw_mean(expo: float, lo: float, hi: float) -> float:
    g = 1.0 - expo
    norm = (hi ** g - lo ** g) / g
    m1 = (hi ** (g + 1) - lo ** (g + 1)) / (g + 1)
    return m1 / norm


def lfr_graph(n: int = 260_000, target_edges: int = 6_900_000, degree_exp: float = 2.3,
              community_exp: float = 1.5, cmin: int = 800, cmax: int = 20_000,
              mu: float = 0.1, dmax: int = 4_000, seed: int = 1) -> Graph:
    """LFR-style power-law community graph (configuration-model stub matching).

    Stand-in for the Orkut-communities graph of the teaser (259,019 nodes /
    6,893,156 edges): degrees ~ power law (exponent 2.3) with the minimum
    calibrated so that the mean degree is 2*target_edges/n, community sizes ~
    power law in [cmin, cmax] summing to n, and a fraction mu of each node's
    stubs matched across communities.  Duplicates and self-loops are removed.
    """
    rng = _rng(seed, 31)
    # community sizes
    sizes: list[int] = []
    total = 0
    while total < n:
        s = int(_powerlaw_sample(rng, 1, community_exp, cmin, cmax + 1)[0])
        sizes.append(s)
        total += s
    over = total - n
    sizes[-1] -= over
    if sizes[-1] < cmin:
        rest = sizes.pop()
        i = 0
        while rest > 0:
            room = cmax - sizes[i % len(sizes)]
            take = min(room, rest)
            sizes[i % len(sizes)] += take
            rest -= take
            i += 1
    sizes_a = np.array(sizes, dtype=np.int64)
    labels = np.repeat(np.arange(sizes_a.size, dtype=np.int32), sizes_a)
    labels = labels[rng.permutation(n)]
    comm_size = sizes_a[labels]

    # degrees: calibrate the lower cut-off so the mean degree is on target,
    # then correct once for the edges lost to clipping and de-duplication
    want_mean = 2.0 * target_edges / n
    lo_d, hi_d = 1.0, want_mean
    for _ in range(60):
        mid = 0.5 * (lo_d + hi_d)
        if _powerlaw_mean(degree_exp, mid, dmax) < want_mean:
            lo_d = mid
        else:
            hi_d = mid
    dmin = 0.5 * (lo_d + hi_d)
    cap = np.floor((comm_size - 1) / (1.0 - mu))
    order = np.argsort(labels, kind="stable")
    bounds = np.concatenate([[0], np.cumsum(np.bincount(labels, minlength=sizes_a.size))])

    def build(lo_cut: float):
        d = np.floor(_powerlaw_sample(_rng(seed, 32), n, degree_exp, lo_cut, dmax) + 0.5)
        d = np.minimum(d, cap).astype(np.int64)
        k_in = np.rint((1.0 - mu) * d).astype(np.int64)
        k_out = d - k_in
        srng = _rng(seed, 33)
        us: list[np.ndarray] = []
        vs: list[np.ndarray] = []
        for c in range(sizes_a.size):
            members = order[bounds[c]:bounds[c + 1]]
            stubs = np.repeat(members, k_in[members])
            stubs = stubs[srng.permutation(stubs.size)]
            h = stubs.size // 2
            us.append(stubs[:h])
            vs.append(stubs[h:2 * h])
        stubs = np.repeat(np.arange(n), k_out)
        stubs = stubs[srng.permutation(stubs.size)]
        h = stubs.size // 2
        us.append(stubs[:h])
        vs.append(stubs[h:2 * h])
        return edges_to_csr(n, np.concatenate(us), np.concatenate(vs))

    row_ptr, col_idx = build(dmin)
    for _ in range(2):
        got = row_ptr[-1] / 2
        dmin *= (target_edges / got) ** 1.25
        row_ptr, col_idx = build(dmin)
    return Graph(n, row_ptr, col_idx, labels=labels,
                 name=f"lfr-n{n}-s{seed}",
                 meta=dict(degree_exp=degree_exp, mu=mu, communities=int(sizes_a.size), seed=seed))


def rmat_graph(scale: int = 22, num_edges: int = 34_000_000, a: float = 0.57, b: float = 0.19,
               c: float = 0.19, seed: int = 1, batch: int | None = None) -> Graph:
    """R-MAT graph (Chakrabarti et al. 2004) with exactly ``num_edges`` unique
    undirected non-loop edges on 2**scale nodes.

    Stand-in for com-lj (Table 2).  Edges are drawn in batches until at least
    ``num_edges`` distinct ones exist; any surplus is removed by a seeded
    uniform choice so the count is exact.  Nodes left isolated stay in the
    graph (they are empty rows but can still be drawn as negatives).
    """
    n = 1 << scale
    rng = _rng(seed, 41)
    ab = a + b
    abc = a + b + c
    keys = np.empty(0, dtype=np.int64)
    draw = batch or int(num_edges * 1.25)
    while True:
        rows = np.zeros(draw, dtype=np.int64)
        cols = np.zeros(draw, dtype=np.int64)
        for _ in range(scale):
            r = rng.random(draw, dtype=np.float32)
            rbit = r >= ab
            cbit = ((r >= a) & (r < ab)) | (r >= abc)
            rows = (rows << 1) | rbit
            cols = (cols << 1) | cbit
        new = _canonical_unique(n, rows, cols)
        merged = np.sort(np.concatenate([keys, new]))
        if merged.size:
            uniq = np.empty(merged.size, dtype=bool)
            uniq[0] = True
            np.not_equal(merged[1:], merged[:-1], out=uniq[1:])
            merged = merged[uniq]
        keys = merged
        if keys.size >= num_edges:
            break
        # draw about what is still missing, scaled by the observed duplicate rate
        frac_new = max(new.size / draw, 0.05)
        draw = int((num_edges - keys.size) / frac_new * 1.2) + 1024
    surplus = keys.size - num_edges
    if surplus > 0:
        drop = rng.choice(keys.size, size=surplus, replace=False)
        mask = np.ones(keys.size, dtype=bool)
        mask[drop] = False
        keys = keys[mask]
    u = keys // n
    v = keys - u * n
    row_ptr, col_idx = edges_to_csr(n, u, v)
    return Graph(n, row_ptr, col_idx, name=f"rmat-s{scale}-e{num_edges}-s{seed}",
                 meta=dict(a=a, b=b, c=c, d=1 - a - b - c, seed=seed))


_NATIVE = None
_NATIVE_SOURCES = ("rmat_native.c", "relabel.c")


def _native_lib():
    """The C generator (rmat_native.c), compiled with gcc on first use."""
    global _NATIVE
    if _NATIVE is not None:
        return _NATIVE
    import ctypes
    import subprocess
    here = os.path.dirname(os.path.abspath(__file__))
    srcs = [os.path.join(here, f) for f in _NATIVE_SOURCES]
    lib = os.path.join(here, "librmat_native.so")
    if not os.path.exists(lib) or os.path.getmtime(lib) < max(os.path.getmtime(s) for s in srcs):
        tmp = lib + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O3", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, *srcs])
        os.replace(tmp, lib)
    L = ctypes.CDLL(lib)
    L.rmat_native_generate.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_uint64, ctypes.c_int32, ctypes.c_void_p,
                                       ctypes.c_void_p]
    L.rmat_native_generate.restype = ctypes.c_int
    L.synth_bfs_relabel.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p]
    L.synth_bfs_relabel.restype = ctypes.c_int
    _NATIVE = L
    return L


def rmat_graph_native(scale: int, num_edges: int, a: float = 0.57, b: float = 0.19, c: float = 0.19,
                      seed: int = 1, threads: int = 0) -> Graph:
    """R-MAT graph for billions of edges (the C generator rmat_native.c, OpenMP):
    the same model and rules as rmat_graph, drawn from a counter-based stream
    (splitmix64), so the graph depends on the seed only, not on the thread
    count.  A different stream from rmat_graph: the two give different graphs
    of the same distribution."""
    n = 1 << scale
    row_ptr = np.empty(n + 1, dtype=np.int64)
    col_idx = np.empty(2 * num_edges, dtype=np.int32)
    rc = _native_lib().rmat_native_generate(scale, num_edges, a, b, c, seed, threads,
                                            row_ptr.ctypes.data, col_idx.ctypes.data)
    if rc != 0:
        raise MemoryError(f"rmat_native_generate failed ({rc})")
    return Graph(n, row_ptr, col_idx, name=f"rmat-native-s{scale}-e{num_edges}-s{seed}",
                 meta=dict(a=a, b=b, c=c, d=1 - a - b - c, seed=seed))


def bfs_relabel(g: Graph) -> Graph:
    """Breadth-first locality relabelling (synth/relabel.c): searches start at
    the highest-degree vertex not reached yet (ties: smaller id), a vertex
    appends its unreached neighbours in ascending id order, isolated vertices
    come last; rows of the result are sorted ascending.  The relabelled graph
    keeps ``meta["perm"]`` (new label of each old vertex)."""
    n = g.n
    perm = np.empty(n, dtype=np.int32)
    rp = np.empty(n + 1, dtype=np.int64)
    ci = np.empty(g.nnz, dtype=np.int32)
    src_rp = np.ascontiguousarray(g.row_ptr, dtype=np.int64)
    src_ci = np.ascontiguousarray(g.col_idx, dtype=np.int32)
    rc = _native_lib().synth_bfs_relabel(src_rp.ctypes.data, src_ci.ctypes.data, n, perm.ctypes.data,
                                         rp.ctypes.data, ci.ctypes.data)
    if rc == -1:
        raise MemoryError("synth_bfs_relabel: allocation failed")
    if rc != 0:
        raise ValueError("synth_bfs_relabel: malformed CSR")
    labels = None
    if g.labels is not None:
        labels = np.empty_like(g.labels)
        labels[perm] = g.labels
    meta = dict(g.meta)
    meta["perm"] = perm
    return Graph(n, rp, ci, labels=labels, name=g.name + "-bfs", meta=meta)


def source_digest() -> str:
    """Hash of the generator sources (this module and the C files): the key
    under which a generated input may be cached on disk, so that a change to
    a generator never reuses a stale graph."""
    import hashlib
    here = os.path.dirname(os.path.abspath(__file__))
    h = hashlib.sha256()
    for f in ("graphs.py",) + _NATIVE_SOURCES:
        with open(os.path.join(here, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def planted_partition_graph(n: int, communities: int, avg_degree: float, mu: float, rng: np.random.Generator,
                            name: str = "") -> Graph:
    """Planted-partition graph drawn as uniform random pairs: a share 1 - mu
    of the n * avg_degree / 2 edges joins two vertices of one community
    (chosen with probability proportional to its pair count), the rest two
    uniform vertices; duplicates and self-loops are removed."""
    communities = max(1, min(communities, n // 4 if n >= 8 else 1))
    m = int(round(n * avg_degree / 2))
    labels = (np.arange(n) * communities // n).astype(np.int32)
    starts = np.searchsorted(labels, np.arange(communities))
    sizes = np.diff(np.append(starts, n))
    m_in = int(round(m * (1 - mu)))
    w = sizes.astype(np.float64) ** 2
    comm = rng.choice(communities, size=m_in, p=w / w.sum())
    u_in = starts[comm] + (rng.random(m_in) * sizes[comm]).astype(np.int64)
    v_in = starts[comm] + (rng.random(m_in) * sizes[comm]).astype(np.int64)
    m_out = m - m_in
    u_out = rng.integers(0, n, m_out)
    v_out = rng.integers(0, n, m_out)
    row_ptr, col_idx = edges_to_csr(n, np.concatenate([u_in, u_out]), np.concatenate([v_in, v_out]))
    return Graph(n, row_ptr, col_idx, labels=labels, name=name)


def batch_sbm_graphs(count: int = 4096, nmin: int = 100, nmax: int = 20_000, cmin: int = 4,
                     cmax: int = 32, dmin: float = 6.0, dmax: float = 20.0, mu: float = 0.1,
                     seed: int = 1) -> list[Graph]:
    """Many small planted-partition graphs: n log-uniform in [nmin, nmax],
    U{cmin..cmax} communities, mean degree U[dmin, dmax], mixing mu."""
    rng = _rng(seed, 51)
    out = []
    for g in range(count):
        n = int(np.exp(rng.uniform(np.log(nmin), np.log(nmax))))
        ncomm = int(rng.integers(cmin, cmax + 1))
        avg = rng.uniform(dmin, dmax)
        out.append(planted_partition_graph(n, ncomm, avg, mu, rng, name=f"bsbm-{g}"))
    return out


def serving_graph_pool(count: int = 48, emin: int = 1_000, emax: int = 2_000_000, seed: int = 1) -> list[Graph]:
    """Graphs for the serving workload: half R-MAT (a, b, c = .57, .19, .19;
    n = 2^ceil(log2(|E|/4))), half 8-community planted partitions (n = |E|/5,
    mixing 0.1); |E| log-uniform in [emin, emax]."""
    rng = _rng(seed, 71)
    out = []
    for q in range(count):
        e = int(np.exp(rng.uniform(np.log(emin), np.log(emax))))
        if q % 2 == 0:
            scale = max(4, int(np.ceil(np.log2(max(e / 4, 2)))))
            out.append(rmat_graph(scale=scale, num_edges=min(e, (1 << scale) * ((1 << scale) - 1) // 4),
                                  seed=seed * 1000 + q))
        else:
            n = max(16, e // 5)
            out.append(planted_partition_graph(n, 8, 2 * e / n, 0.1, rng, name=f"pp-{q}"))
    return out


def initial_positions(n: int, seed: int = 1) -> np.ndarray:
    """(n, 2) float32 positions uniform in [-1, 1), exactly representable."""
    rng = _rng(seed, 61)
    return (rng.random((n, 2), dtype=np.float32) * np.float32(2.0) - np.float32(1.0)).astype(np.float32)

"""FP64 sequential CPU oracle for SNAP-tFDP -- TEST INFRASTRUCTURE ONLY.

(Also the bench's multi-threaded FP32 CPU baseline, ``cpu_hogwild``, from
``cpu_hogwild.c``: the paper's lock-free bundle scheme of Section 3.4.)

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never calls it and
shares no code with it: the C source ``snap_oracle.c`` restates every formula
from the paper (Table 1, Eq. 2, Eq. 4, Section 3.3, Algorithm 1, the NP metric
of Section 4.1) independently of the CUDA kernels.

Parity status per function:
  philox4x32_10               pinned (published known-answer vectors)
  uniform_negative            pinned (closed-form end points, exclusion, chi^2)
  pair_terms                  pinned (finite differences of the energies, Eq. 2)
  objective / objective_sampled pinned (n = 2 closed form, finite-difference
                              gradient, sampled vs exact)
  exact_gradient              pinned (finite differences of the objective)
  epoch_displacement          pinned (Monte-Carlo mean -> -2 grad U, Section 3.3)
  seq (Algorithm 1)           pinned (two-node closed form, n = 2 forced draw,
                              centroid invariance, rotation equivariance,
                              actual-vs-effective energy of Fig. 3a, the
                              objective and NP of full-gradient descent on
                              Eq. 4 (Fig. 3b), connectivity mapped to
                              proximity (Section 3.2))
  edge_negatives (uniform)    pinned (one epoch's updates obey Section 3.4's
                              sparsity: Delta ~ d_max/|E| + k/(|V|-1),
                              conflict probability <= (k+2) Delta)
  sync                        pinned (S = 1 equals Y + eta * displacement;
                              chunk bounds by hand; cap by closed form)
  sync_chunks                 pinned (one chunk of one equals Y + eta *
                              displacement at any Y and epoch; the chunks'
                              moves from one Y add up to it; a chunk moves
                              only the vertices its rows touch; chunks in
                              order equal sync's epoch)
  neighborhood_preservation   pinned (hand-computed 6-node case, lattice case)
  alias_build                 pinned (hand-worked two-node table; the table's
                              exact distribution equals q/Q within 2^-32 per
                              column; equal weights give full columns)
  edge_negatives (weighted)   pinned (chi^2 against P(s|i) including the
                              16-rejection fallback; forced fallback word count)
  silhouette                  pinned (hand-worked four-point value; separated
                              clusters -> 1; label permutation invariance)
  adjusted_rand               pinned (hand-worked contingency table; identical
                              and relabelled partitions -> 1; independent ~ 0)
  kmeans / cluster_quality    pinned (separated blobs recovered exactly; CQ of
                              the planted layout = 1)
  weighted objective/gradient pinned (Monte-Carlo displacement mean -> -2 grad U
                              with P(s|i); finite differences; uniform q equals
                              the uniform objective)
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "snap_oracle.c")
_LIB = os.path.join(_HERE, "libsnap_oracle.so")
_lib = None

ALPHA = 0.1
BETA = 8.0
GAMMA = 2.0


_HOG_SRC = os.path.join(_HERE, "cpu_hogwild.c")
_HOG_LIB = os.path.join(_HERE, "libcpu_hogwild.so")
_hog = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, no fused multiply-add), and the
    multi-threaded CPU Hogwild baseline (-O3, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    if force or not os.path.exists(_HOG_LIB) or os.path.getmtime(_HOG_LIB) < os.path.getmtime(_HOG_SRC):
        tmp = _HOG_LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O3", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _HOG_SRC])
        os.replace(tmp, _HOG_LIB)
    return _LIB


def cpu_hogwild(row_ptr, col_idx, n, Y0, epochs, k, schedule=None, seed=1, threads=0, epoch_begin=0,
                bundle_order=None, order_seed=7):
    """The CPU baseline (cpu_hogwild.c): FP32 lock-free epochs of Algorithm 1
    with one bundle (a source's out-edges) per thread at a time, bundles in a
    seeded random order.  Returns (positions float32 (n,2), threads used)."""
    global _hog
    if _hog is None:
        build()
        lib = ctypes.CDLL(_HOG_LIB)
        P, i32, u64, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint64, ctypes.c_double
        lib.cpu_hogwild_epochs.argtypes = [P, P, i32, P, i32, i32, i32, i32, f64, f64, i32, u64, i32, P]
        lib.cpu_hogwild_epochs.restype = ctypes.c_int
        _hog = lib
    rp, ci = _csr(row_ptr, col_idx)
    Y = np.ascontiguousarray(Y0, dtype=np.float32).copy()
    if bundle_order is None:
        bundle_order = np.random.default_rng(order_seed).permutation(n)
    order = np.ascontiguousarray(bundle_order, dtype=np.int32)
    kind, eta0, eta_min, total = _sched(schedule)
    used = _hog.cpu_hogwild_epochs(_p(rp), _p(ci), n, _p(Y), epoch_begin, epochs, k, kind, eta0, eta_min, total,
                                   seed, threads, _p(order))
    return Y, used


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    P = ctypes.c_void_p
    i32, i64, u32, u64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double
    lib.oracle_philox4x32_10.argtypes = [P, P, P]
    lib.oracle_philox4x32_10.restype = None
    lib.oracle_edge_word.argtypes = [u64, u32, u32, u64]
    lib.oracle_edge_word.restype = u32
    lib.oracle_uniform_negative.argtypes = [u32, i32, i32]
    lib.oracle_uniform_negative.restype = i32
    lib.oracle_step_size.argtypes = [i32, f64, f64, i32, i32]
    lib.oracle_step_size.restype = f64
    lib.oracle_pair_terms.argtypes = [f64, f64, P]
    lib.oracle_pair_terms.restype = None
    lib.oracle_seq.argtypes = [P, P, i32, P, i32, i32, i32, i32, f64, f64, i32, u64, i32, u64, i64, P, P, P, P]
    lib.oracle_seq.restype = ctypes.c_int
    lib.oracle_sync_chunk_bounds.argtypes = [P, i32, i32, P]
    lib.oracle_sync_chunk_bounds.restype = None
    lib.oracle_epoch_displacement.argtypes = [P, P, i32, P, i32, i32, u64, P, P, P]
    lib.oracle_epoch_displacement.restype = ctypes.c_int
    lib.oracle_sync.argtypes = [P, P, i32, P, i32, i32, i32, i32, f64, f64, i32, u64, i32, f64, P, P]
    lib.oracle_sync.restype = ctypes.c_int
    lib.oracle_sync_chunks.argtypes = [P, P, i32, P, i32, i32, i32, i32, i32, i32, f64, f64, i32, u64, f64, P, P]
    lib.oracle_sync_chunks.restype = ctypes.c_int
    lib.oracle_objective.argtypes = [P, P, i32, P, i32, P, P]
    lib.oracle_objective.restype = ctypes.c_int
    lib.oracle_objective_sampled.argtypes = [P, P, i32, P, i32, i64, u64, P, P]
    lib.oracle_objective_sampled.restype = ctypes.c_int
    lib.oracle_exact_gradient.argtypes = [P, P, i32, P, i32, P, P]
    lib.oracle_quantize_weights.argtypes = [P, i32, P]
    lib.oracle_quantize_weights.restype = ctypes.c_int
    lib.oracle_alias_build.argtypes = [P, i32, P, P]
    lib.oracle_alias_build.restype = ctypes.c_int
    lib.oracle_edge_negatives.argtypes = [u64, u32, u64, i32, i32, i32, P, P, P]
    lib.oracle_edge_negatives.restype = u32
    lib.oracle_exact_gradient.restype = ctypes.c_int
    lib.oracle_silhouette.argtypes = [P, P, i32, i32, P, i32]
    lib.oracle_silhouette.restype = f64
    lib.oracle_adjusted_rand.argtypes = [P, P, i32, i32, i32]
    lib.oracle_adjusted_rand.restype = f64
    lib.oracle_kmeans.argtypes = [P, i32, i32, i32, i32, u64, P]
    lib.oracle_kmeans.restype = f64
    lib.oracle_neighborhood_preservation.argtypes = [P, P, i32, P, P, i32]
    lib.oracle_neighborhood_preservation.restype = f64
    _lib = lib
    return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _csr(row_ptr, col_idx):
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    return rp, ci


def _positions(Y) -> np.ndarray:
    return np.array(Y, dtype=np.float64, order="C").reshape(-1, 2)


def _sched(schedule):
    if schedule is None:
        schedule = {}
    kind = int(schedule.get("kind", 0))
    eta0 = float(schedule.get("eta0", 1.0))
    eta_min = float(schedule.get("eta_min", eta0 * 1e-3))
    total = int(schedule.get("total_epochs", 30))
    return kind, eta0, eta_min, total


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().oracle_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def edge_word(e: int, t: int, w: int, seed: int) -> int:
    return int(_load().oracle_edge_word(e, t, w, seed))


def uniform_negative(word: int, i: int, n: int) -> int:
    return int(_load().oracle_uniform_negative(word, i, n))


def step_size(schedule, t: int) -> float:
    kind, eta0, eta_min, total = _sched(schedule)
    return float(_load().oracle_step_size(kind, eta0, eta_min, total, t))


def pair_terms(dx: float, dy: float) -> np.ndarray:
    """{Fa_x, Fa_y, Fr_x, Fr_y, Ua, Ur} for y_i - y_other = (dx, dy)."""
    out = np.zeros(6)
    _load().oracle_pair_terms(dx, dy, _p(out))
    return out


class Sampler:
    """Weighted negatives: integer weights q (uint64, n) and their alias table.

    ``Sampler.degree(row_ptr)`` weighs a node by its degree;
    ``Sampler.weights(w)`` quantises caller weights (float32 >= 0)."""

    def __init__(self, q):
        self.q = np.ascontiguousarray(q, dtype=np.uint64)
        self.prob, self.alias = alias_build(self.q)

    @classmethod
    def degree(cls, row_ptr):
        return cls(np.diff(np.asarray(row_ptr, dtype=np.int64)).astype(np.uint64))

    @classmethod
    def weights(cls, w):
        return cls(quantize_weights(w))


def _tables(sampler):
    if sampler is None:
        return None, None
    return _p(sampler.prob), _p(sampler.alias)


def _q(sampler):
    return _p(sampler.q) if sampler is not None else None


def quantize_weights(w) -> np.ndarray:
    wf = np.ascontiguousarray(w, dtype=np.float32)
    q = np.zeros(wf.size, dtype=np.uint64)
    if _load().oracle_quantize_weights(_p(wf), wf.size, _p(q)) != 0:
        raise ValueError("weights must be finite, >= 0 and not all zero")
    return q


def alias_build(q):
    qa = np.ascontiguousarray(q, dtype=np.uint64)
    prob = np.zeros(qa.size, dtype=np.uint32)
    alias = np.zeros(qa.size, dtype=np.int32)
    if _load().oracle_alias_build(_p(qa), qa.size, _p(prob), _p(alias)) != 0:
        raise ValueError("alias table needs n >= 1 and a positive total weight")
    return prob, alias


def edge_negatives(e, t, seed, i, n, k, sampler=None):
    """The k negatives of directed edge e (source i) in epoch t and the words used."""
    out = np.zeros(max(k, 1), dtype=np.int32)
    pr, al = _tables(sampler)
    used = _load().oracle_edge_negatives(e, t, seed, i, n, k, pr, al, _p(out))
    return out[:k], int(used)


def seq(row_ptr, col_idx, n, Y0, epochs, k, schedule=None, seed=1, shuffle_seed=None,
        epoch_begin=0, max_edges_per_epoch=-1, return_energy=False, shuffle=True, order=None,
        sampler=None):
    """Algorithm 1 (sequential, immediate updates).  Returns the final (n,2) float64.

    shuffle=False visits the directed edges in CSR order; `order` (a
    permutation of the CSR edge indices) fixes the visiting order; `sampler`
    (a Sampler) draws weighted negatives instead of uniform ones."""
    rp, ci = _csr(row_ptr, col_idx)
    Y = _positions(Y0).copy()
    kind, eta0, eta_min, total = _sched(schedule)
    en = np.zeros(max(epochs, 1))
    shuffle_seed = seed ^ 0x5DEECE66D if shuffle_seed is None else shuffle_seed
    od = None
    if order is not None:
        od = np.ascontiguousarray(order, dtype=np.int64)
        if od.size != rp[-1] or not np.array_equal(np.sort(od), np.arange(rp[-1])):
            raise ValueError("order must be a permutation of the CSR edge indices")
    rc = _load().oracle_seq(_p(rp), _p(ci), n, _p(Y), epoch_begin, epochs, k, kind, eta0, eta_min,
                            total, seed, int(bool(shuffle)), shuffle_seed, max_edges_per_epoch,
                            _p(en) if return_energy else None, _p(od) if od is not None else None,
                            *_tables(sampler))
    if rc != 0:
        raise MemoryError("oracle_seq failed to allocate")
    return (Y, en[:epochs]) if return_energy else Y


def sync_chunk_bounds(row_ptr, n, S) -> np.ndarray:
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    out = np.zeros(S + 1, dtype=np.int32)
    _load().oracle_sync_chunk_bounds(_p(rp), n, S, _p(out))
    return out


def epoch_displacement(row_ptr, col_idx, n, Y, t, k, seed, sampler=None) -> np.ndarray:
    rp, ci = _csr(row_ptr, col_idx)
    Yd = _positions(Y)
    D = np.zeros((n, 2))
    _load().oracle_epoch_displacement(_p(rp), _p(ci), n, _p(Yd), t, k, seed, *_tables(sampler), _p(D))
    return D


def sync(row_ptr, col_idx, n, Y0, epochs, k, schedule=None, seed=1, substeps=1, cap=0.0,
         epoch_begin=0, sampler=None):
    """Chunked synchronous (Jacobi) epochs.  Returns the final (n,2) float64."""
    rp, ci = _csr(row_ptr, col_idx)
    Y = _positions(Y0).copy()
    kind, eta0, eta_min, total = _sched(schedule)
    rc = _load().oracle_sync(_p(rp), _p(ci), n, _p(Y), epoch_begin, epochs, k, kind, eta0, eta_min,
                             total, seed, substeps, cap, *_tables(sampler))
    if rc != 0:
        raise MemoryError("oracle_sync failed to allocate")
    return Y


def sync_chunks(row_ptr, col_idx, n, Y, t, c_begin, c_end, substeps, k, schedule=None, seed=1, cap=0.0,
                sampler=None):
    """Chunks [c_begin, c_end) of `substeps` of epoch t of the synchronous
    mode, started from Y (any positions, e.g. another implementation's at a
    chunk boundary).  Returns the (n,2) float64 result."""
    rp, ci = _csr(row_ptr, col_idx)
    Yd = _positions(Y).copy()
    kind, eta0, eta_min, total = _sched(schedule)
    rc = _load().oracle_sync_chunks(_p(rp), _p(ci), n, _p(Yd), t, c_begin, c_end, substeps, k, kind, eta0,
                                    eta_min, total, seed, cap, *_tables(sampler))
    if rc == -2:
        raise ValueError("chunk range outside [0, substeps]")
    if rc != 0:
        raise MemoryError("oracle_sync_chunks failed to allocate")
    return Yd


def objective(row_ptr, col_idx, n, Y, k, sampler=None) -> dict:
    rp, ci = _csr(row_ptr, col_idx)
    Yd = _positions(Y)
    out = np.zeros(4)
    _load().oracle_objective(_p(rp), _p(ci), n, _p(Yd), k, _q(sampler), _p(out))
    return dict(attr=out[0], rep=out[1], total=out[2], rep_designed=out[3])


def objective_sampled(row_ptr, col_idx, n, Y, k, pairs, seed, sampler=None) -> dict:
    rp, ci = _csr(row_ptr, col_idx)
    Yd = _positions(Y)
    out = np.zeros(4)
    _load().oracle_objective_sampled(_p(rp), _p(ci), n, _p(Yd), k, pairs, seed, _q(sampler), _p(out))
    return dict(attr=out[0], rep=out[1], total=out[2])


def exact_gradient(row_ptr, col_idx, n, Y, k, sampler=None) -> np.ndarray:
    rp, ci = _csr(row_ptr, col_idx)
    Yd = _positions(Y)
    G = np.zeros((n, 2))
    _load().oracle_exact_gradient(_p(rp), _p(ci), n, _p(Yd), k, _q(sampler), _p(G))
    return G


def neighborhood_preservation(row_ptr, col_idx, n, Y, nodes=None) -> float:
    rp, ci = _csr(row_ptr, col_idx)
    Yd = _positions(Y)
    if nodes is None:
        return float(_load().oracle_neighborhood_preservation(_p(rp), _p(ci), n, _p(Yd), None, 0))
    nd = np.ascontiguousarray(nodes, dtype=np.int32)
    return float(_load().oracle_neighborhood_preservation(_p(rp), _p(ci), n, _p(Yd), _p(nd), nd.size))


def silhouette(Y, labels, nodes=None) -> float:
    """Silhouette index (Section 4.1, SI) of a layout under ground-truth labels."""
    Yd = _positions(Y)
    lab = np.ascontiguousarray(labels, dtype=np.int32)
    K = int(lab.max()) + 1
    if nodes is None:
        return float(_load().oracle_silhouette(_p(Yd), _p(lab), lab.size, K, None, 0))
    nd = np.ascontiguousarray(nodes, dtype=np.int32)
    return float(_load().oracle_silhouette(_p(Yd), _p(lab), lab.size, K, _p(nd), nd.size))


def adjusted_rand(a, b) -> float:
    la = np.ascontiguousarray(a, dtype=np.int32)
    lb = np.ascontiguousarray(b, dtype=np.int32)
    return float(_load().oracle_adjusted_rand(_p(la), _p(lb), la.size, int(la.max()) + 1, int(lb.max()) + 1))


def kmeans(Y, K, iters=100, restarts=4, seed=1):
    """(labels, inertia) of k-means on the layout."""
    Yd = _positions(Y)
    out = np.zeros(Yd.shape[0], dtype=np.int32)
    inertia = _load().oracle_kmeans(_p(Yd), Yd.shape[0], K, iters, restarts, seed, _p(out))
    if inertia < 0:
        raise ValueError("kmeans needs 1 <= K <= n")
    return out, float(inertia)


def cluster_quality(Y, labels, seed=1) -> float:
    """CQ of Section 4.1: ARI of the ground truth against k-means of the layout
    with as many clusters as labels."""
    lab = np.ascontiguousarray(labels, dtype=np.int32)
    pred, _ = kmeans(Y, int(lab.max()) + 1, seed=seed)
    return adjusted_rand(lab, pred)

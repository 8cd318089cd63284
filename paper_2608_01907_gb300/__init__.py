"""Python binding of the SNAP-tFDP C ABI (include/snap_layout.h).

Argument marshalling only: every step of a layout runs in the CUDA kernels of
libsnap_layout.so.  Device buffers are torch CUDA tensors (only their data
pointers cross the boundary), streams are torch streams, host buffers are
numpy arrays.  There is no CPU fallback: if the library is missing every
call raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import _build

__all__ = [
    "SnapError", "SnapOptions", "SnapSchedule", "MODE_HOGWILD", "MODE_HOGWILD_RED", "MODE_SYNC",
    "SAMPLER_UNIFORM", "SAMPLER_DEGREE", "SAMPLER_WEIGHTS", "build", "library_path", "load_library",
    "snap_options_default", "snap_layout_create", "snap_layout_epochs", "snap_layout_objective",
    "snap_layout_check", "snap_layout_device_bytes", "snap_memory_cached", "snap_memory_trim",
    "snap_layout_destroy", "snap_graph_reorder",
    "snap_layout_run", "snap_last_error", "Layout", "linear_schedule", "snap_sync_epochs_noalloc",
    "snap_layout_create_batch", "batch_union", "snap_layout_autotune", "MultiEpoch", "snap_sampler_table",
    "snap_layout_epochs_energy", "snap_layout_sync_chunks", "snap_layout_neighborhood_preservation",
]

MODE_HOGWILD, MODE_HOGWILD_RED, MODE_SYNC = 0, 1, 2
SAMPLER_UNIFORM, SAMPLER_DEGREE, SAMPLER_WEIGHTS = 0, 1, 2
STATUS_NAMES = {0: "SNAP_OK", 1: "SNAP_ERR_INVALID_ARG", 2: "SNAP_ERR_OUT_OF_MEMORY", 3: "SNAP_ERR_CUDA",
                4: "SNAP_ERR_TIMEOUT", 5: "SNAP_ERR_NOT_SUPPORTED", 6: "SNAP_ERR_NUMERIC"}


class SnapError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class SnapSchedule(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("total_epochs", ctypes.c_int32),
                ("eta0", ctypes.c_double), ("eta_min", ctypes.c_double)]


class SnapOptions(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("sampler", ctypes.c_int32),
                ("node_weights", ctypes.c_void_p), ("sync_substeps", ctypes.c_int32),
                ("sync_cap", ctypes.c_float), ("segment_edges", ctypes.c_int32),
                ("block_threads", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("max_inflight", ctypes.c_float)]


FLAG_CUDA_GRAPH = 1
FLAG_KEEP_CSR = 2
FLAG_ASCENDING_ROWS = 4


def linear_schedule(eta0: float = 1.0, total_epochs: int = 30, eta_min: float | None = None,
                    kind: int = 0) -> SnapSchedule:
    return SnapSchedule(kind, total_epochs, eta0, eta0 * 1e-3 if eta_min is None else eta_min)


_lib = None


def library_path() -> str:
    return _build.LIB


def build(force: bool = False, verbose: bool = False) -> str:
    return _build.build(force=force, verbose=verbose)


def load_library():
    """Load libsnap_layout.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"{_build.LIB} is missing: the CUDA library must be built first "
                           "(python -m paper_2608_01907_gb300._build)")
    lib = ctypes.CDLL(_build.LIB)
    P, i32, i64, u64, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
    st = ctypes.c_int
    lib.snap_options_default.argtypes = [P]
    lib.snap_options_default.restype = None
    lib.snap_layout_create.argtypes = [P, P, P, i32, P, P, P]
    lib.snap_layout_create.restype = st
    lib.snap_layout_create_batch.argtypes = [P, P, i32, P, i32, P, P, P]
    lib.snap_layout_create_batch.restype = st
    lib.snap_layout_epochs.argtypes = [P, P, i32, i32, i32, P, u64, P]
    lib.snap_layout_epochs.restype = st
    lib.snap_layout_epochs_energy.argtypes = [P, P, i32, i32, i32, P, u64, P, P]
    lib.snap_layout_epochs_energy.restype = st
    lib.snap_layout_sync_chunks.argtypes = [P, P, i32, i32, i32, i32, P, u64, P]
    lib.snap_layout_sync_chunks.restype = st
    lib.snap_layout_objective.argtypes = [P, P, i32, i32, i64, u64, P, P, P, P]
    lib.snap_layout_objective.restype = st
    lib.snap_layout_check.argtypes = [P, P]
    lib.snap_layout_check.restype = st
    lib.snap_layout_autotune.argtypes = [P, P, P, i32, P, u64, f64, P, P, P, P, P, P, P]
    lib.snap_layout_neighborhood_preservation.argtypes = [P, P, P, i32, P, P, P]
    lib.snap_layout_neighborhood_preservation.restype = st
    lib.snap_layout_autotune.restype = st
    lib.snap_layout_device_bytes.argtypes = [P]
    lib.snap_layout_device_bytes.restype = i64
    lib.snap_memory_cached.argtypes = [i32, P]
    lib.snap_memory_cached.restype = st
    lib.snap_memory_trim.argtypes = [i32, u64]
    lib.snap_memory_trim.restype = st
    lib.snap_layout_destroy.argtypes = [P]
    lib.snap_layout_destroy.restype = None
    lib.snap_sampler_table.argtypes = [i32, P, P, i32, P, P]
    lib.snap_sampler_table.restype = st
    lib.snap_graph_reorder.argtypes = [P, P, i32, P, P, P]
    lib.snap_graph_reorder.restype = st
    lib.snap_layout_run.argtypes = [P, P, i32, P, P, i32, i32, P, u64, P]
    lib.snap_layout_run.restype = st
    lib.snap_sync_epochs_noalloc.argtypes = [P, P, i64, i32, P, i32, i32, i32, P, u64, i32, ctypes.c_float, P]
    lib.snap_sync_epochs_noalloc.restype = st
    lib.snap_multi_create.argtypes = [i32, P]
    lib.snap_multi_create.restype = st
    lib.snap_multi_epoch.argtypes = [P, P, P, P, P, P, i32, i32, P]
    lib.snap_multi_epoch.restype = st
    lib.snap_multi_check.argtypes = [P, P]
    lib.snap_multi_check.restype = st
    lib.snap_multi_destroy.argtypes = [P]
    lib.snap_multi_destroy.restype = None
    lib.snap_last_error.argtypes = []
    lib.snap_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def snap_last_error() -> str:
    return load_library().snap_last_error().decode()


def _check(status: int):
    if status != 0:
        raise SnapError(status, snap_last_error())


def _host(a: np.ndarray, dtype) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=dtype)
    return a


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a is not None and a.size else None


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _device_positions(positions, n: int | None = None, writable: bool = True):
    import torch
    if not isinstance(positions, torch.Tensor) or not positions.is_cuda:
        raise TypeError("positions must be a CUDA torch.Tensor")
    if positions.dtype != torch.float32 or not positions.is_contiguous() or positions.dim() != 2 \
            or positions.shape[1] != 2:
        raise TypeError("positions must be a contiguous (n, 2) float32 tensor")
    if n is not None and positions.shape[0] != n:
        raise ValueError(f"positions has {positions.shape[0]} rows, the graph has {n} vertices")
    return ctypes.c_void_p(positions.data_ptr())


def snap_options_default() -> SnapOptions:
    o = SnapOptions()
    load_library().snap_options_default(ctypes.byref(o))
    return o


def make_options(mode: int = MODE_HOGWILD_RED, sync_substeps: int = 1, sync_cap: float = 0.0,
                 segment_edges: int = 0, block_threads: int = 0, sampler: int = SAMPLER_UNIFORM,
                 cuda_graph: bool = False, max_inflight: float = 0.0, node_weights=None,
                 keep_csr: bool = False, ascending_rows: bool = False) -> SnapOptions:
    """Options for snap_layout_create; node_weights (n floats) goes with SAMPLER_WEIGHTS
    and is kept alive by the returned object."""
    o = snap_options_default()
    o.mode, o.sync_substeps, o.sync_cap = mode, sync_substeps, sync_cap
    o.segment_edges, o.block_threads, o.sampler = segment_edges, block_threads, sampler
    o.flags = ((FLAG_CUDA_GRAPH if cuda_graph else 0) | (FLAG_KEEP_CSR if keep_csr else 0)
               | (FLAG_ASCENDING_ROWS if ascending_rows else 0))
    o.max_inflight = max_inflight
    if node_weights is not None:
        w = _host(node_weights, np.float32)
        o.node_weights = w.ctypes.data
        o._node_weights = w
    return o


def snap_layout_create(row_ptr, col_idx, degrees=None, n: int | None = None, opts: SnapOptions | None = None,
                       stream=None) -> ctypes.c_void_p:
    rp = _host(row_ptr, np.int64)
    ci = _host(col_idx, np.int32)
    n = rp.size - 1 if n is None else n
    dg = None if degrees is None else _host(degrees, np.int32)
    out = ctypes.c_void_p()
    _check(load_library().snap_layout_create(_ptr(rp), _ptr(ci), _ptr(dg), n,
                                             ctypes.byref(opts) if opts is not None else None,
                                             _stream(stream), ctypes.byref(out)))
    return out


def snap_layout_create_batch(row_ptr, col_idx, graph_offsets, opts: SnapOptions | None = None,
                             stream=None) -> ctypes.c_void_p:
    """Handle over the disjoint union of several graphs (see the C header)."""
    rp = _host(row_ptr, np.int64)
    ci = _host(col_idx, np.int32)
    go = _host(graph_offsets, np.int32)
    out = ctypes.c_void_p()
    _check(load_library().snap_layout_create_batch(_ptr(rp), _ptr(ci), rp.size - 1, _ptr(go), go.size - 1,
                                                   ctypes.byref(opts) if opts is not None else None,
                                                   _stream(stream), ctypes.byref(out)))
    return out


def snap_layout_epochs(h, positions, epoch_begin: int, epochs: int, neg_samples: int, schedule: SnapSchedule,
                       seed: int, stream=None) -> None:
    _check(load_library().snap_layout_epochs(h, _device_positions(positions), epoch_begin, epochs, neg_samples,
                                             ctypes.byref(schedule), seed, _stream(stream)))


def snap_layout_epochs_energy(h, positions, epoch_begin: int, epochs: int, neg_samples: int,
                              schedule: SnapSchedule, seed: int, energy, stream=None) -> None:
    """As snap_layout_epochs, also writing each epoch's actual energy into
    `energy` (a CUDA float64 tensor of `epochs` elements)."""
    if not (energy.is_cuda and energy.dtype.is_floating_point and energy.element_size() == 8
            and energy.is_contiguous() and energy.numel() >= epochs):
        raise ValueError("energy must be a contiguous CUDA float64 tensor with `epochs` elements")
    _check(load_library().snap_layout_epochs_energy(h, _device_positions(positions), epoch_begin, epochs,
                                                    neg_samples, ctypes.byref(schedule), seed,
                                                    ctypes.c_void_p(energy.data_ptr()), _stream(stream)))


def snap_layout_sync_chunks(h, positions, epoch: int, chunk_begin: int, chunk_end: int, neg_samples: int,
                            schedule: SnapSchedule, seed: int, stream=None) -> None:
    """Chunks [chunk_begin, chunk_end) of epoch `epoch` of a SYNC handle."""
    _check(load_library().snap_layout_sync_chunks(h, _device_positions(positions), epoch, chunk_begin, chunk_end,
                                                  neg_samples, ctypes.byref(schedule), seed, _stream(stream)))


def snap_layout_objective(h, positions, neg_samples: int, exact: bool = True, pair_samples: int = 0,
                          seed: int = 0, stream=None) -> tuple[float, float, float]:
    a, r, t = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(load_library().snap_layout_objective(h, _device_positions(positions), neg_samples, int(bool(exact)),
                                                pair_samples, seed, ctypes.byref(a), ctypes.byref(r),
                                                ctypes.byref(t), _stream(stream)))
    return a.value, r.value, t.value


def snap_layout_check(h, stream=None) -> None:
    _check(load_library().snap_layout_check(h, _stream(stream)))


def snap_layout_autotune(h, scratch_positions, neg_samples: int, schedule: SnapSchedule, seed: int,
                         initial_positions=None, tolerance: float = 0.02, stream=None):
    """Returns (chunk entries, block threads, ms per epoch, objective, NP, row
    order) chosen for the handle; tolerance < 0 (or no initial positions) times
    the candidates only.  NP is NaN unless the handle keeps its CSR
    (keep_csr); row order 0 is the affine order, 1 ascending partner id."""
    if initial_positions is None:
        tolerance = -1.0
    seg, blk, order = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    ms, u, npv = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    init = _device_positions(initial_positions) if initial_positions is not None else None
    _check(load_library().snap_layout_autotune(h, init, _device_positions(scratch_positions), neg_samples,
                                               ctypes.byref(schedule), seed, tolerance, ctypes.byref(seg),
                                               ctypes.byref(blk), ctypes.byref(order), ctypes.byref(ms),
                                               ctypes.byref(u), ctypes.byref(npv), _stream(stream)))
    return seg.value, blk.value, ms.value, u.value, npv.value, order.value


def snap_layout_neighborhood_preservation(h, positions, nodes, stream=None):
    """NP (Section 4.1, r = 2) of device positions on the sampled vertices
    `nodes`; returns (mean over samples with neighbours, their count)."""
    nd = _host(nodes, np.int32)
    mean, used = ctypes.c_double(), ctypes.c_int32()
    _check(load_library().snap_layout_neighborhood_preservation(h, _device_positions(positions), _ptr(nd), nd.size,
                                                                ctypes.byref(mean), ctypes.byref(used),
                                                                _stream(stream)))
    return mean.value, used.value


def snap_layout_device_bytes(h) -> int:
    return int(load_library().snap_layout_device_bytes(h))


def snap_memory_cached(device: int = 0) -> int:
    """Device bytes the library's memory pool on `device` holds for reuse."""
    out = ctypes.c_uint64()
    _check(load_library().snap_memory_cached(device, ctypes.byref(out)))
    return int(out.value)


def snap_memory_trim(device: int = 0, keep_bytes: int = 0) -> None:
    """Give the pool's cached memory on `device` back, down to keep_bytes."""
    _check(load_library().snap_memory_trim(device, keep_bytes))


def snap_layout_destroy(h) -> None:
    load_library().snap_layout_destroy(h)


def snap_sampler_table(sampler: int, row_ptr=None, node_weights=None, n: int | None = None):
    """(threshold uint32[n], alias int32[n]) of a weighted sampler (see the C header)."""
    rp = None if row_ptr is None else _host(row_ptr, np.int64)
    w = None if node_weights is None else _host(node_weights, np.float32)
    if n is None:
        n = rp.size - 1 if rp is not None else w.size
    thr = np.zeros(n, np.uint32)
    al = np.zeros(n, np.int32)
    _check(load_library().snap_sampler_table(sampler, _ptr(rp), _ptr(w), n, _ptr(thr), _ptr(al)))
    return thr, al


def snap_graph_reorder(row_ptr, col_idx, n: int | None = None):
    """Returns (perm[old] = new, row_ptr_out, col_idx_out)."""
    rp = _host(row_ptr, np.int64)
    ci = _host(col_idx, np.int32)
    n = rp.size - 1 if n is None else n
    perm = np.empty(n, dtype=np.int32)
    rpo = np.empty(n + 1, dtype=np.int64)
    cio = np.empty(ci.size, dtype=np.int32)
    _check(load_library().snap_graph_reorder(_ptr(rp), _ptr(ci), n, _ptr(perm), _ptr(rpo), _ptr(cio)))
    return perm, rpo, cio


def snap_layout_run(row_ptr, col_idx, positions_host, epochs: int, neg_samples: int, schedule: SnapSchedule,
                    seed: int, n: int | None = None, opts: SnapOptions | None = None, stream=None):
    """Whole layout from host buffers; positions_host ((n,2) float32, C order) is updated in place.

    positions_host may be a numpy array or a (pinned) CPU torch tensor."""
    rp = _host(row_ptr, np.int64)
    ci = _host(col_idx, np.int32)
    n = rp.size - 1 if n is None else n
    try:
        import torch
        is_tensor = isinstance(positions_host, torch.Tensor)
    except ImportError:
        is_tensor = False
    if is_tensor:
        if positions_host.is_cuda or positions_host.dtype != torch.float32 or not positions_host.is_contiguous():
            raise TypeError("positions_host must be a contiguous float32 CPU tensor")
        pp = ctypes.c_void_p(positions_host.data_ptr())
    else:
        if not (isinstance(positions_host, np.ndarray) and positions_host.dtype == np.float32
                and positions_host.flags.c_contiguous):
            raise TypeError("positions_host must be a C-contiguous float32 numpy array")
        pp = ctypes.c_void_p(positions_host.ctypes.data)
    _check(load_library().snap_layout_run(_ptr(rp), _ptr(ci), n, ctypes.byref(opts) if opts is not None else None,
                                          pp, epochs, neg_samples, ctypes.byref(schedule), seed, _stream(stream)))
    return positions_host


def batch_union(graphs):
    """Disjoint union of (row_ptr, col_idx) CSRs: returns (row_ptr, col_idx,
    graph_offsets) with graph g's vertices relabelled by its offset."""
    offs = [0]
    rps, cis = [], []
    ebase = 0
    for rp, ci in graphs:
        rp = np.asarray(rp, dtype=np.int64)
        ci = np.asarray(ci, dtype=np.int32)
        rps.append(rp[:-1] + ebase)
        cis.append(ci + offs[-1])
        ebase += int(rp[-1])
        offs.append(offs[-1] + rp.size - 1)
    row_ptr = np.concatenate(rps + [np.array([ebase], dtype=np.int64)])
    col_idx = np.concatenate(cis) if cis else np.zeros(0, np.int32)
    return row_ptr, col_idx.astype(np.int32), np.array(offs, dtype=np.int32)


def snap_sync_epochs_noalloc(row_ptr, col_idx, positions, epoch_begin: int, epochs: int, neg_samples: int,
                             schedule: SnapSchedule, seed: int, substeps: int = 1, cap: float = 0.0,
                             stream=None) -> None:
    """Synchronous epochs without any device allocation (see the C header).

    row_ptr (int64), col_idx (int32) and positions ((n, 2) float32) are CUDA
    tensors the caller owns, all on one device; n is positions.shape[0] (at
    most 262,144) and nnz is col_idx.numel().  The call runs with that device
    current."""
    import torch
    for t, dt in ((row_ptr, torch.int64), (col_idx, torch.int32)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dt or not t.is_contiguous():
            raise TypeError("row_ptr / col_idx must be contiguous CUDA tensors (int64 / int32)")
    p = _device_positions(positions)
    if not (row_ptr.device == col_idx.device == positions.device):
        raise ValueError("row_ptr, col_idx and positions must be on the same CUDA device")
    n = int(positions.shape[0])
    if row_ptr.numel() != n + 1:
        raise ValueError("row_ptr must have n + 1 entries")
    with torch.cuda.device(positions.device):
        _check(load_library().snap_sync_epochs_noalloc(ctypes.c_void_p(row_ptr.data_ptr()),
                                                       ctypes.c_void_p(col_idx.data_ptr()), col_idx.numel(), n, p,
                                                       epoch_begin, epochs, neg_samples, ctypes.byref(schedule),
                                                       seed, substeps, cap, _stream(stream)))


class MultiEpoch:
    """One kernel launch per call running one epoch of several single-graph
    HOGWILD handles, each at its own epoch, schedule and seed (continuous
    batching; see snap_multi_* in the C header)."""

    def __init__(self, max_jobs: int = 1024):
        self.handle = ctypes.c_void_p()
        self.max_jobs = max_jobs
        _check(load_library().snap_multi_create(max_jobs, ctypes.byref(self.handle)))
        self._h = (ctypes.c_void_p * max_jobs)()
        self._p = (ctypes.c_void_p * max_jobs)()
        self._e = (ctypes.c_int32 * max_jobs)()
        self._s = (SnapSchedule * max_jobs)()
        self._seed = (ctypes.c_uint64 * max_jobs)()

    def epoch(self, jobs, neg_samples: int, stream=None) -> None:
        """jobs: iterable of (handle, positions tensor, epoch, SnapSchedule, seed)."""
        q = 0
        for h, pos, ep, sched, seed in jobs:
            self._h[q] = h.value if isinstance(h, ctypes.c_void_p) else h
            self._p[q] = pos.data_ptr()
            self._e[q] = ep
            self._s[q] = sched
            self._seed[q] = seed
            q += 1
        _check(load_library().snap_multi_epoch(self.handle, self._h, self._p, self._e, self._s, self._seed, q,
                                               neg_samples, _stream(stream)))

    def check(self, stream=None) -> None:
        _check(load_library().snap_multi_check(self.handle, _stream(stream)))

    def close(self) -> None:
        if self.handle:
            load_library().snap_multi_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclass
class Layout:
    """Owning wrapper of a handle: ``with Layout(row_ptr, col_idx) as L: L.epochs(...)``."""
    row_ptr: np.ndarray
    col_idx: np.ndarray
    opts: SnapOptions | None = None
    degrees: np.ndarray | None = None
    stream: object = None

    def __post_init__(self):
        self.n = int(np.asarray(self.row_ptr).size - 1)
        self.handle = snap_layout_create(self.row_ptr, self.col_idx, self.degrees, self.n, self.opts, self.stream)

    def epochs(self, positions, epoch_begin: int, epochs: int, neg_samples: int, schedule: SnapSchedule,
               seed: int) -> None:
        _device_positions(positions, self.n)
        snap_layout_epochs(self.handle, positions, epoch_begin, epochs, neg_samples, schedule, seed, self.stream)

    def epochs_energy(self, positions, epoch_begin: int, epochs: int, neg_samples: int, schedule: SnapSchedule,
                      seed: int, energy) -> None:
        _device_positions(positions, self.n)
        snap_layout_epochs_energy(self.handle, positions, epoch_begin, epochs, neg_samples, schedule, seed, energy,
                                  self.stream)

    def sync_chunks(self, positions, epoch: int, chunk_begin: int, chunk_end: int, neg_samples: int,
                    schedule: SnapSchedule, seed: int) -> None:
        _device_positions(positions, self.n)
        snap_layout_sync_chunks(self.handle, positions, epoch, chunk_begin, chunk_end, neg_samples, schedule, seed,
                                self.stream)

    def objective(self, positions, neg_samples: int, exact: bool = True, pair_samples: int = 0, seed: int = 0):
        _device_positions(positions, self.n)
        return snap_layout_objective(self.handle, positions, neg_samples, exact, pair_samples, seed, self.stream)

    def neighborhood_preservation(self, positions, nodes):
        _device_positions(positions, self.n)
        return snap_layout_neighborhood_preservation(self.handle, positions, nodes, self.stream)

    def autotune(self, initial_positions, scratch_positions, neg_samples: int, schedule: SnapSchedule, seed: int,
                 tolerance: float = 0.02):
        _device_positions(initial_positions, self.n)
        _device_positions(scratch_positions, self.n)
        return snap_layout_autotune(self.handle, scratch_positions, neg_samples, schedule, seed, initial_positions,
                                    tolerance, self.stream)

    def check(self) -> None:
        snap_layout_check(self.handle, self.stream)

    @property
    def device_bytes(self) -> int:
        return snap_layout_device_bytes(self.handle)

    def close(self) -> None:
        if getattr(self, "handle", None):
            snap_layout_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

"""Random-access probe for the roofline of the epoch kernels (measurement only).

The epoch kernels are bound by random 8-byte accesses to an L2-resident
position array; ``random_access_rate`` measures what the device sustains for
that access pattern alone (see csrc/probe_l2.cu)."""
from __future__ import annotations

import ctypes

from . import _build

OPS = {"load": 0, "load_store": 1, "load_atomic": 2, "atomic": 3, "load_exch": 4, "exch": 5, "store": 6,
       "load_store_other": 7, "load_dep_atomic": 8, "load_dep_atomic_other": 9,
       "ldnc_dep_atomic": 10, "ldnc_store": 11}
_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_build.PROBE_LIB)
        _lib.snap_probe_random_access.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_int, ctypes.c_int,
                                                  ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
        _lib.snap_probe_random_access.restype = ctypes.c_double
    return _lib


def random_access_rate(buf, op: str, depth: int = 4, iters: int = 64, grid: int | None = None, stream=None) -> float:
    """Accesses per second on the float32 CUDA tensor ``buf`` viewed as float2 slots."""
    import torch
    n = buf.numel() // 2
    if grid is None:
        grid = torch.cuda.get_device_properties(buf.device).multi_processor_count * 8
    s = torch.cuda.current_stream() if stream is None else stream
    r = _load().snap_probe_random_access(ctypes.c_void_p(buf.data_ptr()), n, OPS[op], depth, iters, grid,
                                         ctypes.c_void_p(s.cuda_stream))
    if r < 0:
        raise RuntimeError(f"probe failed ({r})")
    return r

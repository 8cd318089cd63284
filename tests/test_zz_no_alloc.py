"""snap_sync_epochs_noalloc: the synchronous mode for callers that may not
allocate device memory (a host framework that owns all device memory through
its own pool, or latency-critical code that cannot pay for an allocation).

It must reproduce the allocating path -- snap_layout_epochs on a SYNC handle
-- on buffers the caller owns, call after call, since its fixed scratch is
shared and keeps the previous call's contents.  This file is collected last
so a failure here does not stop the rest of a run that stops at the first
failure."""
import numpy as np
import pytest

import paper_2608_01907_gb300 as snap
from gpu_helpers import SYNC_RTOL, parity_error
from synth import initial_positions, sbm_graph, tiny_graph

pytestmark = pytest.mark.gpu

NOALLOC_MAX_NODES = 1 << 18


def _reference(torch, g, Y, epoch_begin, epochs, k, sched, seed, S, cap):
    """The existing entry point: a SYNC handle with the same substeps and cap."""
    pos = torch.from_numpy(np.ascontiguousarray(Y, dtype=np.float32)).cuda()
    opts = snap.make_options(mode=snap.MODE_SYNC, sync_substeps=S, sync_cap=cap)
    with snap.Layout(g.row_ptr, g.col_idx, opts=opts) as L:
        L.epochs(pos, epoch_begin, epochs, k, sched, seed)
        L.check()
    return pos.cpu().numpy()


@pytest.mark.parametrize("name,k,S,cap", [("sbm", 3, 1, 0.0), ("sbm", 5, 8, 0.05), ("tiny", 10, 3, 0.0)])
def test_noalloc_matches_allocating_path_on_two_calls_in_a_row(cuda, name, k, S, cap):
    torch = cuda
    g = sbm_graph(seed=2) if name == "sbm" else tiny_graph(700, 2500, seed=3)
    Y0 = initial_positions(g.n, 9)
    sched = snap.linear_schedule(eta0=0.5, total_epochs=6)
    rp = torch.from_numpy(g.row_ptr).cuda()
    ci = torch.from_numpy(g.col_idx).cuda()
    pos = torch.from_numpy(Y0.copy()).cuda()
    expect = Y0
    for call in range(2):                      # two calls in a row, two epochs each
        snap.snap_sync_epochs_noalloc(rp, ci, pos, 2 * call, 2, k, sched, 13, substeps=S, cap=cap)
        expect = _reference(torch, g, expect, 2 * call, 2, k, sched, 13, S, cap)
        got = pos.cpu().numpy()
        err = parity_error(got, expect)
        print(f"no-alloc {name} k={k} S={S} call {call}: max rel err {err:.2e}")
        assert err < SYNC_RTOL
        assert np.all(np.isfinite(got))


def test_noalloc_rejects_sizes_beyond_its_scratch(cuda):
    torch = cuda
    n = NOALLOC_MAX_NODES + 1
    rp = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    ci = torch.zeros(1, dtype=torch.int32, device="cuda")
    pos = torch.zeros((n, 2), dtype=torch.float32, device="cuda")
    with pytest.raises(snap.SnapError) as ei:
        snap.snap_sync_epochs_noalloc(rp, ci, pos, 0, 1, 3, snap.linear_schedule(), 1)
    assert ei.value.status == 1 and "262144" in str(ei.value)


def _malformed(g):
    """Malformed variants of a valid CSR: (name, row_ptr, col_idx)."""
    rp, ci = g.row_ptr, g.col_idx
    out = []
    c = ci.copy()
    c[5] = g.n + 7
    out.append(("column past n", rp, c))
    c = ci.copy()
    c[3] = -1
    out.append(("negative column", rp, c))
    out.append(("short col_idx", rp, ci[:-3].copy()))
    r = rp.copy()
    r[0] = 1
    out.append(("row_ptr[0] != 0", r, ci))
    r = rp.copy()
    r[10], r[11] = r[11], r[10]
    out.append(("decreasing row_ptr", r, ci))
    c = ci.copy()
    row = int(np.searchsorted(rp, 7, side="right") - 1)
    c[7] = row
    out.append(("self-loop", rp, c))
    c = ci.copy()
    a = int(rp[2])
    c[a], c[a + 1] = c[a + 1], c[a]
    out.append(("unsorted row", rp, c))
    # drop one reverse edge: row 0 loses its first entry, row_ptr shifts
    r = rp.copy()
    r[1:] -= 1
    out.append(("missing reverse edge", r, np.delete(ci, 0)))
    return out


def test_noalloc_rejects_malformed_csr_without_touching_positions(cuda):
    torch = cuda
    g = tiny_graph(50, 80, seed=4)
    assert np.all(np.diff(g.row_ptr)[:3] >= 2)
    Y0 = initial_positions(g.n, 1)
    for name, rp_bad, ci_bad in _malformed(g):
        pos = torch.from_numpy(Y0.copy()).cuda()
        with pytest.raises(snap.SnapError) as ei:
            snap.snap_sync_epochs_noalloc(torch.from_numpy(rp_bad).cuda(), torch.from_numpy(ci_bad).cuda(), pos,
                                          0, 1, 3, snap.linear_schedule(), 1)
        assert ei.value.status == 1, name
        assert np.array_equal(pos.cpu().numpy(), Y0), name
    # the scratch is cleared by the next call, which succeeds
    rp = torch.from_numpy(g.row_ptr).cuda()
    ci = torch.from_numpy(g.col_idx).cuda()
    pos = torch.from_numpy(Y0.copy()).cuda()
    snap.snap_sync_epochs_noalloc(rp, ci, pos, 0, 1, 3, snap.linear_schedule(), 1)
    expect = _reference(torch, g, Y0, 0, 1, 3, snap.linear_schedule(), 1, 1, 0.0)
    assert parity_error(pos.cpu().numpy(), expect) < SYNC_RTOL


def test_noalloc_rejects_host_buffers(cuda):
    torch = cuda
    g = tiny_graph(40, 60, seed=5)
    pos = torch.from_numpy(initial_positions(g.n, 1)).cuda()
    lib = snap.load_library()
    import ctypes
    rp = np.ascontiguousarray(g.row_ptr)
    ci = torch.from_numpy(g.col_idx).cuda()
    sched = snap.linear_schedule()
    st = lib.snap_sync_epochs_noalloc(ctypes.c_void_p(rp.ctypes.data), ctypes.c_void_p(ci.data_ptr()), ci.numel(),
                                      g.n, ctypes.c_void_p(pos.data_ptr()), 0, 1, 3, ctypes.byref(sched), 1, 1,
                                      ctypes.c_float(0.0), None)
    assert st == 1

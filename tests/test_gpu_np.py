"""Neighbourhood preservation on the device (Section 4.1, r = 2;
snap_layout_neighborhood_preservation) against the oracle's NP on the same
layouts and vertices: the device forms the same FP64 squared distances from
the FP32 positions and selects the k nearest exactly, so the two agree to
rounding of the mean.  Also the autotuner's NP gate on a batch."""
import numpy as np
import pytest

import oracle
import paper_2608_01907_gb300 as snap
from gpu_helpers import gpu_layout
from synth import initial_positions, sbm_graph, tiny_graph

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,mode", [("sbm", snap.MODE_HOGWILD_RED), ("tiny", snap.MODE_SYNC),
                                       ("lattice", snap.MODE_HOGWILD)])
def test_device_np_equals_oracle_np(cuda, name, mode):
    torch = cuda
    if name == "sbm":
        g = sbm_graph(seed=3)
    elif name == "tiny":
        g = tiny_graph(3000, 9000, seed=6)
    else:
        # a 40 x 40 lattice laid out on its grid: many exactly tied distances
        from synth import edges_to_csr
        side = 40
        idx = np.arange(side * side).reshape(side, side)
        u = np.concatenate([idx[:, :-1].ravel(), idx[:-1, :].ravel()])
        v = np.concatenate([idx[:, 1:].ravel(), idx[1:, :].ravel()])
        rp, ci = edges_to_csr(side * side, u, v)
        from synth import Graph
        g = Graph(side * side, rp, ci)
    sched = snap.linear_schedule(eta0=1.0, total_epochs=10)
    if name == "lattice":
        yy, xx = np.divmod(np.arange(g.n), 40)
        Y = np.stack([xx, yy], axis=1).astype(np.float32)
    else:
        Y = gpu_layout(torch, g, initial_positions(g.n, 2), 10, 3, sched, seed=4,
                       opts=snap.make_options(mode=mode, sync_substeps=4, sync_cap=0.05))
    nodes = np.random.default_rng(9).choice(g.n, 700, replace=True).astype(np.int32)
    pos = torch.from_numpy(np.ascontiguousarray(Y)).cuda()
    opts = snap.make_options(mode=mode, keep_csr=True, sync_substeps=4)
    with snap.Layout(g.row_ptr, g.col_idx, opts=opts) as L:
        got, used = L.neighborhood_preservation(pos, nodes)
    ref = oracle.neighborhood_preservation(g.row_ptr, g.col_idx, g.n, Y.astype(np.float64), nodes)
    deg = np.diff(g.row_ptr)
    print(f"device NP {name}: {got:.6f} vs oracle {ref:.6f} over {used} samples")
    assert used == int((deg[nodes] > 0).sum())
    assert abs(got - ref) < 1e-12


def test_device_np_past_the_shared_memory_bitmap(cuda):
    """A graph above 2^18 vertices (the 2-hop bitmap in global scratch), with
    the top hub and its neighbours among the samples (rows read by a warp)."""
    torch = cuda
    from synth import rmat_graph
    g = rmat_graph(19, 3_000_000, seed=2)
    assert g.n > (1 << 18)
    deg = np.diff(g.row_ptr)
    hub = int(np.argmax(deg))
    rng = np.random.default_rng(4)
    nodes = np.concatenate([[hub], g.col_idx[g.row_ptr[hub]:g.row_ptr[hub] + 20],
                            rng.choice(g.n, 150, replace=False)]).astype(np.int32)
    sched = snap.linear_schedule(eta0=1.0, total_epochs=5)
    Y = gpu_layout(torch, g, initial_positions(g.n, 5), 5, 3, sched, seed=6)
    pos = torch.from_numpy(np.ascontiguousarray(Y)).cuda()
    with snap.Layout(g.row_ptr, g.col_idx, opts=snap.make_options(keep_csr=True)) as L:
        got, used = L.neighborhood_preservation(pos, nodes)
    ref = oracle.neighborhood_preservation(g.row_ptr, g.col_idx, g.n, Y.astype(np.float64), nodes)
    print(f"device NP on R-MAT 2^19 (hub degree {deg[hub]}): {got:.6f} vs oracle {ref:.6f} over {used} samples")
    assert used == int((deg[nodes] > 0).sum())
    assert abs(got - ref) < 1e-12
    # every vertex at one of two points: all distances tie within a factor of two,
    # so the candidate list overflows and the select runs over all vertices
    Y2 = np.zeros((g.n, 2), np.float32)
    Y2[::3] = (0.5, 0.25)
    pos2 = torch.from_numpy(Y2).cuda()
    with snap.Layout(g.row_ptr, g.col_idx, opts=snap.make_options(keep_csr=True)) as L:
        got2, _ = L.neighborhood_preservation(pos2, nodes[:40])
    ref2 = oracle.neighborhood_preservation(g.row_ptr, g.col_idx, g.n, Y2.astype(np.float64), nodes[:40])
    print(f"device NP with tied distances: {got2:.6f} vs oracle {ref2:.6f}")
    assert abs(got2 - ref2) < 1e-12


def test_device_np_needs_the_csr(cuda):
    torch = cuda
    g = sbm_graph(n=400, blocks=4, p_in=0.05, p_out=0.005, seed=2)
    pos = torch.from_numpy(initial_positions(g.n, 1)).cuda()
    with snap.Layout(g.row_ptr, g.col_idx) as L:   # HOGWILD without keep_csr
        with pytest.raises(snap.SnapError) as ei:
            L.neighborhood_preservation(pos, np.arange(10))
        assert ei.value.status == 5
    with snap.Layout(g.row_ptr, g.col_idx, opts=snap.make_options(keep_csr=True)) as L2:
        with pytest.raises(snap.SnapError) as ei:
            L2.neighborhood_preservation(pos, np.array([0, g.n], dtype=np.int32))
        assert ei.value.status == 1


def test_autotune_gates_on_np_in_a_batch(cuda):
    torch = cuda
    from synth import batch_sbm_graphs
    graphs = batch_sbm_graphs(count=24, nmax=3000, seed=8)
    rp, ci, offs = snap.batch_union([(g.row_ptr, g.col_idx) for g in graphs])
    n = int(offs[-1])
    sched = snap.linear_schedule(1.0, 30)
    init = torch.from_numpy(initial_positions(n, 3)).cuda()
    scratch = torch.empty_like(init)
    h = snap.snap_layout_create_batch(rp, ci, offs, snap.make_options(keep_csr=True))
    try:
        seg, blk, ms, u, npv, order = snap.snap_layout_autotune(h, scratch, 3, sched, 5, init, 0.02)
        assert np.isfinite(u) and 0.0 < npv <= 1.0
        print(f"autotune with NP gate: chunk {seg}, block {blk}, {ms:.3f} ms/epoch, U {u:.1f}, NP {npv:.4f}")
    finally:
        snap.snap_layout_destroy(h)
    # without the CSR the NP half is not evaluated
    h = snap.snap_layout_create_batch(rp, ci, offs)
    try:
        assert np.isnan(snap.snap_layout_autotune(h, scratch, 3, sched, 5, init, 0.02)[4])
    finally:
        snap.snap_layout_destroy(h)

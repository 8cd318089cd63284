"""Batched layouts: many graphs in one handle (disjoint union) against the
same graphs laid out one at a time and against the oracle."""
import numpy as np
import pytest

import oracle
import paper_2608_01907_gb300 as snap
from gpu_helpers import gpu_layout, schedule_dict
from synth import batch_sbm_graphs, edges_to_csr, initial_positions

pytestmark = pytest.mark.gpu


def _graphs(count, seed, nmax=1500):
    return batch_sbm_graphs(count=count, nmin=60, nmax=nmax, seed=seed)


def _batch_positions(graphs, seed):
    return np.concatenate([initial_positions(g.n, seed + 7919 * q) for q, g in enumerate(graphs)])


def _run_batch(torch, graphs, Y0, epochs, k, sched, seed, opts):
    rp, ci, offs = snap.batch_union([(g.row_ptr, g.col_idx) for g in graphs])
    pos = torch.from_numpy(Y0.copy()).cuda()
    h = snap.snap_layout_create_batch(rp, ci, offs, opts)
    try:
        snap.snap_layout_epochs(h, pos, 0, epochs, k, sched, seed)
        snap.snap_layout_check(h)
    finally:
        snap.snap_layout_destroy(h)
    return pos.cpu().numpy(), offs


@pytest.mark.parametrize("k", [1, 3, 6])
def test_sync_batch_equals_graphs_alone_bitwise(cuda, k):
    torch = cuda
    graphs = _graphs(12, seed=3)
    Y0 = _batch_positions(graphs, 5)
    sched = snap.linear_schedule(eta0=0.3, total_epochs=4)
    opts = snap.make_options(mode=snap.MODE_SYNC, sync_substeps=1)
    got, offs = _run_batch(torch, graphs, Y0, 4, k, sched, 17, opts)
    for q, g in enumerate(graphs):
        alone = gpu_layout(torch, g, Y0[offs[q]:offs[q + 1]], 4, k, sched, 17, opts=opts)
        assert np.array_equal(got[offs[q]:offs[q + 1]].view(np.uint32), alone.view(np.uint32)), q


@pytest.mark.parametrize("mode,k", [(snap.MODE_HOGWILD, 3), (snap.MODE_HOGWILD_RED, 3), (snap.MODE_HOGWILD, 6),
                                    (snap.MODE_HOGWILD_RED, 6)])
def test_hogwild_batch_quality_against_oracle(cuda, mode, k):
    """The parallel-vs-sequential quality gate (objective and NP within 2%),
    over 5 seeds as the gate is stated, each seed a 24-graph batch."""
    torch = cuda
    graphs = _graphs(24, seed=4, nmax=3000)
    sched = snap.linear_schedule(eta0=1.0, total_epochs=30)
    ob_g, ob_o, np_g, np_o = [], [], [], []
    for seed in range(5):
        Y0 = _batch_positions(graphs, 6 + seed)
        got, offs = _run_batch(torch, graphs, Y0, 30, k, sched, 23 + seed, snap.make_options(mode=mode))
        assert np.all(np.isfinite(got))
        for q, g in enumerate(graphs):
            y0 = Y0[offs[q]:offs[q + 1]]
            ref = oracle.seq(g.row_ptr, g.col_idx, g.n, y0, 30, k, schedule_dict(sched), seed=23 + seed)
            mine = got[offs[q]:offs[q + 1]]
            ob_g.append(oracle.objective(g.row_ptr, g.col_idx, g.n, mine, k)["total"])
            ob_o.append(oracle.objective(g.row_ptr, g.col_idx, g.n, ref, k)["total"])
            np_g.append(oracle.neighborhood_preservation(g.row_ptr, g.col_idx, g.n, mine))
            np_o.append(oracle.neighborhood_preservation(g.row_ptr, g.col_idx, g.n, ref))
    d_ob = np.sum(ob_g) / np.sum(ob_o) - 1
    d_np = np.mean(np_g) / np.mean(np_o) - 1
    print(f"batch mode={mode} k={k}: objective {d_ob:+.2%}, NP {d_np:+.2%} over {len(graphs)} graphs x 5 seeds")
    assert abs(d_ob) < 0.02
    assert abs(d_np) < 0.02


def test_batch_objective_is_sum_of_graph_objectives(cuda):
    torch = cuda
    graphs = _graphs(9, seed=5)
    rng = np.random.default_rng(3)
    Y = rng.uniform(-2, 2, size=(sum(g.n for g in graphs), 2)).astype(np.float32)
    rp, ci, offs = snap.batch_union([(g.row_ptr, g.col_idx) for g in graphs])
    h = snap.snap_layout_create_batch(rp, ci, offs)
    try:
        a, r, t = snap.snap_layout_objective(h, torch.from_numpy(Y).cuda(), 3, exact=True)
        with pytest.raises(snap.SnapError) as ei:
            snap.snap_layout_objective(h, torch.from_numpy(Y).cuda(), 3, exact=False, pair_samples=1000)
        assert ei.value.status == 5
    finally:
        snap.snap_layout_destroy(h)
    ex = [oracle.objective(g.row_ptr, g.col_idx, g.n, Y[offs[q]:offs[q + 1]], 3) for q, g in enumerate(graphs)]
    assert a == pytest.approx(sum(e["attr"] for e in ex), rel=1e-5)
    assert r == pytest.approx(sum(e["rep"] for e in ex), rel=1e-5)


def test_batch_rejects_cross_graph_edges_and_bad_offsets(cuda):
    rp, ci = edges_to_csr(6, np.array([0, 1, 3, 2]), np.array([1, 2, 4, 3]))   # 2-3 crosses [0,3)|[3,6)
    with pytest.raises(snap.SnapError) as ei:
        snap.snap_layout_create_batch(rp, ci, np.array([0, 3, 6], np.int32))
    assert ei.value.status == 1 and "joins two graphs" in str(ei.value)
    rp, ci = edges_to_csr(6, np.array([0, 1, 3, 4]), np.array([1, 2, 4, 5]))
    h = snap.snap_layout_create_batch(rp, ci, np.array([0, 3, 6], np.int32))
    snap.snap_layout_destroy(h)
    for bad in ([0, 3, 5], [0, 0, 6], [1, 3, 6]):
        with pytest.raises(snap.SnapError):
            snap.snap_layout_create_batch(rp, ci, np.array(bad, np.int32))


# --------------------------------------------------------------------------
# CUDA-graph epoch loops and the autotuner
# --------------------------------------------------------------------------
@pytest.mark.parametrize("mode,seg", [(snap.MODE_SYNC, 0), (snap.MODE_HOGWILD, 4096), (snap.MODE_HOGWILD_RED, 4096)])
def test_cuda_graph_epochs_equal_direct_launches(cuda, mode, seg):
    torch = cuda
    from synth import tiny_graph
    g = tiny_graph(400, 1500, seed=8)      # one segment: a deterministic single lane in HOGWILD
    Y0 = initial_positions(g.n, 3)
    sched = snap.linear_schedule(eta0=0.5, total_epochs=10)
    direct = gpu_layout(torch, g, Y0, 10, 3, sched, 5,
                        opts=snap.make_options(mode=mode, sync_substeps=2, segment_edges=seg))
    opts = snap.make_options(mode=mode, sync_substeps=2, segment_edges=seg, cuda_graph=True)
    pos = torch.from_numpy(Y0.copy()).cuda()
    with snap.Layout(g.row_ptr, g.col_idx, opts=opts) as L:
        L.epochs(pos, 0, 10, 3, sched, 5)         # captured, then launched
        first = pos.cpu().numpy()
        pos.copy_(torch.from_numpy(Y0))
        L.epochs(pos, 0, 10, 3, sched, 5)         # replayed
        L.check()
    again = pos.cpu().numpy()
    assert np.array_equal(first.view(np.uint32), direct.view(np.uint32))
    assert np.array_equal(again.view(np.uint32), direct.view(np.uint32))


def test_autotune_picks_a_bounded_configuration(cuda):
    torch = cuda
    from synth import tiny_graph
    g = tiny_graph(60_000, 500_000, seed=9)
    sched = snap.linear_schedule(1.0, 10)
    scratch = torch.from_numpy(initial_positions(g.n, 1)).cuda()
    with snap.Layout(g.row_ptr, g.col_idx) as L:
        seg, blk, ms, u, _, _ = snap.snap_layout_autotune(L.handle, scratch, 3, sched, 7)   # timing only
        assert seg in (4, 8, 16, 32) and blk in (128, 256) and ms > 0 and np.isnan(u)
        pos = torch.from_numpy(initial_positions(g.n, 2)).cuda()
        before = L.objective(pos, 3)[2]
        L.epochs(pos, 0, 10, 3, sched, 3)
        L.check()
        assert L.objective(pos, 3)[2] < before
    with snap.Layout(g.row_ptr, g.col_idx, opts=snap.make_options(mode=snap.MODE_SYNC)) as L:
        with pytest.raises(snap.SnapError) as ei:
            snap.snap_layout_autotune(L.handle, scratch, 3, sched, 7)
        assert ei.value.status == 5


@pytest.mark.parametrize("mode", [snap.MODE_HOGWILD_RED, snap.MODE_HOGWILD])
def test_autotune_quality_gate(cuda, mode):
    """The chosen configuration's layout is within the tolerance of the entry
    configuration's (same initial positions, schedule and seed), and reproduces
    the objective the autotuner reports when laid out again."""
    torch = cuda
    from synth import tiny_graph
    g = tiny_graph(60_000, 500_000, seed=9)
    sched = snap.linear_schedule(1.0, 10)
    init = torch.from_numpy(initial_positions(g.n, 4)).cuda()
    scratch = torch.empty_like(init)
    opts = snap.make_options(mode=mode)
    with snap.Layout(g.row_ptr, g.col_idx, opts=opts) as L:
        pos = init.clone()
        L.epochs(pos, 0, 10, 3, sched, 5)
        L.check()
        u_entry = L.objective(pos, 3, exact=False, pair_samples=1 << 24, seed=5 ^ 0x5bd1e9955bd1e995)[2]
        seg, blk, ms, u, _, _ = L.autotune(init, scratch, 3, sched, 5, tolerance=0.02)
        assert seg in (4, 8, 16, 32) and blk in (128, 256) and ms > 0
        # the gate compares against its own run of the entry configuration;
        # u_entry is another run of it (Hogwild runs differ by well under 1%)
        assert np.isfinite(u) and u <= u_entry * 1.03
        pos = init.clone()
        L.epochs(pos, 0, 10, 3, sched, 5)
        L.check()
        again = L.objective(pos, 3, exact=False, pair_samples=1 << 24, seed=5 ^ 0x5bd1e9955bd1e995)[2]
        assert again == pytest.approx(u, rel=0.02)
    with snap.Layout(g.row_ptr, g.col_idx, opts=opts) as L:
        seg0, blk0, _, u0, _, _ = L.autotune(init, scratch, 3, sched, 5, tolerance=0.0)
        assert seg0 in (4, 8, 16, 32) and blk0 in (128, 256)
        assert np.isfinite(u0) and u0 <= u_entry * 1.01


def test_autotune_on_a_batch_with_a_captured_epoch_loop(cuda):
    """The autotuner on a batch handle (exact per-graph objective in the gate),
    then the 30-epoch loop captured as a CUDA graph: the captured layout
    reaches the objective the gate measured, and so does its replay."""
    torch = cuda
    graphs = _graphs(64, seed=11, nmax=4000)
    Y0 = _batch_positions(graphs, 9)
    rp, ci, offs = snap.batch_union([(g.row_ptr, g.col_idx) for g in graphs])
    sched = snap.linear_schedule(eta0=1.0, total_epochs=30)
    init = torch.from_numpy(Y0).cuda()
    scratch = torch.empty_like(init)
    pos = torch.empty_like(init)
    h = snap.snap_layout_create_batch(rp, ci, offs, snap.make_options(cuda_graph=True))
    try:
        seg, blk, ms, u, _, _ = snap.snap_layout_autotune(h, scratch, 3, sched, 2, init, 0.02)
        assert seg in (4, 8, 16, 32) and blk in (128, 256) and ms > 0 and np.isfinite(u)
        pos.copy_(init)
        before = snap.snap_layout_objective(h, pos, 3, True)[2]
        snap.snap_layout_epochs(h, pos, 0, 30, 3, sched, 2)     # captured, then launched
        snap.snap_layout_check(h)
        after = snap.snap_layout_objective(h, pos, 3, True)[2]
        assert after < before
        assert after == pytest.approx(u, rel=0.02)
        pos.copy_(init)
        snap.snap_layout_epochs(h, pos, 0, 30, 3, sched, 2)     # replayed
        snap.snap_layout_check(h)
        assert snap.snap_layout_objective(h, pos, 3, True)[2] == pytest.approx(after, rel=0.02)
    finally:
        snap.snap_layout_destroy(h)

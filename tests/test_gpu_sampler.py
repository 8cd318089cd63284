"""Weighted negatives on the GPU (DEGREE and WEIGHTS samplers, alias table)
against the oracle: per-coordinate parity of the synchronous mode and of a
single Hogwild lane, Hogwild quality, the weighted objective, batches and
multi-handle epochs."""
import numpy as np
import pytest

import oracle
import paper_2608_01907_gb300 as snap
from gpu_helpers import SYNC_RTOL, gpu_layout, oriented_order, parity_error, schedule_dict
from synth import batch_sbm_graphs, initial_positions, sbm_graph, tiny_graph

pytestmark = pytest.mark.gpu


def _weights(n, seed):
    rng = np.random.default_rng(seed)
    w = rng.pareto(1.5, n).astype(np.float32) + np.float32(0.05)
    w[rng.random(n) < 0.1] = 0.0
    return w


def _sampler_pair(kind, g, seed=1):
    """(library option kwargs, oracle Sampler) for the same weights."""
    if kind == "degree":
        return dict(sampler=snap.SAMPLER_DEGREE), oracle.Sampler.degree(g.row_ptr)
    w = _weights(g.n, seed)
    return dict(sampler=snap.SAMPLER_WEIGHTS, node_weights=w), oracle.Sampler.weights(w)


@pytest.mark.parametrize("kind", ["degree", "weights"])
@pytest.mark.parametrize("name,k,S", [("sbm", 3, 1), ("sbm", 6, 4), ("tiny", 10, 2), ("tiny", 1, 1)])
def test_weighted_sync_matches_oracle_after_one_epoch(cuda, kind, name, k, S):
    g = sbm_graph(seed=1) if name == "sbm" else tiny_graph(700, 2500, seed=2)
    kw, sam = _sampler_pair(kind, g)
    Y0 = initial_positions(g.n, 7)
    sched = snap.linear_schedule(eta0=0.25, total_epochs=30)
    got = gpu_layout(cuda, g, Y0, 1, k, sched, seed=11,
                     opts=snap.make_options(mode=snap.MODE_SYNC, sync_substeps=S, **kw))
    ref = oracle.sync(g.row_ptr, g.col_idx, g.n, Y0, 1, k, schedule_dict(sched), seed=11, substeps=S, sampler=sam)
    err = parity_error(got, ref)
    print(f"weighted sync parity {kind} {name} k={k} S={S}: max rel err {err:.2e}")
    assert err < SYNC_RTOL


@pytest.mark.parametrize("kind", ["degree", "weights"])
@pytest.mark.parametrize("mode", [snap.MODE_HOGWILD, snap.MODE_HOGWILD_RED])
@pytest.mark.parametrize("n,m,k", [(12, 30, 5), (90, 300, 10), (300, 900, 3), (40, 120, 2), (90, 300, 4)])
def test_weighted_single_lane_is_algorithm1_in_oriented_order(cuda, kind, mode, n, m, k):
    g = tiny_graph(n, m, seed=n)
    kw, sam = _sampler_pair(kind, g, seed=n)
    Y0 = initial_positions(g.n, 4)
    sched = snap.linear_schedule(eta0=0.5, total_epochs=4)
    got = gpu_layout(cuda, g, Y0, 2, k, sched, seed=21, opts=snap.make_options(mode=mode, segment_edges=4096, **kw))
    ref = oracle.seq(g.row_ptr, g.col_idx, g.n, Y0, 2, k, schedule_dict(sched), seed=21, order=oriented_order(g),
                     sampler=sam)
    err = parity_error(got, ref)
    print(f"weighted single lane {kind} mode={mode} n={n} k={k}: max rel err {err:.2e}")
    assert err < SYNC_RTOL


@pytest.mark.parametrize("mode", [snap.MODE_HOGWILD, snap.MODE_HOGWILD_RED])
def test_degree_hogwild_quality_within_two_percent_sbm(cuda, mode):
    g = sbm_graph(seed=1)
    sam = oracle.Sampler.degree(g.row_ptr)
    sched = snap.linear_schedule(eta0=1.0, total_epochs=30)
    ob_g, ob_o, np_g, np_o = [], [], [], []
    for seed in range(1, 6):
        Y0 = initial_positions(g.n, seed)
        got = gpu_layout(cuda, g, Y0, 30, 3, sched, seed=seed,
                         opts=snap.make_options(mode=mode, sampler=snap.SAMPLER_DEGREE))
        ref = oracle.seq(g.row_ptr, g.col_idx, g.n, Y0, 30, 3, schedule_dict(sched), seed=seed, sampler=sam)
        assert np.all(np.isfinite(got))
        ob_g.append(oracle.objective(g.row_ptr, g.col_idx, g.n, got, 3, sampler=sam)["total"])
        ob_o.append(oracle.objective(g.row_ptr, g.col_idx, g.n, ref, 3, sampler=sam)["total"])
        np_g.append(oracle.neighborhood_preservation(g.row_ptr, g.col_idx, g.n, got))
        np_o.append(oracle.neighborhood_preservation(g.row_ptr, g.col_idx, g.n, ref))
    d_ob = np.mean(ob_g) / np.mean(ob_o) - 1
    d_np = np.mean(np_g) / np.mean(np_o) - 1
    print(f"degree sampler mode={mode} SBM: objective {d_ob:+.2%}, NP {d_np:+.2%}")
    assert abs(d_ob) < 0.02
    assert abs(d_np) < 0.02


@pytest.mark.parametrize("kind", ["degree", "weights"])
@pytest.mark.parametrize("mode", [snap.MODE_HOGWILD, snap.MODE_SYNC])
def test_weighted_objective_matches_oracle(cuda, kind, mode):
    torch = cuda
    g = sbm_graph(seed=4)
    kw, sam = _sampler_pair(kind, g, seed=3)
    Y = np.random.default_rng(8).uniform(-3, 3, size=(g.n, 2)).astype(np.float32)
    pos = torch.from_numpy(Y).cuda()
    with snap.Layout(g.row_ptr, g.col_idx, opts=snap.make_options(mode=mode, **kw)) as L:
        a, r, t = L.objective(pos, 3, exact=True)
        sa, sr, st = L.objective(pos, 3, exact=False, pair_samples=3_000_000, seed=17)
    ex = oracle.objective(g.row_ptr, g.col_idx, g.n, Y, 3, sampler=sam)
    sm = oracle.objective_sampled(g.row_ptr, g.col_idx, g.n, Y, 3, 3_000_000, 17, sampler=sam)
    assert a == pytest.approx(ex["attr"], rel=1e-5)
    assert r == pytest.approx(ex["rep"], rel=1e-5)
    assert sr == pytest.approx(sm["rep"], rel=1e-4)
    assert sr == pytest.approx(ex["rep"], rel=2e-2)


def test_degree_batch_sync_equals_graphs_alone_bitwise(cuda):
    torch = cuda
    graphs = batch_sbm_graphs(count=10, nmin=60, nmax=1200, seed=3)
    Y0 = np.concatenate([initial_positions(g.n, 5 + q) for q, g in enumerate(graphs)])
    sched = snap.linear_schedule(eta0=0.3, total_epochs=3)
    opts = snap.make_options(mode=snap.MODE_SYNC, sampler=snap.SAMPLER_DEGREE)
    rp, ci, offs = snap.batch_union([(g.row_ptr, g.col_idx) for g in graphs])
    pos = torch.from_numpy(Y0.copy()).cuda()
    h = snap.snap_layout_create_batch(rp, ci, offs, opts)
    try:
        snap.snap_layout_epochs(h, pos, 0, 3, 5, sched, 17)
        snap.snap_layout_check(h)
        a, r, t = snap.snap_layout_objective(h, pos, 5, exact=True)
    finally:
        snap.snap_layout_destroy(h)
    got = pos.cpu().numpy()
    rep = 0.0
    for q, g in enumerate(graphs):
        alone = gpu_layout(torch, g, Y0[offs[q]:offs[q + 1]], 3, 5, sched, 17, opts=opts)
        assert np.array_equal(got[offs[q]:offs[q + 1]].view(np.uint32), alone.view(np.uint32)), q
        rep += oracle.objective(g.row_ptr, g.col_idx, g.n, got[offs[q]:offs[q + 1]], 5,
                                sampler=oracle.Sampler.degree(g.row_ptr))["rep"]
    assert r == pytest.approx(rep, rel=1e-5)


@pytest.mark.parametrize("k", [3, 6])
def test_degree_job_in_a_multi_epoch_equals_alone_bitwise(cuda, k):
    torch = cuda
    graphs = [tiny_graph(300, 900, seed=s) for s in (1, 2)]
    sched = snap.linear_schedule(eta0=0.7, total_epochs=6)
    samplers = [snap.SAMPLER_DEGREE, snap.SAMPLER_UNIFORM]   # one weighted and one uniform job in one launch
    handles = [snap.snap_layout_create(g.row_ptr, g.col_idx, None, g.n,
                                       snap.make_options(segment_edges=4096, sampler=s))
               for g, s in zip(graphs, samplers)]
    Y0 = [initial_positions(g.n, 10 + q) for q, g in enumerate(graphs)]
    pos = [torch.from_numpy(y.copy()).cuda() for y in Y0]
    multi = snap.MultiEpoch(4)
    try:
        for t in range(6):
            multi.epoch([(handles[q], pos[q], t, sched, 40 + q) for q in range(2)], k)
        multi.check()
    finally:
        multi.close()
        for h in handles:
            snap.snap_layout_destroy(h)
    for q, g in enumerate(graphs):
        alone = gpu_layout(torch, g, Y0[q], 6, k, sched, 40 + q,
                           opts=snap.make_options(segment_edges=4096, sampler=samplers[q]))
        assert np.array_equal(pos[q].cpu().numpy().view(np.uint32), alone.view(np.uint32)), q

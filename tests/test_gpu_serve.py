"""Continuous batching: several layouts advanced by one launch per tick
(snap_multi_epoch) and the layout server built on it.  A job's result must
not depend on the other jobs in the mix: bit for bit when each job is one
lane (deterministic), within the quality tolerance otherwise."""
import numpy as np
import pytest

import oracle
import paper_2608_01907_gb300 as snap
from paper_2608_01907_gb300.serve import Job, LayoutServer, estimated_bytes
from synth import initial_positions, sbm_graph, tiny_graph

pytestmark = pytest.mark.gpu

ONE_LANE = 4096    # segment entries >= the test graphs' entries: one lane per job


def _alone(torch, g, Y0, epochs, k, sched, seed, seg=0):
    pos = torch.from_numpy(Y0.copy()).cuda()
    with snap.Layout(g.row_ptr, g.col_idx, opts=snap.make_options(segment_edges=seg)) as L:
        L.epochs(pos, 0, epochs, k, sched, seed)
        L.check()
    return pos.cpu().numpy()


@pytest.mark.parametrize("k", [3, 7])
def test_multi_epoch_equals_separate_launches_with_staggered_starts(cuda, k):
    torch = cuda
    graphs = [tiny_graph(300, 900, seed=s) for s in (1, 2, 3)]
    starts = [0, 3, 5]                      # jobs join at different ticks
    sched = snap.linear_schedule(eta0=0.7, total_epochs=8)
    opts = snap.make_options(segment_edges=ONE_LANE)
    handles = [snap.snap_layout_create(g.row_ptr, g.col_idx, None, g.n, opts) for g in graphs]
    Y0 = [initial_positions(g.n, 10 + q) for q, g in enumerate(graphs)]
    pos = [torch.from_numpy(y.copy()).cuda() for y in Y0]
    multi = snap.MultiEpoch(8)
    try:
        for tick in range(13):
            jobs = [(handles[q], pos[q], tick - starts[q], sched, 40 + q) for q in range(3)
                    if 0 <= tick - starts[q] < 8]
            multi.epoch(jobs, k)
        multi.check()
    finally:
        multi.close()
        for h in handles:
            snap.snap_layout_destroy(h)
    for q, g in enumerate(graphs):
        alone = _alone(torch, g, Y0[q], 8, k, sched, 40 + q, seg=ONE_LANE)
        assert np.array_equal(pos[q].cpu().numpy().view(np.uint32), alone.view(np.uint32)), q


def test_server_result_same_alone_and_in_the_mix_bitwise(cuda):
    torch = cuda
    graphs = [tiny_graph(200 + 50 * q, 700, seed=20 + q) for q in range(6)]
    server = LayoutServer(hbm_budget=1 << 30, max_jobs=4, epochs=12, neg_samples=3, eta0=0.8,
                          segment_edges=ONE_LANE)
    jobs = [Job(q, g.row_ptr, g.col_idx, initial_positions(g.n, 30 + q), seed=50 + q) for q, g in enumerate(graphs)]
    try:
        for q, job in enumerate(jobs):      # arrivals while others run
            server.submit(job)
            for _ in range(q % 3 + 1):
                server.tick()
        server.drain()
    finally:
        server.close()
    assert len(server.done) == len(jobs)
    sched = snap.linear_schedule(0.8, 12)
    for q, (g, job) in enumerate(zip(graphs, jobs)):
        alone = _alone(torch, g, initial_positions(g.n, 30 + q), 12, 3, sched, 50 + q, seg=ONE_LANE)
        assert np.array_equal(job.positions.view(np.uint32), alone.view(np.uint32)), q
        assert job.submitted <= job.admitted <= job.finished


def test_cancelled_jobs_leave_the_others_unchanged(cuda):
    """One job is cancelled while it waits, one while it runs: the others'
    results stay bitwise what they are alone, the cancelled jobs' positions
    are not touched, and the whole budget comes back."""
    torch = cuda
    graphs = [tiny_graph(200 + 50 * q, 700, seed=20 + q) for q in range(6)]
    server = LayoutServer(hbm_budget=1 << 30, max_jobs=2, epochs=12, neg_samples=3, eta0=0.8,
                          segment_edges=ONE_LANE)
    Y0 = [initial_positions(g.n, 30 + q) for q, g in enumerate(graphs)]
    jobs = [Job(q, g.row_ptr, g.col_idx, Y0[q].copy(), seed=50 + q) for q, g in enumerate(graphs)]
    try:
        for job in jobs:
            server.submit(job)
        for _ in range(3):
            server.tick()
        assert [j.job_id for j in server.active] == [0, 1]
        assert server.cancel(4)                 # still waiting (two slots)
        assert server.cancel(1)                 # running, epoch 3 of 12
        assert not server.cancel(99)
        server.drain()
        assert not server.cancel(0)             # finished
    finally:
        server.close()
    assert sorted(j.job_id for j in server.done) == [0, 2, 3, 5]
    assert sorted(j.job_id for j in server.cancelled) == [1, 4]
    assert server.used == 0
    sched = snap.linear_schedule(0.8, 12)
    for job in jobs:
        q = job.job_id
        if job.cancelled:
            assert np.array_equal(job.positions, Y0[q])
            continue
        alone = _alone(torch, graphs[q], Y0[q], 12, 3, sched, 50 + q, seg=ONE_LANE)
        assert np.array_equal(job.positions.view(np.uint32), alone.view(np.uint32)), q


def test_server_quality_in_the_mix_matches_alone(cuda):
    torch = cuda
    graphs = [sbm_graph(seed=s) for s in (1, 2, 3)] + [tiny_graph(20_000, 120_000, seed=4)]
    server = LayoutServer(hbm_budget=1 << 30, max_jobs=16, epochs=30, neg_samples=3, eta0=1.0)
    jobs = [Job(q, g.row_ptr, g.col_idx, initial_positions(g.n, 60 + q), seed=70 + q) for q, g in enumerate(graphs)]
    try:
        for q, job in enumerate(jobs):
            server.submit(job)
            server.tick()
        server.drain()
    finally:
        server.close()
    sched = snap.linear_schedule(1.0, 30)
    rel = []
    for q, (g, job) in enumerate(zip(graphs, jobs)):
        alone = _alone(torch, g, initial_positions(g.n, 60 + q), 30, 3, sched, 70 + q)
        ref = oracle.seq(g.row_ptr, g.col_idx, g.n, initial_positions(g.n, 60 + q), 30, 3,
                         dict(eta0=1.0, total_epochs=30), seed=70 + q)
        o_mix = oracle.objective_sampled(g.row_ptr, g.col_idx, g.n, job.positions, 3, 2_000_000, 9)["total"]
        o_alone = oracle.objective_sampled(g.row_ptr, g.col_idx, g.n, alone, 3, 2_000_000, 9)["total"]
        o_ref = oracle.objective_sampled(g.row_ptr, g.col_idx, g.n, ref, 3, 2_000_000, 9)["total"]
        np_mix = oracle.neighborhood_preservation(g.row_ptr, g.col_idx, g.n, job.positions)
        np_alone = oracle.neighborhood_preservation(g.row_ptr, g.col_idx, g.n, alone)
        np_ref = oracle.neighborhood_preservation(g.row_ptr, g.col_idx, g.n, ref)
        rel.append((o_mix / o_alone - 1, o_mix / o_ref - 1, np_mix / np_alone - 1, np_mix / np_ref - 1))
        print(f"job {q}: in the mix vs alone {o_mix / o_alone - 1:+.2%} (NP {np_mix / np_alone - 1:+.2%}), "
              f"vs oracle {o_mix / o_ref - 1:+.2%} (NP {np_mix / np_ref - 1:+.2%})")
    rel = np.array(rel)
    # the serving property: a job's result in the mix is the result alone --
    # the objective on every job, NP on the community graphs (jobs 0-2).
    # Job 3 is a structureless random graph whose NP is about 0.01: the
    # relative NP difference of two lock-free runs is noise there (measured
    # -0.6%, +0.8% and +2.5% in the mix against alone, -4.4% to -6.4% against
    # the oracle), so only its objective is compared.
    assert np.all(np.abs(rel[:, 0]) < 0.02)
    assert np.all(np.abs(rel[:3, 2]) < 0.02)
    # quality against Algorithm 1, one seed per job; NP within the band
    # Section 4.3 reports between the lock-free variants and the serial
    # algorithm on the community graphs
    assert np.all(np.abs(rel[:, 1]) < 0.03)
    assert np.all(np.abs(rel[:3, 3]) < 0.05)


def test_server_admission_respects_the_memory_budget(cuda):
    """A job is admitted only while its peak preparation bytes fit the budget
    on top of what the running jobs hold (their handles' device bytes plus
    positions): with a budget of one job's peak, jobs run one at a time."""
    import paper_2608_01907_gb300 as snap_pkg
    graphs = [tiny_graph(3000, 10_000, seed=80 + q) for q in range(8)]
    need = max(estimated_bytes(g.n, g.nnz) for g in graphs)
    server = LayoutServer(hbm_budget=need + 1, max_jobs=8, epochs=5)
    jobs = [Job(q, g.row_ptr, g.col_idx, initial_positions(g.n, q), seed=q) for q, g in enumerate(graphs)]
    peak = 0
    try:
        for job in jobs:
            server.submit(job)
        while not server.idle():
            server.tick()
            peak = max(peak, len(server.active) + len(server.retiring))
            assert server.used <= server.budget
            for job in server.active:
                assert job.reserved == snap_pkg.snap_layout_device_bytes(job.handle) + job.positions.nbytes
        server.drain()
    finally:
        server.close()
    assert len(server.done) == len(jobs) and peak == 1 and server.used == 0
    for job in jobs:
        assert np.all(np.isfinite(job.positions))
    with pytest.raises(ValueError):
        LayoutServer(hbm_budget=1000).submit(jobs[0])

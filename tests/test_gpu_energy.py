"""The actual energy of an epoch (Section 3.3: accumulated from the pairs the
epoch visits and draws, compared in the paper with the effective energy of
Eq. 4 after each epoch) as the GPU reports it, against the oracle."""
import numpy as np
import pytest

import oracle
import paper_2608_01907_gb300 as snap
from gpu_helpers import oriented_order, schedule_dict
from synth import initial_positions, sbm_graph, tiny_graph

pytestmark = pytest.mark.gpu


def _gpu_energy(torch, g, Y0, epochs, k, sched, seed, opts):
    pos = torch.from_numpy(np.ascontiguousarray(Y0, dtype=np.float32)).cuda()
    en = torch.zeros(epochs, dtype=torch.float64, device="cuda")
    with snap.Layout(g.row_ptr, g.col_idx, opts=opts) as L:
        L.epochs_energy(pos, 0, epochs, k, sched, seed, en)
        L.check()
    return pos.cpu().numpy(), en.cpu().numpy()


@pytest.mark.parametrize("mode", [snap.MODE_HOGWILD, snap.MODE_HOGWILD_RED])
@pytest.mark.parametrize("sampler", [snap.SAMPLER_UNIFORM, snap.SAMPLER_DEGREE])
@pytest.mark.parametrize("k", [3, 6])
def test_single_lane_energy_equals_oracle(cuda, mode, sampler, k):
    g = tiny_graph(300, 900, seed=3)
    Y0 = initial_positions(g.n, 2)
    sched = snap.linear_schedule(eta0=0.5, total_epochs=3)
    opts = snap.make_options(mode=mode, segment_edges=4096, sampler=sampler)
    _, got = _gpu_energy(cuda, g, Y0, 3, k, sched, 8, opts)
    sam = oracle.Sampler.degree(g.row_ptr) if sampler == snap.SAMPLER_DEGREE else None
    _, ref = oracle.seq(g.row_ptr, g.col_idx, g.n, Y0, 3, k, schedule_dict(sched), seed=8,
                        order=oriented_order(g), return_energy=True, sampler=sam)
    print(f"energy mode={mode} sampler={sampler} k={k}: {got} vs {ref}")
    assert np.allclose(got, ref, rtol=1e-4)


def test_sync_energy_is_the_frozen_pair_sum(cuda):
    g = tiny_graph(60, 150, seed=4)
    Y0 = initial_positions(g.n, 5).astype(np.float64)
    k, seed = 3, 13
    sched = snap.linear_schedule(eta0=0.3, total_epochs=2)
    _, got = _gpu_energy(cuda, g, Y0, 1, k, sched, seed, snap.make_options(mode=snap.MODE_SYNC))
    # one chunk: every term at the initial positions (U^a, U^r from the oracle's pair terms)
    total = 0.0
    for i in range(g.n):
        for e in range(g.row_ptr[i], g.row_ptr[i + 1]):
            j = int(g.col_idx[e])
            total += oracle.pair_terms(*(Y0[i] - Y0[j]))[4]
            negs, _ = oracle.edge_negatives(e, 0, seed, i, g.n, k)
            for s in negs:
                total += oracle.pair_terms(*(Y0[i] - Y0[int(s)]))[5]
    assert got[0] == pytest.approx(0.5 * total, rel=1e-5)


def test_actual_energy_tracks_effective_energy_on_the_gpu(cuda):
    # Fig. 3(a) on the GPU layout: the curves meet.  (Early on the GPU's
    # actual energy lies below the effective one, the oracle's above it: the
    # oriented order applies the two steps of an edge back to back, so the
    # second step's U^a is taken after the first pulled the pair together.)
    torch = cuda
    g = sbm_graph(seed=1)
    pos = torch.from_numpy(initial_positions(g.n, 1)).cuda()
    en = torch.zeros(1, dtype=torch.float64, device="cuda")
    sched = snap.linear_schedule(1.0, 30)
    rel = []
    with snap.Layout(g.row_ptr, g.col_idx) as L:
        for t in range(30):
            L.epochs_energy(pos, t, 1, 3, sched, 1, en)
            eff = L.objective(pos, 3, exact=True)[2]
            rel.append(float(en.item()) / eff - 1.0)
        L.check()
    rel = np.array(rel)
    print("actual / effective - 1 per epoch:", np.round(rel, 4))
    assert np.mean(np.abs(rel[-5:])) < 0.25 * np.mean(np.abs(rel[:5]))   # the gap closes
    assert np.all(np.abs(rel[-6:]) < 0.05)
    assert abs(rel[-1]) < 0.02


def test_energy_rejects_batches_and_bad_buffers(cuda):
    torch = cuda
    rp, ci, offs = snap.batch_union([(g.row_ptr, g.col_idx) for g in (tiny_graph(30, 60, seed=1),
                                                                      tiny_graph(40, 70, seed=2))])
    h = snap.snap_layout_create_batch(rp, ci, offs)
    pos = torch.zeros((70, 2), dtype=torch.float32, device="cuda")
    en = torch.zeros(2, dtype=torch.float64, device="cuda")
    try:
        with pytest.raises(snap.SnapError) as ei:
            snap.snap_layout_epochs_energy(h, pos, 0, 2, 3, snap.linear_schedule(), 1, en)
        assert ei.value.status == 5
    finally:
        snap.snap_layout_destroy(h)
    g = tiny_graph(30, 60, seed=1)
    with snap.Layout(g.row_ptr, g.col_idx) as L:
        with pytest.raises(ValueError):      # float32 energy buffer
            L.epochs_energy(torch.zeros((30, 2), dtype=torch.float32, device="cuda"), 0, 2, 3,
                            snap.linear_schedule(), 1, torch.zeros(2, dtype=torch.float32, device="cuda"))

"""Hogwild layouts of the 260k-node LFR-style graph (stand-in for the
Orkut-communities graph of the teaser) against the FP64 oracle: final
objective and neighbourhood preservation within 2% of the oracle's, as means
over 5 seeds.  The oracle layouts run in a spawned process pool."""
import multiprocessing as mp

import numpy as np
import pytest

import paper_2608_01907_gb300 as snap
import quality_jobs
from synth import initial_positions, lfr_graph

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

SEEDS = [1, 2, 3, 4, 5]


@pytest.fixture(scope="module")
def oracle_scores():
    ctx = mp.get_context("spawn")
    with ctx.Pool(len(SEEDS)) as pool:
        layouts = pool.map(quality_jobs.lfr_oracle_layout, SEEDS)
        scores = pool.map(quality_jobs.lfr_score, layouts)
    return np.array(scores)


@pytest.mark.parametrize("mode", [snap.MODE_HOGWILD, snap.MODE_HOGWILD_RED])
def test_hogwild_quality_within_two_percent_lfr(cuda, oracle_scores, mode):
    torch = cuda
    g = lfr_graph(seed=1)
    sched = snap.linear_schedule(1.0, 30)
    layouts = []
    with snap.Layout(g.row_ptr, g.col_idx, opts=snap.make_options(mode=mode)) as L:
        for seed in SEEDS:
            pos = torch.from_numpy(initial_positions(g.n, seed)).cuda()
            L.epochs(pos, 0, 30, 3, sched, seed)
            L.check()
            layouts.append(pos.cpu().numpy().astype(np.float64))
    ctx = mp.get_context("spawn")
    with ctx.Pool(len(SEEDS)) as pool:
        gpu = np.array(pool.map(quality_jobs.lfr_score, layouts))
    o, m = oracle_scores.mean(0), gpu.mean(0)
    d_ob, d_np = m[0] / o[0] - 1, m[1] / o[1] - 1
    print(f"LFR mode={mode}: objective {m[0]:.1f} vs {o[0]:.1f} ({d_ob:+.2%}), NP {m[1]:.4f} vs {o[1]:.4f} "
          f"({d_np:+.2%})")
    assert abs(d_ob) < 0.02
    assert abs(d_np) < 0.02

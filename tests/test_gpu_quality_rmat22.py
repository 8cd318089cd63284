"""Hogwild quality at the bench's full size against stored oracle values:
R-MAT 2^22 / 34,000,000 edges (BFS relabelling), k = 3, 30 epochs, eta0 = 1,
seeds 1..5, both lock-free modes.  The mean objective of Eq. 4 and the mean
neighbourhood preservation (Section 4.1, r = 2) of the GPU layouts must be
within 2% of the means of the oracle's layouts (Algorithm 1, FP64), which
tests/golden/make_quality_rmat22.py computed with the oracle alone and stored
in tests/golden/quality_rmat22_k3.txt.  The GPU layouts are scored by the same
oracle functions on the same pair and vertex samples."""
import multiprocessing as mp
import os
import sys

import numpy as np
import pytest

import paper_2608_01907_gb300 as snap
from conftest import read_golden
from gpu_helpers import rmat22_bfs
from synth import initial_positions

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))


def _stored():
    rows = np.array([[float(x) for x in r[:4]] for r in read_golden("quality_rmat22_k3.txt")])
    return rows[:, 0].astype(int).tolist(), rows[:, 1], rows[:, 2], rows[:, 3]


def _score(path):
    import make_quality_rmat22 as mq
    Y = np.load(path)
    return mq.score(mq.graph(), Y)


@pytest.mark.parametrize("mode", [snap.MODE_HOGWILD_RED, snap.MODE_HOGWILD])
def test_full_size_hogwild_quality_within_two_percent_of_oracle(cuda, mode, tmp_path):
    import make_quality_rmat22 as mq
    torch = cuda
    seeds, ob_ref, np_ref, hub_ref = _stored()
    g = rmat22_bfs()
    sched = snap.linear_schedule(eta0=1.0, total_epochs=mq.EPOCHS)
    paths, drift = [], []
    with snap.Layout(g.row_ptr, g.col_idx, opts=snap.make_options(mode=mode)) as L:
        for seed in seeds:
            pos = torch.from_numpy(initial_positions(g.n, seed)).cuda()
            L.epochs(pos, 0, mq.EPOCHS, mq.K, sched, seed)
            L.check()
            Y = pos.cpu().numpy().astype(np.float64)
            assert np.all(np.isfinite(Y))
            Y0 = initial_positions(g.n, seed).astype(np.float64)
            # Algorithm 1 keeps the centroid (every update is +-F on two vertices)
            drift.append(np.linalg.norm(Y.mean(0) - Y0.mean(0)) / np.sqrt(((Y - Y0) ** 2).sum(1).mean()))
            p = str(tmp_path / f"layout_{seed}.npy")
            np.save(p, Y)
            paths.append(p)
    with mp.get_context("spawn").Pool(len(paths)) as pool:
        scores = np.array(pool.map(_score, paths))
    d_ob = scores[:, 0].mean() / ob_ref.mean() - 1
    d_np = scores[:, 1].mean() / np_ref.mean() - 1
    print(f"R-MAT 2^22 quality mode={mode}: objective {scores[:, 0].mean():.1f} vs oracle {ob_ref.mean():.1f} "
          f"({d_ob:+.2%}), NP {scores[:, 1].mean():.5f} vs {np_ref.mean():.5f} ({d_np:+.2%}); "
          f"per seed objective {' '.join(f'{v:.0f}' for v in scores[:, 0])}; hub offset "
          f"{scores[:, 2].mean():.3f} vs oracle {hub_ref.mean():.3f}; centroid drift / rms move "
          f"{np.mean(drift):.2e}")
    assert abs(d_ob) < 0.02
    assert abs(d_np) < 0.02

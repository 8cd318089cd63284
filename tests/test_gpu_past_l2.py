"""A graph whose positions do not fit in L2 (Section 5's scale, reduced to
what the oracle lays out in hours): R-MAT 2^25 / 268,435,456 undirected edges
(native generator, BFS relabelling; positions 268 MB, L2 126 MB), k = 3.

* Synchronous mode, chunk by chunk in the bench's configuration (16 chunks,
  cap 1, eta0 = 1): the GPU runs every chunk; after chunks 0, 7 and 15 the
  oracle takes the same chunk step from the GPU's positions before it, and
  every vertex must meet the 1e-4 gate.
* Hogwild (both modes), 30 epochs, seeds 1..3: mean objective (Eq. 4) and
  mean NP (Section 4.1) within 2% of the oracle's layouts stored by
  tests/golden/make_quality_rmat25.py (oracle and input generators only)."""
import multiprocessing as mp
import os
import sys

import numpy as np
import pytest

import oracle
import paper_2608_01907_gb300 as snap
from conftest import read_golden
from gpu_helpers import SYNC_RTOL, coordinate_error, rmat25_bfs, schedule_dict
from synth import initial_positions

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))


@pytest.fixture(scope="module")
def g25():
    return rmat25_bfs()


def test_past_l2_sync_chunk_steps_match_oracle(cuda, g25):
    torch = cuda
    g = g25
    S, cap, seed, K = 16, 1.0, 1, 3
    sched = snap.linear_schedule(eta0=1.0, total_epochs=30)
    sd = schedule_dict(sched)
    pos = torch.from_numpy(initial_positions(g.n, seed)).cuda()
    errs = {}
    with snap.Layout(g.row_ptr, g.col_idx,
                     opts=snap.make_options(mode=snap.MODE_SYNC, sync_substeps=S, sync_cap=cap)) as L:
        for c in range(S):
            check = c in (0, 7, 15)
            before = pos.cpu().numpy().astype(np.float64) if check else None
            L.sync_chunks(pos, 0, c, c + 1, K, sched, seed)
            L.check()
            if check:
                ref = oracle.sync_chunks(g.row_ptr, g.col_idx, g.n, before, 0, c, c + 1, S, K, sd, seed=seed,
                                         cap=cap)
                errs[c] = float(coordinate_error(pos.cpu().numpy(), ref).max())
    print(f"past-L2 sync chunk parity (R-MAT 2^25, n={g.n}, nnz={g.nnz}): max rel err per checked chunk {errs}")
    assert max(errs.values()) < SYNC_RTOL


def _score(path):
    import make_quality_rmat25 as mq
    return mq.score(mq.graph(), np.load(path))


@pytest.mark.parametrize("mode", [snap.MODE_HOGWILD_RED, snap.MODE_HOGWILD])
def test_past_l2_hogwild_quality_within_two_percent_of_oracle(cuda, g25, mode, tmp_path):
    import make_quality_rmat25 as mq
    torch = cuda
    rows = np.array([[float(x) for x in r[:4]] for r in read_golden("quality_rmat25_k3.txt")])
    seeds = rows[:, 0].astype(int).tolist()
    g = g25
    sched = snap.linear_schedule(eta0=1.0, total_epochs=mq.EPOCHS)
    paths = []
    with snap.Layout(g.row_ptr, g.col_idx, opts=snap.make_options(mode=mode)) as L:
        for seed in seeds:
            pos = torch.from_numpy(initial_positions(g.n, seed)).cuda()
            L.epochs(pos, 0, mq.EPOCHS, mq.K, sched, seed)
            L.check()
            Y = pos.cpu().numpy().astype(np.float64)
            assert np.all(np.isfinite(Y))
            p = str(tmp_path / f"layout_{seed}.npy")
            np.save(p, Y)
            paths.append(p)
            del Y
    with mp.get_context("spawn").Pool(len(paths)) as pool:
        scores = np.array(pool.map(_score, paths))
    d_ob = scores[:, 0].mean() / rows[:, 1].mean() - 1
    d_np = scores[:, 1].mean() / rows[:, 2].mean() - 1
    print(f"R-MAT 2^25 quality mode={mode}: objective {scores[:, 0].mean():.1f} vs oracle {rows[:, 1].mean():.1f} "
          f"({d_ob:+.2%}), NP {scores[:, 1].mean():.5f} vs {rows[:, 2].mean():.5f} ({d_np:+.2%}); hub offset "
          f"{scores[:, 2].mean():.3f} vs {rows[:, 3].mean():.3f}")
    assert abs(d_ob) < 0.02
    assert abs(d_np) < 0.02

"""Convergence against the number of epochs T (Section 4.2, Fig. 5a) on the
LFR-style community graph (260,000 vertices, ~6.9M edges): GPU layouts of both
lock-free modes after T = 10 and T = 30 epochs against the oracle's stored
scores (tests/golden/convergence_lfr.txt, written by
tests/golden/make_convergence_lfr.py from the oracle alone).

Section 4.3 reports the lock-free variants within [-5%, 5%] of the serial
algorithm in SI and NP; after 30 epochs both GPU modes must be within that
band in SI and within 2% in NP, and SI must rise from 10 to 30 epochs as it
does for the oracle.  The GPU side is a mean over runs (16 at T = 30, 3 at
T = 10): the lock-free modes' races differ from run to run (SI spread about
0.009 at T = 30)."""
import multiprocessing as mp
import os
import sys

import numpy as np
import pytest

import paper_2608_01907_gb300 as snap
from conftest import read_golden
from gpu_helpers import lfr260k
from synth import initial_positions

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))


def _score(path):
    import make_convergence_lfr as mc
    return mc.score(mc.graph(), np.load(path))


@pytest.mark.parametrize("mode", [snap.MODE_HOGWILD_RED, snap.MODE_HOGWILD])
def test_gpu_convergence_in_T_matches_oracle(cuda, mode, tmp_path):
    import make_convergence_lfr as mc
    torch = cuda
    ref = {int(r[0]): (float(r[1]), float(r[2])) for r in read_golden("convergence_lfr.txt")}
    g = lfr260k()
    # the racy modes' layouts differ from run to run (SI spread about 0.009 at
    # T = 30): the scores are means over several runs, 16 at T = 30 where the
    # band is asserted, 3 at T = 10
    runs = {10: 3, 30: 16}
    paths = {T: [] for T in mc.TS}
    with snap.Layout(g.row_ptr, g.col_idx, opts=snap.make_options(mode=mode)) as L:
        for T in mc.TS:
            for run in range(runs[T]):
                pos = torch.from_numpy(initial_positions(g.n, mc.SEED)).cuda()
                L.epochs(pos, 0, T, mc.K, snap.linear_schedule(1.0, T), mc.SEED)
                L.check()
                p = str(tmp_path / f"T{T}_{run}.npy")
                np.save(p, pos.cpu().numpy().astype(np.float64))
                paths[T].append(p)
    flat = [p for T in mc.TS for p in paths[T]]
    with mp.get_context("spawn").Pool(min(len(flat), 12)) as pool:
        flat_scores = pool.map(_score, flat)
    scores, at = {}, 0
    for T in mc.TS:
        scores[T] = np.array(flat_scores[at:at + runs[T]])
        at += runs[T]
    got = {T: scores[T].mean(axis=0) for T in mc.TS}
    print(f"LFR mode={mode} SI per run: " + "; ".join(f"T={T}: " + " ".join(f"{x:.4f}" for x in scores[T][:, 0])
                                                         for T in mc.TS))
    for T in mc.TS:
        print(f"LFR mode={mode} T={T}: SI {got[T][0]:.4f} vs oracle {ref[T][0]:.4f} "
              f"({got[T][0] / ref[T][0] - 1:+.2%}), NP {got[T][1]:.4f} vs {ref[T][1]:.4f} "
              f"({got[T][1] / ref[T][1] - 1:+.2%})")
    assert ref[30][0] > ref[10][0] and got[30][0] > got[10][0]
    assert abs(got[30][0] / ref[30][0] - 1) < 0.05
    assert abs(got[30][1] / ref[30][1] - 1) < 0.02

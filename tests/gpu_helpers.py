"""Helpers shared by the GPU tests: run the CUDA path through the C ABI and
compare with the oracle."""
import numpy as np

import paper_2608_01907_gb300 as snap

# Per-coordinate parity gate of the synchronous mode after one epoch: FP32
# kernel against the FP64 oracle on the same Philox streams.  The error of a
# difference y_i - y_j in FP32 scales with the magnitude of the positions, not
# of the difference, so each coordinate's error is measured relative to
# max(|y|, rms(Y)).
SYNC_RTOL = 1e-4


def parity_error(gpu: np.ndarray, ref: np.ndarray) -> float:
    ref = np.asarray(ref, dtype=np.float64)
    gpu = np.asarray(gpu, dtype=np.float64)
    scale = max(float(np.sqrt((ref ** 2).mean())), 1e-30)
    return float((np.abs(gpu - ref) / np.maximum(np.abs(ref), scale)).max())


def schedule_dict(s: snap.SnapSchedule) -> dict:
    return dict(kind=s.kind, eta0=s.eta0, eta_min=s.eta_min, total_epochs=s.total_epochs)


def gpu_layout(torch, g, Y0, epochs, k, sched, seed, opts=None, epoch_begin=0):
    """Runs epochs on the GPU through the C ABI; returns the float32 positions."""
    pos = torch.from_numpy(np.ascontiguousarray(Y0, dtype=np.float32)).cuda()
    with snap.Layout(g.row_ptr, g.col_idx, opts=opts) as L:
        L.epochs(pos, epoch_begin, epochs, k, sched, seed)
        L.check()
    torch.cuda.synchronize()
    return pos.cpu().numpy()

"""Learned per-pose selector: training labels and the selection rule, both
computed by the library's kernels (ligate_selector_labels,
ligate_select_poses); this module only moves arrays.  Paper Sec. 3.5: a
high-throughput pose selector that gives up a little accuracy for a large
gain in throughput.

Labels: the exact rescored energy of a pose that passes the filter, clipped
to `fail_label`; `fail_label` for a pose that fails.  Selection for one
ligand: among its poses in docking order, the first whose predicted label is
below fail_label / 2 (predicted to pass); if none, the lowest prediction.
Empty slots never win.
"""
from __future__ import annotations

import numpy as np

from . import native as N

FAIL_LABEL = 30.0


def _dev(a, dtype=None):
    import torch
    if isinstance(a, np.ndarray):
        t = torch.from_numpy(np.ascontiguousarray(a))
        return (t.to(dtype) if dtype is not None else t).cuda()
    return a


def labels(rescored, fail_label: float = FAIL_LABEL):
    """Training labels (CUDA float32 tensor) of RESCORED_DTYPE records given
    as a host array or a CUDA byte tensor."""
    import torch
    if isinstance(rescored, np.ndarray):
        n = rescored.size
        buf = _dev(np.ascontiguousarray(rescored).reshape(-1).view(np.uint8))
    else:
        n = rescored.numel() // N.RESCORED_DTYPE.itemsize
        buf = rescored
    out = torch.empty(max(n, 1), dtype=torch.float32, device="cuda")
    N.ligate_selector_labels(buf, n, fail_label, out)
    return out[:n]


def select(pred, poses, fail_label: float = FAIL_LABEL):
    """Slot of the kept pose per row (host int32 [n]): pred [n, K] FP32 and
    poses POSE_DTYPE [n, K] (host arrays or CUDA tensors; a slot with
    start_id < 0 is empty); -1 for a row without a pose."""
    import torch
    if isinstance(poses, np.ndarray):
        n, k = poses.shape
        pz = _dev(np.ascontiguousarray(poses).reshape(-1).view(np.uint8))
    else:
        n, k = pred.shape
        pz = poses
    pr = _dev(np.asarray(pred, np.float32)) if isinstance(pred, np.ndarray) else pred
    idx = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    N.ligate_select_poses(pr, pz, n, k, 0.5 * fail_label, idx)
    torch.cuda.synchronize()
    return idx[:n].cpu().numpy()

"""Learned per-pose selector: labels and selection rule (host side; the
features, the exact rescoring and the network run on the GPU through the C
ABI).  Paper Sec. 3.5: a high-throughput pose selector that gives up a
little accuracy for a large gain in throughput.

Labels: the exact rescored energy of a pose that passes the filter, clipped
to `fail_label`; `fail_label` for a pose that fails.  Selection for one
ligand: among its poses in docking order, the first whose predicted label is
below fail_label / 2 (predicted to pass); if none, the lowest prediction.
Empty slots never win.
"""
from __future__ import annotations

import numpy as np

FAIL_LABEL = 30.0


def labels(rescored: np.ndarray, fail_label: float = FAIL_LABEL) -> np.ndarray:
    """Training labels of RESCORED_DTYPE records (any shape)."""
    e = rescored["energy"].astype(np.float64)
    return np.where(rescored["pass"] == 1, np.minimum(e, fail_label), fail_label).astype(np.float32)


def select(pred: np.ndarray, live: np.ndarray, fail_label: float = FAIL_LABEL) -> np.ndarray:
    """Index of the kept pose per row of pred [n, K] (docking order along
    K); live [n, K] marks real poses.  -1 for a row without any."""
    p = np.where(live, pred, np.inf)
    ok = live & (p < 0.5 * fail_label)
    best = np.argmin(p, axis=1)
    pick = np.where(ok.any(axis=1), np.argmax(ok, axis=1), best)
    return np.where(live.any(axis=1), pick, -1)

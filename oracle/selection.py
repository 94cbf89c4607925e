"""Oracle of the per-ligand selection rules that follow docking.

TEST INFRASTRUCTURE ONLY (like the rest of this package).  Plain Python,
written from the definitions, one row at a time:

  best_passing  (paper Sec. 2: the generated poses are rescored and
      filtered, and a ligand scores as its best pose): per row, the slot of
      the lowest energy among the poses that pass the filter, ties to the
      smaller slot; -1 (energy +inf) when none passes.
  select_poses  (paper Sec. 3.5: a learned pose selector keeps one pose per
      ligand): per row of poses in docking order, the first live pose whose
      predicted label is below `pass_below`; else the live pose with the
      lowest prediction (ties: the smaller slot); -1 without a live pose.
  selector_labels: the training label of a rescored pose, its energy
      clipped to `fail_label` when it passes, `fail_label` otherwise.
"""
from __future__ import annotations

import math


def best_passing(energy, passed):
    idx, best = [], []
    for row_e, row_p in zip(energy, passed):
        k_best, e_best = -1, math.inf
        for k, (e, p) in enumerate(zip(row_e, row_p)):
            if p and (k_best < 0 or e < e_best):
                k_best, e_best = k, float(e)
        idx.append(k_best)
        best.append(e_best)
    return idx, best


def select_poses(pred, live, pass_below):
    out = []
    for row_v, row_l in zip(pred, live):
        first, low, low_v = -1, -1, math.inf
        for k, (v, l) in enumerate(zip(row_v, row_l)):
            if not l:
                continue
            if first < 0 and v < pass_below:
                first = k
            if low < 0 or v < low_v:
                low, low_v = k, float(v)
        out.append(first if first >= 0 else low)
    return out


def selector_labels(energy, passed, fail_label):
    return [min(float(e), fail_label) if p else fail_label for e, p in zip(energy, passed)]

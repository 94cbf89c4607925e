"""Host-side triage bookkeeping (paper Sec. 3.5: a learned predictor ranks
the library so that only its top fraction is docked; full docking stays the
arbiter of recall).

Scores are docking scores (lower = better).  The true top set is the
ceil(n * top_frac) ligands with the lowest full-docking score (ties: smaller
index), the same order as the ranking kernel uses.
"""
from __future__ import annotations

import math

import numpy as np


def _order(scores):
    scores = np.asarray(scores)
    return np.lexsort((np.arange(len(scores)), scores))


def _count(n, frac):
    return int(math.ceil(n * frac - 1e-9))


def true_top(scores, top_frac=0.01):
    """Indices of the true top set."""
    return _order(scores)[:_count(len(scores), top_frac)]


def recall(truth_scores, kept, top_frac=0.01):
    """Fraction of the true top set that is among `kept` (indices)."""
    top = true_top(truth_scores, top_frac)
    if len(top) == 0:
        return 1.0
    return len(set(top.tolist()) & set(np.asarray(kept).tolist())) / len(top)


def recall_curve(pred, truth_scores, fracs, top_frac=0.01):
    """Recall of the true top set when keeping the predicted best fraction f."""
    order = _order(pred)
    return {float(f): recall(truth_scores, order[:_count(len(pred), f)], top_frac) for f in fracs}


def keep_for_recall(pred, truth_scores, target=0.99, top_frac=0.01):
    """Smallest keep fraction whose predicted-best set holds `target` of the
    true top set (exact, from the predicted ranks of the true top items)."""
    n = len(pred)
    top = true_top(truth_scores, top_frac)
    if n == 0 or len(top) == 0:
        return 0.0
    rank = np.empty(n, np.int64)
    rank[_order(pred)] = np.arange(n)
    need = _count(len(top), target)
    r = np.sort(rank[top])[need - 1] if need > 0 else -1
    return (r + 1) / n

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


def calibration_target(n_library, recall_target=0.99, top_frac=0.01, confidence=0.95):
    """Per-ligand hit rate to calibrate the keep fraction for, so that a
    library of `n_library` ligands meets `recall_target` with probability
    `confidence`.

    The library's true top set holds P = ceil(n_library * top_frac) ligands,
    and it meets the target while at most a = floor(P * (1 - recall_target))
    of them are missed.  If each is missed independently at rate m, the
    misses are close to Poisson(P * m); the returned 1 - m is the rate whose
    Poisson tail P(misses > a) equals 1 - confidence.  A small library needs
    a wide margin (100 true top ligands: 0.9964), a large one almost none
    (10,000: about 0.9916)."""
    P = _count(n_library, top_frac)
    if P == 0:
        return recall_target
    a = int(math.floor(P * (1.0 - recall_target) + 1e-9))

    def tail(lam):  # P(Poisson(lam) > a), summed in log space
        if lam <= 0.0:
            return 0.0
        logs = [-lam + i * math.log(lam) - math.lgamma(i + 1) for i in range(a + 1)]
        top = max(logs)
        cdf = math.exp(top) * sum(math.exp(v - top) for v in logs)
        return max(0.0, 1.0 - cdf)

    lo, hi = 0.0, float(a + 1) + 10.0 * math.sqrt(a + 1) + 10.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if tail(mid) > 1.0 - confidence:
            hi = mid
        else:
            lo = mid
    return max(recall_target, 1.0 - lo / P)

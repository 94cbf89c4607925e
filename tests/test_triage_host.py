"""Triage bookkeeping on the host: recall and the keep fraction that reaches
a recall target, checked against brute force."""
import numpy as np

from paper_2304_09953_gb300 import triage as T


def brute_keep(pred, truth, target, top_frac):
    n = len(pred)
    for m in range(0, n + 1):
        kept = np.lexsort((np.arange(n), pred))[:m]
        if T.recall(truth, kept, top_frac) >= target - 1e-12:
            return m / n
    return 1.0


def test_perfect_and_reversed_predictions():
    truth = np.arange(1000, dtype=np.float64)
    assert T.keep_for_recall(truth, truth, 0.99) == 0.01
    assert T.keep_for_recall(-truth, truth, 0.99) == 1.0
    assert T.recall_curve(truth, truth, [0.01, 0.5])[0.01] == 1.0


def test_keep_fraction_matches_brute_force():
    rng = np.random.default_rng(5)
    for n in (50, 333, 1000):
        truth = rng.normal(size=n)
        pred = truth + rng.normal(scale=1.5, size=n)
        for target in (0.5, 0.9, 0.99, 1.0):
            for top in (0.01, 0.05):
                assert abs(T.keep_for_recall(pred, truth, target, top) - brute_keep(pred, truth, target, top)) < 1e-12


def test_ties_resolve_to_smaller_index():
    truth = np.zeros(200)
    assert list(T.true_top(truth, 0.01)) == [0, 1]
    assert T.recall(truth, [0, 1]) == 1.0

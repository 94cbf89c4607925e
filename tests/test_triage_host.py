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


def test_calibration_target_poisson_tail():
    import math
    # 100 true top ligands, one miss allowed: 1 - exp(-lam) (1 + lam) = 0.05
    t = T.calibration_target(10000)
    lam = (1.0 - t) * 100
    assert abs(1.0 - math.exp(-lam) * (1.0 + lam) - 0.05) < 1e-9
    # 10 true top ligands, no miss allowed: 1 - exp(-lam) = 0.05
    lam = (1.0 - T.calibration_target(1000)) * 10
    assert abs(lam + math.log(0.95)) < 1e-9
    # the normal limit for a large top set: lam ~ a - 1.645 sqrt(a), a = 100
    lam = (1.0 - T.calibration_target(1_000_000)) * 10000
    assert 80.0 < lam < 86.0
    # never below the recall target itself; a stricter confidence asks more
    assert T.calibration_target(100) == 0.99
    assert T.calibration_target(10000, confidence=0.99) > T.calibration_target(10000)


def test_calibration_target_by_simulation():
    # misses drawn at the returned rate meet the target in ~95% of libraries
    rng = np.random.default_rng(9)
    t = T.calibration_target(10000)
    misses = rng.binomial(100, 1.0 - t, size=20000)
    frac_ok = np.mean(misses <= 1)
    assert 0.94 < frac_ok < 0.96

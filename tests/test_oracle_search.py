"""Pins for the oracle's greedy multi-start search and top-K.

Brute force fixes the search: for R <= 1 the greedy sweep IS the exhaustive
per-start optimum; for larger R the exhaustive minimum bounds the greedy
result from below and contains each greedy pose's score at its torsion
combination; each bond's choice is the argmin of its trial row, and the next
bond's k = 0 trial repeats the chosen pose.  Top-K is a sort on (E, start).
"""
import numpy as np
import pytest

import oracle
from paper_2304_09953_gb300.workload import Sampling, make_ligands


def _small(seed, n_atoms, n_rot, S=6, n_orient=8, n_anchor=4, pocket=None):
    ligs = make_ligands(seed, np.array([n_atoms], np.int32), np.array([n_rot], np.int32), 6)
    rng = np.random.default_rng(seed)
    samp = Sampling(rng.normal(size=(n_orient, 4)), n_anchor, S, 4)
    return ligs.ligand(0), samp


def test_r0_greedy_is_rigid_score(tiny):
    lig, samp = _small(11, 14, 0)
    P = tiny.pocket
    e, tors = oracle.greedy(lig, P, samp)
    want = oracle.score_poses(lig, P, samp, np.arange(samp.n_starts), np.zeros((samp.n_starts, 0)))
    np.testing.assert_array_equal(e, want)
    assert tors.shape == (samp.n_starts, 0)


def test_r1_greedy_equals_exhaustive(tiny):
    lig, samp = _small(12, 16, 1, S=8)
    P = tiny.pocket
    e, tors = oracle.greedy(lig, P, samp)
    ex = oracle.exhaustive(lig, P, samp, np.arange(samp.n_starts))
    np.testing.assert_array_equal(e, ex.min(axis=1))
    # ties -> smaller k: argmin returns the first minimum
    np.testing.assert_array_equal(tors[:, 0], ex.argmin(axis=1))


@pytest.mark.parametrize("n_rot", [2, 3])
def test_exhaustive_bounds_greedy(tiny, n_rot):
    lig, samp = _small(13 + n_rot, 18, n_rot, S=5, n_orient=4, n_anchor=4)
    R = int(lig[3].sum())
    assert R == n_rot
    P = tiny.pocket
    e, tors = oracle.greedy(lig, P, samp)
    ex = oracle.exhaustive(lig, P, samp, np.arange(samp.n_starts))
    assert np.all(ex.min(axis=1) <= e)
    code = np.zeros(samp.n_starts, np.int64)
    for b in reversed(range(R)):
        code = code * samp.torsion_steps + tors[:, b]
    np.testing.assert_array_equal(ex[np.arange(samp.n_starts), code], e)


def test_greedy_trial_rows_are_consistent(tiny):
    """Each bond's choice is the first argmin of its S trials; the chosen
    score equals the k = 0 trial of the next bond (unchanged pose)."""
    lig, samp = _small(21, 30, 5, S=8, n_orient=16, n_anchor=4)
    e, tors, tr = oracle.greedy(lig, tiny.pocket, samp, trials=True)
    R = tors.shape[1]
    for b in range(R):
        np.testing.assert_array_equal(tors[:, b], tr[:, b].argmin(axis=1))
        best = tr[np.arange(len(e)), b, tors[:, b]]
        if b + 1 < R:
            np.testing.assert_array_equal(best, tr[:, b + 1, 0])
        else:
            np.testing.assert_array_equal(best, e)
    # the greedy result is reproduced by scoring its pose directly
    np.testing.assert_array_equal(oracle.score_poses(lig, tiny.pocket, samp, np.arange(len(e)), tors), e)


def test_top_k_is_sort_on_score_then_start():
    e = np.array([3.0, 1.0, 2.0, 1.0, -5.0, 2.0, 1.0])
    idx = oracle.top_k(e, 5)
    assert list(idx) == [4, 1, 3, 6, 2]
    rng = np.random.default_rng(0)
    e = rng.integers(0, 20, size=1000).astype(float)
    idx = oracle.top_k(e, 50)
    pairs = sorted(zip(e, range(len(e))))[:50]
    assert list(idx) == [p[1] for p in pairs]


def test_tiny_config_shape(tiny):
    """1 ligand, 24 atoms, 4 rotatable bonds, 512 starts of 1 + 4 * 7 poses."""
    assert tiny.ligands.n == 1 and tiny.ligands.n_atoms()[0] == 24
    assert tiny.ligands.n_rot[0] == 4
    assert tiny.sampling.n_starts == 512 and tiny.sampling.torsion_steps == 8
    s, st, t = oracle.dock_ligand(tiny.ligands.ligand(0), tiny.pocket, tiny.sampling)
    assert len(s) == 4 and np.all(np.diff(s) >= 0)

"""Pins of the FP64 pose-feature oracle (inputs of the learned pose
selector): the histogram counts every atom once, a constant map puts every
atom in the bin of that constant, per-type means and the score entry agree
with the docking score of the same pose, and the trailing entries are the
atom and bond counts."""
import dataclasses

import numpy as np

import oracle


def test_features_follow_their_definition(tiny):
    w = tiny
    lig = w.ligands.ligand(0)
    n = len(lig[1])
    R_n = int(np.sum(lig[3] != 0))
    rng = np.random.default_rng(9)
    starts = rng.integers(0, w.sampling.n_starts, size=40)
    tors = rng.integers(0, w.sampling.torsion_steps, size=(40, R_n))
    x = oracle.pose_coords(lig, w.pocket.anchors, w.sampling, starts, tors)
    f = oracle.pose_features(lig, w.pocket, w.sampling, x)
    np.testing.assert_allclose(np.sum(np.expm1(f[:, :64]), axis=1), n, rtol=1e-12)
    score = oracle.score_poses(lig, w.pocket, w.sampling, starts, tors)
    np.testing.assert_allclose(f[:, 72] * n, score, rtol=1e-12)
    assert np.all(f[:, 74] == np.log1p(n)) and np.all(f[:, 75] == R_n)
    assert np.all(f[:, 77:] == 0)
    # the per-type means weighted by the type counts give the grid sum
    counts = np.bincount(lig[1], minlength=8)[:8]
    grid_sum = f[:, 72] * n - f[:, 73]
    np.testing.assert_allclose(f[:, 64:72] @ counts, grid_sum, rtol=1e-10, atol=1e-9)


def test_constant_map_fills_one_bin(tiny):
    w = tiny
    lig = w.ligands.ligand(0)
    n = len(lig[1])
    P = dataclasses.replace(w.pocket, maps=np.full_like(w.pocket.maps, 1.3))
    x = oracle.pose_coords(lig, w.pocket.anchors, w.sampling, [0], np.zeros((1, int(np.sum(lig[3] != 0))), int))
    f = oracle.pose_features(lig, P, w.sampling, x)[0]
    inside = np.all((x[0] >= 0) & (x[0] <= (np.array(w.pocket.dims) - 1) * w.pocket.spacing), axis=1).sum()
    b = int(np.floor((np.float32(1.3) + 4) * 4))
    assert f[b] == np.log1p(inside)
    if inside < n:  # the rest score the penalty (10: bin 56)
        assert f[56] == np.log1p(n - inside)
    assert f[76] == np.log1p(n - inside)

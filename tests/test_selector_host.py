"""Pins of the oracle's post-docking selection rules on hand-made records
(the expected slots worked out by hand from the definitions), and the
library's versions of them against the oracle on the GPU."""
import math

import numpy as np
import pytest

from oracle import selection as O


def test_best_passing_by_hand():
    energy = [[-3.0, -5.0, -4.0, 1.0],   # slot 1 passes with the lowest energy
              [-9.0, 2.0, 2.0, 0.5],     # the lowest (slot 0) fails; tie 2.0 at slots 1, 2 loses to 0.5
              [1.0, 1.0, 3.0, -2.0],     # tie between slots 0 and 1 -> 0 (slot 3 fails)
              [0.0, 0.0, 0.0, 0.0]]      # nothing passes
    passed = [[1, 1, 1, 0], [0, 1, 1, 1], [1, 1, 1, 0], [0, 0, 0, 0]]
    idx, best = O.best_passing(energy, passed)
    assert idx == [1, 3, 0, -1]
    assert best[:3] == [-5.0, 0.5, 1.0] and math.isinf(best[3])


def test_select_poses_by_hand():
    pred = [[20.0, 3.0, -5.0], [40.0, 35.0, 29.0], [1.0, 2.0, 3.0], [0.0, 0.0, 0.0], [16.0, 15.0, 15.0]]
    live = [[1, 1, 1], [1, 1, 1], [0, 1, 1], [0, 0, 0], [1, 1, 1]]
    # row 0: slot 1 is the first below 15; row 1: none below, lowest 29 at 2;
    # row 2: slot 0 empty, slot 1 first below; row 3: no pose; row 4: 15 is
    # not below 15, lowest 15.0 tie -> slot 1
    assert O.select_poses(pred, live, 15.0) == [1, 2, 1, -1, 1]


def test_selector_labels_by_hand():
    assert O.selector_labels([-3.0, 50.0, -1.0, math.inf], [1, 1, 0, 0], 30.0) == [-3.0, 30.0, 30.0, 30.0]


@pytest.mark.gpu
def test_library_rules_equal_the_oracle():
    """ligate_plan_best_passing, ligate_select_poses and
    ligate_selector_labels on seeded records with ties, failures and empty
    slots, bit for bit against the oracle (integer slots; the energies and
    labels are copies or a min with a constant)."""
    torch = pytest.importorskip("torch")
    from paper_2304_09953_gb300 import docking as D
    from paper_2304_09953_gb300 import native as N
    from paper_2304_09953_gb300 import selector as SEL
    from paper_2304_09953_gb300.workload import make_workload
    w = make_workload("batched", n_ligands=64)
    ph = D.PocketHandle(w.pocket)
    bh = D.BatchHandle(w.ligands)
    pl = D.Plan(ph, bh, w.sampling, mode="fp32")
    n, K = 64, w.sampling.top_k
    rng = np.random.default_rng(3)
    for trial in range(5):
        rec = np.zeros((n, K), N.RESCORED_DTYPE)
        rec["energy"] = rng.choice([-2.0, -1.0, 0.0, 5.0, 40.0, np.inf], size=(n, K))
        rec["pass"] = rng.integers(0, 2, size=(n, K))
        rec["pass"][::7] = 0  # rows where nothing passes
        idx, e = pl.best_passing(rec)
        oi, oe = O.best_passing(rec["energy"], rec["pass"] == 1)
        assert list(idx) == oi and list(e) == [np.float32(v) for v in oe]
        assert np.any(idx == -1) and np.any(idx >= 0)
        lab = SEL.labels(rec).cpu().numpy()
        assert list(lab) == [np.float32(v) for v in O.selector_labels(rec["energy"].reshape(-1),
                                                                       rec["pass"].reshape(-1) == 1, 30.0)]
    m = 300
    poses = np.zeros((m, K), N.POSE_DTYPE)
    poses["start_id"] = np.where(rng.random((m, K)) < 0.2, -1, 7)
    pred = rng.choice([-3.0, 0.0, 14.0, 15.0, 16.0, 40.0], size=(m, K)).astype(np.float32)
    got = SEL.select(pred, poses)
    want = O.select_poses(pred, poses["start_id"] >= 0, 15.0)
    assert list(got) == want
    pl.close()

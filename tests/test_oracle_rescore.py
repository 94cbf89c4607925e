"""Pins of the FP64 exact-rescoring oracle.

The exact receptor term is the function the grid maps tabulate: at grid
nodes it must reproduce the maps (computed by the workload generator, a
separate FP64 implementation, then rounded to FP32).  Closed forms: one
receptor atom at distance r0 gives -eps, beyond the cutoff nothing, closer
than the radius floor the floor's value (capped).  The clash part equals the
docking score's clash term; the filter counts out-of-box and capped atoms."""
import dataclasses

import numpy as np

import oracle


def one_atom(xyz, t):
    return (np.asarray([xyz], np.float32), np.array([t], np.uint8), np.zeros((0, 2), np.int32),
            np.zeros(0, np.uint8))


def test_exact_term_reproduces_the_maps_at_nodes(tiny):
    w = tiny
    P = w.pocket
    rec = P.receptor()
    rng = np.random.default_rng(4)
    nx, ny, nz = P.dims
    checked = 0
    for _ in range(60):
        ix, iy, iz = rng.integers(0, nx), rng.integers(0, ny), rng.integers(0, nz)
        t = int(rng.integers(0, P.n_types))
        x = np.asarray(P.origin) + P.spacing * np.array([ix, iy, iz])
        lig = one_atom(x, t)
        r = oracle.rescore_coords(lig, P, w.sampling, rec, x[None, None, :])
        want = float(P.maps[t, iz, iy, ix])
        # the maps used FP64 receptor coordinates, the rescoring their FP32 copy
        assert abs(r["e_inter"][0] - want) <= 1e-5 * max(abs(want), 1.0), (ix, iy, iz, t)
        assert r["n_capped"][0] == (want >= P.cap)
        checked += 1
    assert checked == 60


def test_single_receptor_atom_closed_forms(tiny):
    w = tiny
    P = w.pocket
    radius, eps = np.array([1.6, 1.9]), np.array([0.15, 0.25])
    rec = {"xyz": np.zeros((1, 3), np.float32) + 5.0, "type": np.array([1], np.int32),
           "radius": radius, "eps": eps, "cutoff": 8.0, "cap": 10.0, "rmin": 0.5}
    r0 = radius[0] + radius[1]
    e = np.sqrt(eps[0] * eps[1])
    pts = np.array([[5.0 + r0, 5, 5], [5, 5.0 + 8.5, 5], [5, 5, 5.0 + 0.2], [5.0 + 2 * r0, 5, 5]])
    got = [oracle.rescore_coords(one_atom(p, 0), P, w.sampling, rec, p[None, None, :])["e_inter"][0]
           for p in pts]
    np.testing.assert_allclose(got[0], -e, rtol=1e-12)
    assert got[1] == 0.0
    assert got[2] == 10.0  # floor 0.5 A: (r0/0.5)^12 eps is far above the cap
    np.testing.assert_allclose(got[3], e * (0.5 ** 12 - 2 * 0.5 ** 6), rtol=1e-12)


def test_clash_part_is_the_docking_clash_term_and_flags(tiny):
    w = tiny
    lig = w.ligands.ligand(0)
    P0 = dataclasses.replace(w.pocket, maps=np.zeros_like(w.pocket.maps))
    rng = np.random.default_rng(6)
    R_n = int(np.sum(lig[3] != 0))
    starts = rng.integers(0, w.sampling.n_starts, size=80)
    tors = rng.integers(0, w.sampling.torsion_steps, size=(80, R_n))
    x = oracle.pose_coords(lig, w.pocket.anchors, w.sampling, starts, tors)
    r = oracle.rescore_coords(lig, w.pocket, w.sampling, w.pocket.receptor(), x)
    dock = oracle.score_poses(lig, P0, w.sampling, starts, tors)
    inside = r["n_outside"] == 0
    assert inside.sum() >= 5
    # zero maps: inside the box the docking score is the clash term alone
    np.testing.assert_allclose(r["e_clash"][inside], dock[inside], rtol=1e-12, atol=1e-12)
    # out-of-box atoms counted: push a pose far away
    far = x[:1] + 100.0
    rf = oracle.rescore_coords(lig, w.pocket, w.sampling, w.pocket.receptor(), far)
    assert rf["n_outside"][0] == x.shape[1] and rf["e_inter"][0] == 0.0

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


def test_per_atom_inputs_reproduce_the_filter_and_closed_forms(tiny):
    """rescore_atoms: its per-atom sums, capped and summed, are e_inter; the
    atoms at or above the cap are n_capped and those with a negative face
    distance n_outside; one receptor atom at r0 gives -eps with magnitude
    eps; the face distance is the closed form for points placed by hand."""
    w = tiny
    P = w.pocket
    lig = w.ligands.ligand(0)
    rec = P.receptor()
    rng = np.random.default_rng(8)
    R_n = int(np.sum(lig[3] != 0))
    starts = rng.integers(0, w.sampling.n_starts, size=40)
    tors = rng.integers(0, w.sampling.torsion_steps, size=(40, R_n))
    x = oracle.pose_coords(lig, P.anchors, w.sampling, starts, tors)
    x[:3] += 30.0 * rng.normal(size=(3, 1, 3))  # some poses leave the box
    r = oracle.rescore_coords(lig, P, w.sampling, rec, x)
    s, m, f = oracle.rescore_atoms(lig, P, rec, x)
    np.testing.assert_allclose(np.minimum(s, P.cap).sum(axis=1), r["e_inter"], rtol=1e-12, atol=1e-12)
    np.testing.assert_array_equal((s >= P.cap).sum(axis=1), r["n_capped"])
    np.testing.assert_array_equal((f < 0).sum(axis=1), r["n_outside"])
    assert np.all(m >= np.abs(s) - 1e-12)
    assert r["n_outside"][:3].sum() > 0 and np.any(r["n_capped"] > 0)
    # closed forms: one receptor atom; faces of the box
    radius, eps = np.array([1.6, 1.9]), np.array([0.15, 0.25])
    one = {"xyz": np.zeros((1, 3), np.float32) + 5.0, "type": np.array([1], np.int32),
           "radius": radius, "eps": eps, "cutoff": 8.0, "cap": 10.0, "rmin": 0.5}
    r0 = radius[0] + radius[1]
    p = np.array([5.0 + r0, 5.0, 5.0])
    s1, m1, f1 = oracle.rescore_atoms(one_atom(p, 0), P, one, p[None, None, :])
    np.testing.assert_allclose(s1[0, 0], -np.sqrt(eps[0] * eps[1]), rtol=1e-12)
    np.testing.assert_allclose(m1[0, 0], np.sqrt(eps[0] * eps[1]), rtol=1e-12)
    nx, ny, nz = P.dims
    o, h = np.asarray(P.origin), P.spacing
    for u, want in (([0.25, 5.0, 7.0], 0.25), ([3.0, ny - 1.5, 9.0], 0.5), ([-0.75, 4.0, 4.0], -0.75),
                    ([4.0, 4.0, nz - 1 + 2.0], -2.0)):
        q = o + h * np.array(u)
        _, _, fq = oracle.rescore_atoms(one_atom(q, 0), P, one, q[None, None, :])
        np.testing.assert_allclose(fq[0, 0], want, atol=1e-12)

"""Pins of the FP64 refinement oracle (gradient descent from docked poses).

The generalised gradient (translation F, rotation tau, torsions psi) is
pinned by central differences of the oracle's own energy along the motions
it claims to differentiate, by closed forms on linear maps (constant
per-atom gradient; zero torque of a rigid ligand about its centroid) and by
the pair symmetry of the clash term (no net force or torque).  The descent
is pinned by its invariants (monotone, orthonormal rotation, zero
iterations change nothing, following its own decisions reproduces itself)
and by a closed-form trajectory on a linear map."""
import dataclasses

import numpy as np
import pytest

import oracle


def rand_rot(rng):
    q = rng.normal(size=4)
    return oracle.quat_to_matrix(q / np.linalg.norm(q))


def rot_exp(w):
    th = np.linalg.norm(w)
    if th == 0:
        return np.eye(3)
    n = w / th
    K = np.array([[0, -n[2], n[1]], [n[2], 0, -n[0]], [-n[1], n[0], 0]])
    return np.eye(3) + np.sin(th) * K + (1 - np.cos(th)) * K @ K


def states_for(w, lig, rng, n, spread=1.0):
    R_n = int(np.sum(np.asarray(lig[3]) != 0))
    centre = np.asarray(w.pocket.origin) + 0.5 * (np.array(w.pocket.dims) - 1) * w.pocket.spacing
    out = []
    for _ in range(n):
        R = rand_rot(rng)
        t = centre + rng.normal(scale=spread, size=3)
        phi = rng.uniform(0, 2 * np.pi, size=R_n)
        out.append(np.concatenate([R.reshape(-1), t, phi]))
    return np.array(out)


def moved(state, comp, eps):
    """State moved by eps along generalised coordinate comp."""
    s = state.copy()
    if comp < 3:
        s[9 + comp] += eps
    elif comp < 6:
        w = np.zeros(3)
        w[comp - 3] = eps
        s[:9] = (rot_exp(w) @ s[:9].reshape(3, 3)).reshape(-1)
    else:
        s[12 + comp - 6] += eps
    return s


def test_gradient_matches_central_differences(tiny):
    w = tiny
    lig = w.ligands.ligand(0)
    rng = np.random.default_rng(21)
    st = states_for(w, lig, rng, 40)
    e, g, sc, _, face = oracle.pose_grad(lig, w.pocket, w.sampling, st)
    eps = 1e-6
    checked = 0
    for p in range(len(st)):
        if face[p] < 1e-3:  # an atom next to a cell face: the derivative jumps there
            continue
        plus = np.array([moved(st[p], c, eps) for c in range(g.shape[1])])
        minus = np.array([moved(st[p], c, -eps) for c in range(g.shape[1])])
        ep = oracle.pose_grad(lig, w.pocket, w.sampling, plus)[0]
        em = oracle.pose_grad(lig, w.pocket, w.sampling, minus)[0]
        fd = (ep - em) / (2 * eps)
        np.testing.assert_allclose(fd, g[p], rtol=0, atol=1e-6 * max(sc[p, 0], 1.0))
        checked += 1
    assert checked >= 30
    # the clash term is active in some of these states (its weight shows in E)
    w0 = dataclasses.replace(w.sampling, clash_weight=0.0)
    e0 = oracle.pose_grad(lig, w.pocket, w0, st)[0]
    assert np.sum(np.abs(e - e0) > 1e-6) >= 5


def test_linear_map_closed_forms(tiny):
    """Maps G_t(u) = a.u + t (exact in FP32 at the nodes): every in-grid atom
    has gradient a/h, so F = N a/h; with no torsion applied a rigid pose has
    zero torque about t (sum of R (y_i - c) is zero)."""
    w = tiny
    lig = w.ligands.ligand(0)
    nx, ny, nz = w.pocket.dims
    a = np.array([0.25, -0.5, 0.125])
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    base = a[0] * xx + a[1] * yy + a[2] * zz
    maps = np.stack([base + t for t in range(w.pocket.n_types)]).astype(np.float32)
    pocket = dataclasses.replace(w.pocket, maps=maps)
    samp = dataclasses.replace(w.sampling, clash_weight=0.0)
    rng = np.random.default_rng(3)
    st = states_for(w, lig, rng, 10, spread=0.5)
    st[:, 12:] = 0.0
    e, g, sc, _, _ = oracle.pose_grad(lig, pocket, samp, st)
    n = len(lig[1])
    for p in range(len(st)):
        np.testing.assert_allclose(g[p, :3], n * a / w.pocket.spacing, rtol=1e-12)
        np.testing.assert_allclose(g[p, 3:6], 0.0, atol=1e-9 * sc[p, 4:7].max())


def test_clash_forces_have_no_net_force_or_torque(tiny):
    w = tiny
    lig = w.ligands.ligand(0)
    pocket = dataclasses.replace(w.pocket, maps=np.full_like(w.pocket.maps, 2.5))
    rng = np.random.default_rng(8)
    st = states_for(w, lig, rng, 30)
    e, g, sc, _, _ = oracle.pose_grad(lig, pocket, w.sampling, st)
    n = len(lig[1])
    clashing = e > 2.5 * n + 1e-9
    assert clashing.sum() >= 5
    np.testing.assert_allclose(g[:, :6], 0.0, atol=1e-12 * max(1.0, sc[:, 1:7].max()))
    assert np.abs(g[clashing, 6:]).max() > 1e-6  # the torsions do feel the clash


def test_descent_invariants(tiny):
    w = tiny
    lig = w.ligands.ligand(0)
    rng = np.random.default_rng(5)
    st = states_for(w, lig, rng, 24)
    r = oracle.refine(lig, w.pocket, w.sampling, st, 32, 0.1)
    assert np.all(r["e_out"] <= r["e_in"])
    assert np.mean(r["e_out"] < r["e_in"] - 1e-6) > 0.5
    for s in r["states"]:
        R = s[:9].reshape(3, 3)
        np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-12)
    # the reported energy is the energy of the reported state
    e_chk = oracle.pose_grad(lig, w.pocket, w.sampling, r["states"])[0]
    np.testing.assert_array_equal(e_chk, r["e_out"])
    # following its own decisions reproduces itself, with no disagreement
    r2 = oracle.refine(lig, w.pocket, w.sampling, st, 32, 0.1, follow=r["own_mask"])
    np.testing.assert_array_equal(r2["states"], r["states"])
    assert np.all(r2["n_disagree"] == 0)
    # flipping every decision is counted (a state whose trials all sit within
    # the near-tie band of its energy may count none)
    r3 = oracle.refine(lig, w.pocket, w.sampling, st, 32, 0.1, follow=~r["own_mask"])
    assert np.mean(r3["n_disagree"] >= 1) >= 0.8
    z = oracle.refine(lig, w.pocket, w.sampling, st, 0, 0.1)
    np.testing.assert_array_equal(z["states"], st)
    np.testing.assert_array_equal(z["e_out"], z["e_in"])


def test_descent_on_a_linear_map_follows_the_closed_form(tiny):
    """Rigid ligand, no clash, linear map: every step is accepted, the step
    size grows by 1.25 each time and t moves along -a/h by
    eta0 * sum_k 1.25^k."""
    w = tiny
    xyz, typ, bonds, rot = w.ligands.ligand(0)
    lig = (xyz, typ, bonds, np.zeros_like(rot))
    nx, ny, nz = w.pocket.dims
    a = np.array([0.25, -0.5, 0.125])
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    maps = np.stack([a[0] * xx + a[1] * yy + a[2] * zz + t for t in range(w.pocket.n_types)]).astype(np.float32)
    pocket = dataclasses.replace(w.pocket, maps=maps)
    samp = dataclasses.replace(w.sampling, clash_weight=0.0)
    rng = np.random.default_rng(2)
    st = states_for(w, lig, rng, 4, spread=0.3)
    M, eta0 = 6, 0.05
    r = oracle.refine(lig, pocket, samp, st, M, eta0)
    assert np.all(r["own_mask"] == (1 << M) - 1)
    shift = eta0 * sum(1.25 ** k for k in range(M)) * a / w.pocket.spacing
    np.testing.assert_allclose(r["states"][:, 9:12], st[:, 9:12] - shift, rtol=0, atol=1e-10)
    np.testing.assert_allclose(r["states"][:, :9], st[:, :9], atol=1e-12)
    n = len(typ)
    drop = n * np.dot(a / w.pocket.spacing, shift)
    np.testing.assert_allclose(r["e_in"] - r["e_out"], drop, rtol=1e-9)


def test_docked_state_reproduces_the_docking_score(tiny):
    w = tiny
    lig = w.ligands.ligand(0)
    starts = np.array([0, 5, 77, 300])
    rng = np.random.default_rng(1)
    R_n = int(np.sum(lig[3] != 0))
    tors = rng.integers(0, w.sampling.torsion_steps, size=(4, R_n))
    st = np.array([oracle.docked_state(w.sampling, w.pocket.anchors, s, t) for s, t in zip(starts, tors)])
    e = oracle.pose_grad(lig, w.pocket, w.sampling, st)[0]
    want = oracle.score_poses(lig, w.pocket, w.sampling, starts, tors)
    np.testing.assert_allclose(e, want, rtol=1e-12, atol=1e-12)


def test_state_coords_of_a_docked_state_are_the_docked_pose(tiny):
    w = tiny
    lig = w.ligands.ligand(0)
    R_n = int(np.sum(lig[3] != 0))
    rng = np.random.default_rng(12)
    starts = rng.integers(0, w.sampling.n_starts, size=5)
    tors = rng.integers(0, w.sampling.torsion_steps, size=(5, R_n))
    st = np.array([oracle.docked_state(w.sampling, w.pocket.anchors, s, t) for s, t in zip(starts, tors)])
    np.testing.assert_allclose(oracle.state_coords(lig, st),
                               oracle.pose_coords(lig, w.pocket.anchors, w.sampling, starts, tors),
                               rtol=0, atol=1e-12)

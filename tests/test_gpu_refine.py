"""Pose refinement on the GPU vs the FP64 oracle, through the C ABI.

Energy at seeded states: the docking score's rule (strict 1e-4 relative, or
the FP32 rounding proof with the GPU's own state coordinates from
ligate_state_coords, tests/parity.py).  Generalised gradient: within 2e-4 of
the sum of absolute term values of each component (a gradient component is
a sum of signed per-atom torques and forces that cancel, so its rounding is
measured against that sum); states with an atom within 1e-4 grid units of a
cell face are left out of the gradient check (the trilinear derivative
jumps there, and FP32 and FP64 may sit in different cells).  One descent iteration: the trial state and decision equal
the oracle's.  Several iterations: the oracle replays the GPU's accept
decisions and flags any that contradict its own beyond a near-tie; the GPU's
final energy must be the oracle's energy of the GPU's final state, and never
above the starting energy.  The descent is chaotic past a few iterations (a
1e-7 relative change of the start parts the oracle from itself), so the
replay is held to 97% agreement over 8 iterations and 32 iterations to the
oracle's outcome in distribution."""
import numpy as np
import pytest

import oracle
from paper_2304_09953_gb300 import docking as D
from paper_2304_09953_gb300 import native as N
from tests.parity import Geometry, Stats, check_state_energies

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def rand_rot(rng):
    q = rng.normal(size=4)
    return oracle.quat_to_matrix(q / np.linalg.norm(q))


def seeded_states(w, idx, rng, per_lig, spread=1.0):
    """FP64 state rows per (ligand, copy) and their FP32 device records."""
    centre = np.asarray(w.pocket.origin) + 0.5 * (np.array(w.pocket.dims) - 1) * w.pocket.spacing
    rows, lig = [], []
    for li in idx:
        R_n = int(w.ligands.n_rot[li])
        for _ in range(per_lig):
            R = rand_rot(rng)
            t = centre + rng.normal(scale=spread, size=3)
            phi = rng.uniform(0, 2 * np.pi, size=R_n)
            rows.append((R, t, phi))
            lig.append(li)
    rec = np.zeros(len(rows), N.STATE_DTYPE)
    for k, (R, t, phi) in enumerate(rows):
        rec[k]["rot"] = R.reshape(-1)
        rec[k]["trans"] = t
        rec[k]["tors"][:len(phi)] = phi
    # the oracle evaluates exactly the FP32 values the GPU receives
    st64 = [np.concatenate([rec[k]["rot"].astype(np.float64), rec[k]["trans"].astype(np.float64),
                            rec[k]["tors"][:len(rows[k][2])].astype(np.float64)]) for k in range(len(rows))]
    return np.array(lig, np.int32), rec, st64


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.uint8).copy()).cuda()


def handles(w):
    ph = D.PocketHandle(w.pocket)
    bh = D.BatchHandle(w.ligands)
    s = N.make_sampling(w.sampling, N.LIGATE_FP32, N.LIGATE_LAYOUT_PLAIN, False, None)
    return ph, bh, s


@pytest.mark.parametrize("name", ["tiny", "batched_small"])
def test_energy_and_gradient_match_oracle(name, request):
    w = request.getfixturevalue(name)
    rng = np.random.default_rng(31)
    idx = np.arange(w.ligands.n)
    lig, rec, st64 = seeded_states(w, idx, rng, 64 if name == "tiny" else 6)
    ph, bh, s = handles(w)
    n = len(lig)
    e = torch.zeros(n, dtype=torch.float32, device="cuda")
    g = torch.zeros((n, N.LIGATE_GRAD_DIM), dtype=torch.float32, device="cuda")
    N.ligate_pose_gradient(ph.h, bh.h, s, n, torch.from_numpy(lig).cuda(), to_dev(rec), e, g)
    e, g = e.cpu().numpy(), g.cpu().numpy()
    checked = 0
    st = Stats()
    geo = Geometry(w.pocket)
    for li in np.unique(lig):
        sel = np.nonzero(lig == li)[0]
        R_n = int(w.ligands.n_rot[li])
        e64, g64, sc, _, face = oracle.pose_grad(w.ligands.ligand(li), w.pocket, w.sampling,
                                                 np.array([st64[k] for k in sel]))
        check_state_energies(geo, w.ligands.ligand(li), w.pocket, w.sampling, rec[sel], [st64[k] for k in sel],
                             e[sel], e64, st)
        for m, k in enumerate(sel):
            if face[m] < 1e-4:
                continue
            tol = 2e-4 * np.maximum(sc[m, 1:], 1.0)
            np.testing.assert_array_less(np.abs(g[k, :6 + R_n] - g64[m]), tol)
            assert np.all(g[k, 6 + R_n:] == 0)
            checked += 1
    print(st.line())
    assert checked >= 0.9 * n


def test_descent_matches_oracle_replay(batched_small):
    """8 iterations: the horizon over which the descent is not yet chaotic
    (the oracle perturbed by 1e-7 relative replays itself without a single
    disagreement at 8 iterations, but in 5 of 128 poses at 16 and 43 at 32)."""
    w = batched_small
    rng = np.random.default_rng(32)
    idx = np.arange(0, w.ligands.n, 2)
    lig, rec, st64 = seeded_states(w, idx, rng, 4)
    ph, bh, s = handles(w)
    n = len(lig)
    out = torch.zeros(n * N.REFINED_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    iters, eta0 = 8, 0.1
    N.ligate_refine_states(ph.h, bh.h, s, n, torch.from_numpy(lig).cuda(), to_dev(rec), iters, eta0, out)
    r = out.cpu().numpy().view(N.REFINED_DTYPE)
    assert np.all(r["ligand"] == lig)
    assert np.all(r["score"] <= r["score_in"])
    assert np.mean(r["accepted"] != 0) > 0.9
    agree, total, close, same_e = 0, 0, 0, 0
    st = Stats()
    geo = Geometry(w.pocket)
    for li in np.unique(lig):
        sel = np.nonzero(lig == li)[0]
        R_n = int(w.ligands.n_rot[li])
        L = w.ligands.ligand(li)
        init = np.array([st64[k] for k in sel])
        rep = oracle.refine(L, w.pocket, w.sampling, init, iters, eta0, follow=r["accepted"][sel])
        fin = np.array([np.concatenate([r[k]["state"]["rot"], r[k]["state"]["trans"],
                                        r[k]["state"]["tors"][:R_n]]).astype(np.float64) for k in sel])
        e_fin, _, sc_fin, _, _ = oracle.pose_grad(L, w.pocket, w.sampling, fin)
        e0, _, sc0, _, _ = oracle.pose_grad(L, w.pocket, w.sampling, init)
        np.testing.assert_array_equal(e0, rep["e_in"])
        check_state_energies(geo, L, w.pocket, w.sampling, rec[sel], list(init), r[sel]["score_in"], e0, st)
        # the reported energy is the energy of the reported state
        check_state_energies(geo, L, w.pocket, w.sampling, r[sel]["state"], list(fin), r[sel]["score"], e_fin, st)
        for m, k in enumerate(sel):
            total += 1
            R = fin[m, :9].reshape(3, 3)
            np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-5)
            if rep["n_disagree"][m] == 0:
                agree += 1
                same_e += abs(r[k]["score"] - rep["e_out"][m]) <= 1e-3 * max(rep["scale"][m], 1.0)
                close += np.max(np.abs(fin[m, 9:12] - rep["states"][m, 9:12])) <= 2e-3
    print(st.line())
    assert agree >= 0.97 * total, (agree, total)
    # same decisions, but a step whose gradient was taken on either side of a
    # cell face (or of the grid's edge) moves the path by more than rounding
    assert same_e >= 0.95 * agree and close >= 0.9 * agree, (same_e, close, agree)


def test_long_descent_statistics_match_oracle(batched_small):
    """32 iterations, past the chaotic horizon: paths may part, so the GPU is
    held to the oracle's outcome in distribution (mean energy drop within
    15%, same fraction of improved poses within 0.05), and per pose to the
    invariants (monotone; energy = oracle energy of the returned state)."""
    w = batched_small
    rng = np.random.default_rng(34)
    idx = np.arange(w.ligands.n)
    lig, rec, st64 = seeded_states(w, idx, rng, 4)
    ph, bh, s = handles(w)
    n = len(lig)
    out = torch.zeros(n * N.REFINED_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    N.ligate_refine_states(ph.h, bh.h, s, n, torch.from_numpy(lig).cuda(), to_dev(rec), 32, 0.1, out)
    r = out.cpu().numpy().view(N.REFINED_DTYPE)
    drop_gpu, drop_or = np.zeros(n), np.zeros(n)
    for li in np.unique(lig):
        sel = np.nonzero(lig == li)[0]
        R_n = int(w.ligands.n_rot[li])
        L = w.ligands.ligand(li)
        own = oracle.refine(L, w.pocket, w.sampling, np.array([st64[k] for k in sel]), 32, 0.1)
        fin = np.array([np.concatenate([r[k]["state"]["rot"], r[k]["state"]["trans"],
                                        r[k]["state"]["tors"][:R_n]]).astype(np.float64) for k in sel])
        e_fin, _, sc_fin, _, _ = oracle.pose_grad(L, w.pocket, w.sampling, fin)
        check_state_energies(Geometry(w.pocket), L, w.pocket, w.sampling, r[sel]["state"], list(fin),
                             r[sel]["score"], e_fin)
        for m, k in enumerate(sel):
            assert r[k]["score"] <= r[k]["score_in"]
            drop_gpu[k] = r[k]["score_in"] - r[k]["score"]
            drop_or[k] = own["e_in"][m] - own["e_out"][m]
    print("mean energy drop over 32 iterations: GPU %.4f, oracle %.4f" % (drop_gpu.mean(), drop_or.mean()))
    assert abs(drop_gpu.mean() - drop_or.mean()) <= 0.15 * drop_or.mean()
    assert abs(np.mean(drop_gpu > 1e-6) - np.mean(drop_or > 1e-6)) <= 0.05


def test_one_descent_step_matches_oracle(batched_small):
    """A single iteration depends only on the starting gradient: the trial
    state and the decision match the oracle's for every state away from a
    cell face (decisions up to near-ties)."""
    w = batched_small
    rng = np.random.default_rng(33)
    idx = np.arange(w.ligands.n)
    lig, rec, st64 = seeded_states(w, idx, rng, 4)
    ph, bh, s = handles(w)
    n = len(lig)
    out = torch.zeros(n * N.REFINED_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    for eta0 in (0.02, 0.1):
        N.ligate_refine_states(ph.h, bh.h, s, n, torch.from_numpy(lig).cuda(), to_dev(rec), 1, eta0, out)
        r = out.cpu().numpy().view(N.REFINED_DTYPE)
        checked = 0
        for li in np.unique(lig):
            sel = np.nonzero(lig == li)[0]
            R_n = int(w.ligands.n_rot[li])
            L = w.ligands.ligand(li)
            init = np.array([st64[k] for k in sel])
            face = oracle.pose_grad(L, w.pocket, w.sampling, init)[4]
            own = oracle.refine(L, w.pocket, w.sampling, init, 1, eta0)
            trial = oracle.refine(L, w.pocket, w.sampling, init, 1, eta0, follow=np.ones(len(sel), np.uint32))
            for m, k in enumerate(sel):
                if face[m] < 1e-4:
                    continue
                checked += 1
                acc = int(r[k]["accepted"]) & 1
                if acc != int(own["own_mask"][m]):
                    gap = abs(trial["e_out"][m] - own["e_in"][m])
                    assert gap <= 1e-4 * max(trial["scale"][m], 1.0), (li, k, gap)
                want = trial["states"][m] if acc else init[m]
                got = np.concatenate([r[k]["state"]["rot"], r[k]["state"]["trans"],
                                      r[k]["state"]["tors"][:R_n]]).astype(np.float64)
                np.testing.assert_allclose(got[:9], want[:9], atol=2e-6)
                np.testing.assert_allclose(got[9:12], want[9:12], atol=2e-5)
                np.testing.assert_allclose(got[12:], want[12:], atol=2e-5)
        assert checked >= 0.9 * n


@pytest.mark.parametrize("mode", ["fp32", "bf16"])
def test_plan_refine_starts_from_the_docked_poses(tiny, mode):
    w = tiny
    ph = D.PocketHandle(w.pocket)
    bh = D.BatchHandle(w.ligands)
    pl = D.Plan(ph, bh, w.sampling, mode=mode)
    res = pl.result()
    ref = pl.refine(iterations=32, eta0=0.1)
    zero = pl.refine(iterations=0, eta0=0.1)
    L = w.ligands.ligand(0)
    geo, stt = Geometry(w.pocket), Stats()
    K = res.shape[1]
    assert np.all(ref["ligand"] == 0)
    for j in range(K):
        sid = int(res[0, j]["start_id"])
        if sid < 0:
            continue
        R_n = int(w.ligands.n_rot[0])
        tors = res[0, j]["tors"][:R_n].astype(np.int64)
        st = oracle.docked_state(w.sampling, w.pocket.anchors, sid, tors)
        # zero iterations: the docked state itself
        z = zero[0, j]
        # starting energy = FP32-map score of the docked pose (the record's
        # FP32 state, evaluated exactly)
        z64 = np.concatenate([z["state"]["rot"], z["state"]["trans"], z["state"]["tors"][:R_n]]).astype(np.float64)
        e64, _, sc, _, _ = oracle.pose_grad(L, w.pocket, w.sampling, z64[None])
        check_state_energies(geo, L, w.pocket, w.sampling, z["state"][None], [z64], [ref[0, j]["score_in"]], e64, stt)
        assert ref[0, j]["score"] <= ref[0, j]["score_in"]
        assert z["accepted"] == 0 and z["score"] == z["score_in"]
        np.testing.assert_allclose(z["state"]["trans"], st[9:12], atol=1e-4)
        np.testing.assert_allclose(z["state"]["rot"], st[:9], atol=1e-5)
        np.testing.assert_allclose(z["state"]["tors"][:R_n], st[12:], atol=1e-6)
        fin = np.concatenate([ref[0, j]["state"]["rot"], ref[0, j]["state"]["trans"],
                              ref[0, j]["state"]["tors"][:R_n]]).astype(np.float64)
        e_fin, _, sc_fin, _, _ = oracle.pose_grad(L, w.pocket, w.sampling, fin[None])
        check_state_energies(geo, L, w.pocket, w.sampling, ref[0, j]["state"][None], [fin], [ref[0, j]["score"]],
                             e_fin, stt)
    print(stt.line())
    pl.close()


def test_refine_argument_errors(tiny):
    w = tiny
    ph, bh, s = handles(w)
    lig = torch.zeros(1, dtype=torch.int32, device="cuda")
    rec = to_dev(np.zeros(1, N.STATE_DTYPE))
    out = torch.zeros(N.REFINED_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    for iters, eta in [(33, 0.1), (-1, 0.1), (4, 0.0), (4, float("nan"))]:
        with pytest.raises(RuntimeError):
            N.ligate_refine_states(ph.h, bh.h, s, 1, lig, rec, iters, eta, out)
    N.ligate_refine_states(ph.h, bh.h, s, 0, None, None, 4, 0.1, None)  # empty is fine


def test_largest_ligands_refine_and_rescore():
    """128 atoms and 16 rotatable bonds: gradient, one refinement step and
    exact rescoring of states against the oracle at the library limits."""
    from paper_2304_09953_gb300.workload import Pocket, Sampling, make_ligands, make_workload
    w = make_workload("tiny", n_ligands=0)
    big = make_ligands(5, np.array([128, 100], np.int32), np.array([16, 16], np.int32), 6)
    rng = np.random.default_rng(0)
    maps = (np.zeros((6, 80, 80, 80), np.float32) + w.pocket.maps.mean()
            + rng.normal(size=(6, 80, 80, 80)).astype(np.float32)).astype(np.float32)
    rec_xyz = rng.uniform(0, 39.5, size=(500, 3))
    P = Pocket(maps, np.zeros(3), 0.5, np.array([[19.75, 19.75, 19.75]], np.float32),
               rec_xyz, rng.integers(0, 6, size=500).astype(np.int32),
               np.linspace(1.5, 2.0, 6), np.linspace(0.1, 0.3, 6))
    samp = Sampling(w.sampling.quats[:4], 1, 4, 4)

    class W:
        pocket, ligands, sampling = P, big, samp

    lig, rec, st64 = seeded_states(W, np.arange(2), rng, 8, spread=2.0)
    ph = D.PocketHandle(P)
    bh = D.BatchHandle(big)
    s = N.make_sampling(samp, N.LIGATE_FP32, N.LIGATE_LAYOUT_PLAIN, False, None)
    n = len(lig)
    e = torch.zeros(n, dtype=torch.float32, device="cuda")
    g = torch.zeros((n, N.LIGATE_GRAD_DIM), dtype=torch.float32, device="cuda")
    N.ligate_pose_gradient(ph.h, bh.h, s, n, torch.from_numpy(lig).cuda(), to_dev(rec), e, g)
    out = torch.zeros(n * N.RESCORED_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    N.ligate_rescore_states(ph.h, bh.h, s, n, torch.from_numpy(lig).cuda(), to_dev(rec), out)
    e, g = e.cpu().numpy(), g.cpu().numpy()
    r = out.cpu().numpy().view(N.RESCORED_DTYPE)
    for li in range(2):
        sel = np.nonzero(lig == li)[0]
        L = big.ligand(li)
        init = np.array([st64[k] for k in sel])
        e64, g64, sc, _, face = oracle.pose_grad(L, P, samp, init)
        o = oracle.rescore_coords(L, P, samp, P.receptor(), oracle.state_coords(L, init))
        geo = Geometry(P)
        check_state_energies(geo, L, P, samp, rec[sel], list(init), e[sel], e64)
        check_state_energies(geo, L, P, samp, rec[sel], list(init), r[sel]["e_inter"], o["e_inter"],
                             value=lambda x: oracle.rescore_coords(L, P, samp, P.receptor(), x)["e_inter"])
        for m, k in enumerate(sel):
            if face[m] >= 1e-4:
                np.testing.assert_array_less(np.abs(g[k, :22] - g64[m]), 2e-4 * np.maximum(sc[m, 1:], 1.0))


def test_state_coords_are_the_exact_states_within_the_fp32_envelope(batched_small):
    """ligate_state_coords on seeded states: every atom (input order, Angstrom)
    within the FP32 envelope of the oracle's FP64 coordinates of the same
    FP32 state values; an out-of-range ligand gives NaN rows."""
    from tests.parity import coord_envelope
    w = batched_small
    rng = np.random.default_rng(41)
    lig, rec, st64 = seeded_states(w, np.arange(w.ligands.n), rng, 4)
    lig[-1] = w.ligands.n
    ph, bh, s = handles(w)
    n = len(lig)
    out = torch.full((n * 128 * 3,), 7.0, dtype=torch.float32, device="cuda")
    N.ligate_state_coords(ph.h, bh.h, s, n, torch.from_numpy(lig).cuda(), to_dev(rec), out)
    x = out.cpu().numpy().reshape(n, 128, 3).astype(np.float64)
    assert np.all(np.isnan(x[-1]))
    org, h = np.asarray(w.pocket.origin), w.pocket.spacing
    worst = 0.0
    for k in range(n - 1):
        L = w.ligands.ligand(int(lig[k]))
        na, R = len(L[0]), int(w.ligands.n_rot[lig[k]])
        assert np.all(x[k, na:] == 7.0)
        x64 = oracle.state_coords(L, st64[k][None])[0]
        err = float(np.max(np.abs(x[k, :na] - x64))) / h
        env = coord_envelope((x64 - org) / h, R)
        worst = max(worst, err / env)
        assert err <= env, (k, err, env)
    print(f"largest state coordinate error: {worst:.2f} of the envelope")

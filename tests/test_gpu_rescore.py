"""Exact rescoring and the pose filter on the GPU vs the FP64 oracle.

Explicit poses (seeded starts and torsion steps) and continuous states:
receptor and clash terms by the docking score's parity rules (strict 1e-4
relative, else exact at the GPU's own coordinates -- ligate_pose_coords,
ligate_state_coords -- with the coordinates inside the FP32 envelope); the
filter counts equal the oracle's at the GPU's coordinates except for an atom
on its threshold (a receptor sum within the bar of the cap, a coordinate on
a box face).  The plan path gives the same values as the explicit path for
the plan's own poses, and the per-ligand choice of the best passing pose
follows from them."""
import numpy as np
import pytest

import oracle
from paper_2304_09953_gb300 import docking as D
from paper_2304_09953_gb300 import native as N
from tests.parity import (REL, U32, Geometry, Stats, check_state_energies, coord_envelope, features_check,
                          rescore_check)

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def explicit(w, n_per, seed):
    rng = np.random.default_rng(seed)
    lig, sid, tors = [], [], []
    for li in range(w.ligands.n):
        R_n = int(w.ligands.n_rot[li])
        for _ in range(n_per):
            lig.append(li)
            sid.append(int(rng.integers(0, w.sampling.n_starts)))
            t = np.zeros(16, np.uint8)
            t[:R_n] = rng.integers(0, w.sampling.torsion_steps, size=R_n)
            tors.append(t)
    return np.array(lig, np.int32), np.array(sid, np.int32), np.array(tors, np.uint8)


@pytest.mark.parametrize("name", ["tiny", "batched_small"])
def test_rescore_matches_oracle(name, request):
    w = request.getfixturevalue(name)
    lig, sid, tors = explicit(w, 256 if name == "tiny" else 12, 7)
    ph = D.PocketHandle(w.pocket)
    bh = D.BatchHandle(w.ligands)
    s = N.make_sampling(w.sampling)
    n = len(lig)
    out = torch.zeros(n * N.RESCORED_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    N.ligate_rescore_poses(ph.h, bh.h, s, n, torch.from_numpy(lig).cuda(), torch.from_numpy(sid).cuda(),
                           torch.from_numpy(tors).cuda(), out)
    r = out.cpu().numpy().view(N.RESCORED_DTYPE)
    geo = Geometry(w.pocket)
    st = Stats()
    diff_exact = diff_gpu = 0
    for li in np.unique(lig):
        sel = np.nonzero(lig == li)[0]
        R_n = int(w.ligands.n_rot[li])
        info = rescore_check(geo, w.ligands.ligand(li), w.pocket, w.sampling, sid[sel], tors[sel, :R_n],
                             r[sel], st)
        diff_exact += info["flag_diff_vs_exact"]
        diff_gpu += info["flag_diff_vs_gpu_coords"]
        assert np.allclose(r[sel]["energy"], r[sel]["e_inter"] + r[sel]["e_clash"], rtol=1e-6, atol=1e-5)
    print(f"{st.line()}; filter counts differing from the oracle at the exact poses {diff_exact}, "
          f"at the GPU's coordinates {diff_gpu} (all on a threshold) of {n}")
    assert np.any(r["n_capped"] > 0)  # random poses hit the receptor


def test_plan_rescore_equals_explicit_and_selects_best(batched_small):
    w = batched_small
    ph = D.PocketHandle(w.pocket)
    bh = D.BatchHandle(w.ligands)
    pl = D.Plan(ph, bh, w.sampling, mode="bf16")
    res = pl.result()
    rs = pl.rescore_exact()
    n, K = res.shape
    lig = np.repeat(np.arange(n, dtype=np.int32), K)
    sid = res["start_id"].reshape(-1).astype(np.int32)
    tors = res["tors"].reshape(-1, 16).astype(np.uint8)
    live = sid >= 0
    out = torch.zeros(int(live.sum()) * N.RESCORED_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    N.ligate_rescore_poses(ph.h, bh.h, pl.s, int(live.sum()), torch.from_numpy(lig[live]).cuda(),
                           torch.from_numpy(sid[live]).cuda(), torch.from_numpy(tors[live]).cuda(), out)
    ex = out.cpu().numpy().view(N.RESCORED_DTYPE)
    flat = rs.reshape(-1)
    np.testing.assert_array_equal(flat[live], ex)
    assert np.all(np.isinf(flat[~live]["energy"]))
    idx, best = pl.best_passing(rs)
    # the interpolated maps smooth the steep wall of the pair potential, so
    # many docked poses touch it (a capped atom); a good share still passes
    assert np.mean(idx >= 0) > 0.25
    for i in range(n):
        ok = rs[i]["pass"] == 1
        if ok.any():
            assert best[i] == rs[i]["energy"][ok].min() and rs[i][idx[i]]["pass"] == 1
        else:
            assert idx[i] == -1
    pl.close()


def test_rescore_needs_a_receptor(tiny):
    import dataclasses
    w = tiny
    bare = dataclasses.replace(w.pocket, receptor_xyz=None)
    ph = D.PocketHandle(bare)
    bh = D.BatchHandle(w.ligands)
    s = N.make_sampling(w.sampling)
    z = torch.zeros(1, dtype=torch.int32, device="cuda")
    t = torch.zeros(16, dtype=torch.uint8, device="cuda")
    out = torch.zeros(N.RESCORED_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    with pytest.raises(RuntimeError):
        N.ligate_rescore_poses(ph.h, bh.h, s, 1, z, z, t, out)


@pytest.mark.parametrize("name", ["tiny", "batched_small"])
def test_pose_features_match_oracle(name, request):
    """Histogram counts equal the oracle's at the GPU's coordinates (FP32 bin
    decisions on both sides) except for an atom whose value sits on a bin
    edge; means, score and clash entries by the score rules; the plan path
    equals the explicit path (test_empty_slots and the selector test)."""
    w = request.getfixturevalue(name)
    lig, sid, tors = explicit(w, 128 if name == "tiny" else 8, 11)
    ph = D.PocketHandle(w.pocket)
    bh = D.BatchHandle(w.ligands)
    s = N.make_sampling(w.sampling)
    n = len(lig)
    out = torch.zeros((n, 256), dtype=torch.float32, device="cuda")
    N.ligate_pose_features(ph.h, bh.h, s, n, torch.from_numpy(lig).cuda(), torch.from_numpy(sid).cuda(),
                           torch.from_numpy(tors).cuda(), out)
    f = out.cpu().numpy().astype(np.float64)
    geo = Geometry(w.pocket)
    moved = 0
    for li in np.unique(lig):
        sel = np.nonzero(lig == li)[0]
        R_n = int(w.ligands.n_rot[li])
        moved += features_check(geo, w.ligands.ligand(li), w.pocket, w.sampling, sid[sel], tors[sel, :R_n],
                                f[sel])
    print(f"histograms differing from the oracle at the GPU's coordinates: {moved} of {n} (bin-edge atoms)")


def test_learned_selector_beats_docking_rank(workload_factory):
    """Train the network on pose features of 6,000 seeded training ligands
    (labels from the exact rescoring kernel) and select on 2,000 library
    ligands: the kept pose passes the filter more often than the best-docked
    pose does, and is the exact-best passing pose at least as often."""
    from paper_2304_09953_gb300 import selector as SEL
    w = workload_factory("batched", n_ligands=2000)
    tw = workload_factory("learned_train", n_ligands=6000)
    assert np.array_equal(tw.pocket.maps, w.pocket.maps)
    ph = D.PocketHandle(w.pocket)
    K = w.sampling.top_k

    def features_and_truth(lig_w):
        bh = D.BatchHandle(lig_w.ligands)
        pl = D.Plan(ph, bh, lig_w.sampling, mode="bf16")
        poses = pl.result()
        n = lig_w.ligands.n * K
        f = torch.empty((n, 256), dtype=torch.float32, device="cuda")
        N.ligate_plan_pose_features(pl.h, f)
        r = torch.empty(n * N.RESCORED_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        N.ligate_plan_rescore(pl.h, r)
        best_idx, _ = pl.best_passing(r)
        out = f, r.cpu().numpy().view(N.RESCORED_DTYPE), poses, best_idx
        pl.close()
        bh.close()
        return out

    ftr, rtr, _, _ = features_and_truth(tw)
    live = np.isfinite(rtr["energy"])
    idx = torch.from_numpy(np.nonzero(live)[0]).cuda()
    net = N.ligate_surrogate_create(None, 5)
    try:
        N.ligate_surrogate_train(net, ftr[idx].contiguous(), SEL.labels(rtr[live]).contiguous(),
                                 len(idx), 10, 1024, 1e-3, 5)
        f, r, poses, best_idx = features_and_truth(w)
        pred = torch.empty(f.shape[0], dtype=torch.float32, device="cuda")
        N.ligate_surrogate_predict(net, f, f.shape[0], pred)
        p = pred.cpu().numpy().reshape(-1, K)
    finally:
        N.ligate_surrogate_destroy(net)
    ex = r.reshape(-1, K)
    has = best_idx >= 0
    rows = np.arange(len(ex))
    pick = SEL.select(p, poses)
    rank0 = np.zeros(len(ex), np.int64)
    pass_sel = np.mean(ex["pass"][rows, pick][has] == 1)
    pass_r0 = np.mean(ex["pass"][rows, rank0][has] == 1)
    top_sel = np.mean(pick[has] == best_idx[has])
    top_r0 = np.mean(rank0[has] == best_idx[has])
    print("passes: selector %.3f rank-0 %.3f; exact-best: selector %.3f rank-0 %.3f"
          % (pass_sel, pass_r0, top_sel, top_r0))
    assert pass_sel >= pass_r0 + 0.03
    assert top_sel >= top_r0


def test_rescore_states_matches_oracle_and_refined_plan_path(batched_small):
    """Continuous states: seeded states vs the oracle; and the refined records
    of a plan rescore exactly as their states do through the explicit path."""
    from tests.test_gpu_refine import seeded_states, to_dev
    w = batched_small
    rng = np.random.default_rng(17)
    lig, rec, st64 = seeded_states(w, np.arange(w.ligands.n), rng, 4, spread=1.0)
    ph = D.PocketHandle(w.pocket)
    bh = D.BatchHandle(w.ligands)
    s = N.make_sampling(w.sampling)
    n = len(lig)
    out = torch.zeros(n * N.RESCORED_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    N.ligate_rescore_states(ph.h, bh.h, s, n, torch.from_numpy(lig).cuda(), to_dev(rec), out)
    r = out.cpu().numpy().view(N.RESCORED_DTYPE)
    same = 0
    org, h = np.asarray(w.pocket.origin), w.pocket.spacing
    rcp = w.pocket.receptor()
    geo, stt = Geometry(w.pocket), Stats()
    for li in np.unique(lig):
        sel = np.nonzero(lig == li)[0]
        L = w.ligands.ligand(li)
        R_n = int(np.sum(L[3] != 0))
        x = oracle.state_coords(L, np.array([st64[k] for k in sel]))
        o = oracle.rescore_coords(L, w.pocket, w.sampling, rcp, x)
        for key in ("e_inter", "e_clash"):
            check_state_energies(geo, L, w.pocket, w.sampling, rec[sel], [st64[k] for k in sel], r[sel][key],
                                 o[key], stt,
                                 value=lambda x, key=key: oracle.rescore_coords(L, w.pocket, w.sampling, rcp, x)[key])
        for m, k in enumerate(sel):
            ok = r[k]["n_outside"] == o["n_outside"][m] and r[k]["n_capped"] == o["n_capped"][m]
            same += ok
            if not ok:
                # without the GPU's coordinates of a state, a flag difference
                # must come from an atom that the coordinate envelope can move
                # across its threshold: the face distance within the envelope,
                # or the receptor sum crossing the cap somewhere in the box of
                # that half-width around the atom (a corner of it, first order)
                env = coord_envelope((x[m] - org) / h, R_n)
                s0, mg, fc = oracle.rescore_atoms(L, w.pocket, rcp, x[m:m + 1])
                near = np.abs(fc[0]) <= env
                d = env * h
                lo, hi = s0[0].copy(), s0[0].copy()
                for ax in range(3):
                    for sg in (-1.0, 1.0):
                        xp = x[m:m + 1].copy()
                        xp[0, :, ax] += sg * d
                        sp, _, _ = oracle.rescore_atoms(L, w.pocket, rcp, xp)
                        lo = np.minimum(lo, s0[0] - 3 * np.abs(sp[0] - s0[0]))
                        hi = np.maximum(hi, s0[0] + 3 * np.abs(sp[0] - s0[0]))
                cross = (lo - REL * np.maximum(mg[0], 1) <= w.pocket.cap) & \
                        (hi + REL * np.maximum(mg[0], 1) >= w.pocket.cap)
                dcap = abs(int(r[k]["n_capped"]) - int(o["n_capped"][m]))
                dout = abs(int(r[k]["n_outside"]) - int(o["n_outside"][m]))
                assert dcap <= int(cross.sum()) and dout <= int(near.sum()), (k, dcap, dout)
    print(f"{stt.line()}; states with filter counts equal to the oracle's: {same} of {n}")
    # refined plan records vs their states through the explicit path
    pl = D.Plan(ph, bh, w.sampling, mode="bf16")
    pl.run()
    K = w.sampling.top_k
    rbuf = torch.empty(w.ligands.n * K * N.REFINED_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    N.ligate_plan_refine(pl.h, 16, 0.1, rbuf)
    a = torch.empty(w.ligands.n * K * N.RESCORED_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    N.ligate_plan_rescore_refined(pl.h, rbuf, a)
    torch.cuda.synchronize()
    refined = rbuf.cpu().numpy().view(N.REFINED_DTYPE)
    via_plan = a.cpu().numpy().view(N.RESCORED_DTYPE)
    live = np.isfinite(refined["score_in"])
    st = np.ascontiguousarray(refined["state"][live])
    b = torch.empty(int(live.sum()) * N.RESCORED_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    N.ligate_rescore_states(ph.h, bh.h, pl.s, int(live.sum()),
                           torch.from_numpy(refined["ligand"][live].astype(np.int32)).cuda(), to_dev(st), b)
    np.testing.assert_array_equal(via_plan[live], b.cpu().numpy().view(N.RESCORED_DTYPE))
    assert np.all(np.isinf(via_plan[~live]["energy"]))
    pl.close()


def test_empty_slots_pass_through_every_stage(tiny):
    """Two starts and top-4: slots 2 and 3 of the plan's output are empty;
    refinement, exact rescoring (of docked and of refined poses) and the
    selector features all mark them empty and handle the two real poses."""
    import dataclasses
    w = tiny
    samp = dataclasses.replace(w.sampling, quats=w.sampling.quats[:1], n_anchor=2, top_k=4)
    ph = D.PocketHandle(w.pocket)
    bh = D.BatchHandle(w.ligands)
    pl = D.Plan(ph, bh, samp, mode="fp32")
    res = pl.result()
    assert np.all(res[0]["start_id"][:2] >= 0) and list(res[0]["start_id"][2:]) == [-1, -1]
    ref = pl.refine(iterations=8, eta0=0.1)
    assert np.all(np.isinf(ref[0, 2:]["score_in"])) and np.all(ref[0, 2:]["accepted"] == 0)
    assert np.all(np.isfinite(ref[0, :2]["score"]))
    rs = pl.rescore_exact()
    assert np.all(np.isinf(rs[0, 2:]["energy"])) and np.all(rs[0, 2:]["pass"] == 0)
    rbuf = torch.from_numpy(ref.reshape(-1).view(np.uint8).copy()).cuda()
    out = torch.empty(4 * N.RESCORED_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    N.ligate_plan_rescore_refined(pl.h, rbuf, out)
    torch.cuda.synchronize()
    rr = out.cpu().numpy().view(N.RESCORED_DTYPE)
    assert np.all(np.isinf(rr[2:]["energy"])) and np.all(np.isfinite(rr[:2]["energy"]))
    f = torch.empty((4, 256), dtype=torch.float32, device="cuda")
    N.ligate_plan_pose_features(pl.h, f)
    torch.cuda.synchronize()
    f = f.cpu().numpy()
    assert np.all(f[2:] == 0) and np.all(f[:2, 74] > 0)
    pl.close()

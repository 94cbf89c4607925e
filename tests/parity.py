"""GPU-vs-oracle comparison rules for the docking path.

Tolerance (the "1e-4 relative per-pose score" of the method's statement,
read as |E_gpu - E_64| <= 1e-4 * max(|E_64|, 1), the floor keeping scores
near zero meaningful).  A pose that misses this strict bar passes only with
a proof that the difference is FP32 rounding of the pose's coordinates:

  * arithmetic: the oracle's FP64 score evaluated AT THE GPU'S OWN FP32
    COORDINATES (ligate_pose_coords returns the geometry every kernel builds)
    equals the GPU score within the strict bar, so the kernels' map reads,
    interpolation, clash sums and accumulation are exact to that bar; and
  * geometry: every GPU coordinate lies within the FP32 construction
    envelope of the exact (FP64) pose, |u_gpu - u_64| <= (32 + 16 R) u X
    grid units, with u = 2^-24 the FP32 unit roundoff, X the largest
    grid-unit coordinate of the pose and R its rotatable-bond count.
    Each level of the construction (the rigid move, then each bond's
    rotation about an axis whose direction is itself rounded) adds a few
    u X, amplified by the ratio of the lever arm to the bond length; on
    6,400 poses of the 10,000-ligand library the largest measured error was
    53 u X (R = 11), the median 6 u X.

The greedy search may pick a different torsion step than FP64 where two
trials differ by less than the rounding of the coordinates, after which the
two paths continue from different poses.  The rules therefore check the GPU
along its own choice path:
  * path check: at every bond the GPU's step scores (FP64, other bonds as
    the GPU had them) within the strict bar of the best step; where it does
    not, the S trial poses at that bond are rebuilt by the GPU and scored
    exactly at those coordinates, and the GPU's step must be the best one
    there within the strict bar (its decision is right on the geometry it
    built), with every trial inside the coordinate envelope;
  * list check: a start in the oracle's top-K but not in the GPU's has its
    GPU path recomputed (a run over that start's orientation alone),
    path-checked, and its GPU score must not beat the GPU's K-th entry; a
    start in both lists with different torsion paths is covered by the
    GPU path check.
"""
from __future__ import annotations

import dataclasses

import numpy as np

import oracle

REL = 1e-4
U32 = 2.0 ** -24
ENV_BASE, ENV_PER_BOND = 32.0, 16.0


def tol(e):
    return REL * np.maximum(np.abs(e), 1.0)


def coord_envelope(u64, R):
    """FP32 construction envelope (grid units) of a pose's coordinates."""
    return (ENV_BASE + ENV_PER_BOND * R) * U32 * float(np.max(np.abs(u64)))


@dataclasses.dataclass
class Stats:
    """Counts of the rule each checked pose passed by, and the largest
    ratios seen (printed by the tests for the record)."""
    poses: int = 0
    strict: int = 0
    rounding: int = 0
    max_strict_ratio: float = 0.0
    max_arith_ratio: float = 0.0
    max_coord_ratio: float = 0.0   # coordinate error / envelope
    steps: int = 0
    steps_strict: int = 0
    steps_rounding: int = 0
    rerun_starts: int = 0

    def line(self):
        return (f"poses {self.poses}: strict {self.strict}, rounding proof {self.rounding} "
                f"(max |err|/tol {self.max_strict_ratio:.2f}, arithmetic at GPU coords "
                f"{self.max_arith_ratio:.3f} of tol, coordinates {self.max_coord_ratio:.2f} of envelope); "
                f"greedy steps {self.steps}: strict {self.steps_strict}, rounding proof {self.steps_rounding}; "
                f"re-run starts {self.rerun_starts}")


def _one_ligand(lig):
    from paper_2304_09953_gb300.workload import Ligands
    xyz, typ, bonds, rot = lig
    n, nb = len(xyz), len(bonds)
    return Ligands(np.array([0, n], np.int32), np.ascontiguousarray(xyz, np.float32),
                   np.ascontiguousarray(typ, np.uint8), np.array([0, nb], np.int32),
                   np.ascontiguousarray(bonds, np.int32).reshape(nb, 2), np.ascontiguousarray(rot, np.uint8),
                   np.array([int(np.sum(np.asarray(rot) != 0))], np.int32))


class Geometry:
    """The GPU's side of a pose: its FP32 coordinates (ligate_pose_coords)
    and its greedy path for a single start (a docking run over that start's
    orientation).  One pocket handle per pocket object."""

    _pockets = {}

    def __init__(self, pocket, mode="fp32"):
        from paper_2304_09953_gb300 import docking as D
        key = id(pocket)
        if key not in Geometry._pockets:
            Geometry._pockets[key] = (pocket, D.PocketHandle(pocket))
        self.pocket = pocket
        self.ph = Geometry._pockets[key][1]
        self.mode = mode
        self.org = np.asarray(pocket.origin, np.float64)
        self.h = float(pocket.spacing)

    def coords(self, lig, sampling, starts, tors):
        """GPU coordinates [n, n_atoms, 3] in grid units (FP32 values)."""
        import torch
        from paper_2304_09953_gb300 import docking as D
        from paper_2304_09953_gb300 import native as N
        starts = np.asarray(starts, np.int32).reshape(-1)
        n = len(starts)
        t = np.zeros((n, 16), np.uint8)
        tt = np.asarray(tors).reshape(n, -1)
        t[:, :tt.shape[1]] = tt
        bh = D.BatchHandle(_one_ligand(lig))
        s = N.make_sampling(sampling)
        out = torch.zeros(n * 128 * 3, dtype=torch.float32, device="cuda")
        N.ligate_pose_coords(self.ph.h, bh.h, s, n, torch.zeros(n, dtype=torch.int32, device="cuda"),
                             torch.from_numpy(starts).cuda(), torch.from_numpy(t).cuda(), out)
        bh.close()
        return out.cpu().numpy().reshape(n, 128, 3)[:, :len(lig[0])].astype(np.float64)

    def state_coords(self, lig, sampling, rec):
        """GPU coordinates [n, n_atoms, 3] in Angstrom (FP32 values) of
        continuous states (STATE_DTYPE records), as the refinement and the
        exact rescoring build them."""
        import torch
        from paper_2304_09953_gb300 import docking as D
        from paper_2304_09953_gb300 import native as N
        rec = np.ascontiguousarray(rec)
        n = len(rec)
        bh = D.BatchHandle(_one_ligand(lig))
        s = N.make_sampling(sampling)
        out = torch.zeros(n * 128 * 3, dtype=torch.float32, device="cuda")
        st = torch.from_numpy(rec.view(np.uint8).copy()).cuda()
        N.ligate_state_coords(self.ph.h, bh.h, s, n, torch.zeros(n, dtype=torch.int32, device="cuda"), st, out)
        bh.close()
        return out.cpu().numpy().reshape(n, 128, 3)[:, :len(lig[0])].astype(np.float64)

    def exact_coords(self, lig, sampling, starts, tors):
        """FP64 coordinates of the same poses, grid units."""
        x = oracle.pose_coords(lig, self.pocket.anchors, sampling, starts, np.asarray(tors, np.int32))
        return (x - self.org) / self.h

    def score_at(self, lig, sampling, u):
        """FP64 scores at grid-unit coordinate sets u [n, n_atoms, 3]."""
        return np.array([oracle.score_coords(lig, self.pocket, sampling, self.org + self.h * x) for x in u])

    def path_of(self, lig, sampling, start):
        """(score, tors[R]) the GPU finds for one start, from a run over
        orientation o with anchors 0..a (start (o, a) is the last of them)."""
        from paper_2304_09953_gb300 import docking as D
        o, a = divmod(int(start), int(sampling.n_anchor))
        samp = dataclasses.replace(sampling, quats=np.asarray(sampling.quats)[o:o + 1], n_anchor=a + 1,
                                   top_k=min(a + 1, 32))
        assert a + 1 <= 32, "re-run needs the start among the first 32 anchors"
        res = D.dock(self.pocket, _one_ligand(lig), samp, mode=self.mode)[0]
        j = int(np.nonzero(res["start_id"] == a)[0][0])
        R = int(np.sum(np.asarray(lig[3]) != 0))
        return float(res["score"][j]), res["tors"][j, :R].copy()


def rounding_proof(geo, lig, sampling, starts, tors, scores, stats=None):
    """Assert, for each pose, the two halves of the rounding proof."""
    R = int(np.sum(np.asarray(lig[3]) != 0))
    ug = geo.coords(lig, sampling, starts, tors)
    u64 = geo.exact_coords(lig, sampling, starts, tors)
    e_at = geo.score_at(lig, sampling, ug)
    scores = np.asarray(scores, np.float64)
    for j in range(len(scores)):
        ar = abs(scores[j] - e_at[j]) / tol(e_at[j])
        cerr = float(np.max(np.abs(ug[j] - u64[j])))
        cr = cerr / coord_envelope(u64[j], R)
        if stats is not None:
            stats.max_arith_ratio = max(stats.max_arith_ratio, float(ar))
            stats.max_coord_ratio = max(stats.max_coord_ratio, cr)
        assert ar <= 1.0, (f"GPU score {scores[j]} differs from the FP64 score at its own coordinates "
                           f"{e_at[j]} beyond the strict bar (start {starts[j]})")
        assert cr <= 1.0, f"GPU coordinates {cerr:.3e} grid units from the exact pose (start {starts[j]})"


def check_scores(geo, lig, pocket, sampling, starts, tors, scores, stats=None):
    """Reported pose scores: strict bar, else the rounding proof.  Returns
    the FP64 scores of the poses."""
    R = int(np.sum(np.asarray(lig[3]) != 0))
    starts = np.asarray(starts, np.int64)
    tors = np.asarray(tors)[:, :R].astype(np.int64)
    scores = np.asarray(scores, np.float64)
    e64 = oracle.score_poses(lig, pocket, sampling, starts, tors)
    ratio = np.abs(scores - e64) / tol(e64)
    bad = ratio > 1.0
    if stats is not None:
        stats.poses += len(scores)
        stats.strict += int((~bad).sum())
        stats.rounding += int(bad.sum())
        stats.max_strict_ratio = max(stats.max_strict_ratio, float(ratio.max(initial=0.0)))
    if bad.any():
        rounding_proof(geo, lig, sampling, starts[bad], tors[bad], scores[bad], stats)
    return e64


def path_check(geo, lig, pocket, sampling, starts, tors, scores, stats=None):
    """Scores and every greedy step of GPU poses (start, tors)."""
    R = int(np.sum(np.asarray(lig[3]) != 0))
    S = sampling.torsion_steps
    starts = np.asarray(starts, np.int64)
    tors = np.asarray(tors)[:, :R].astype(np.int64)
    e64 = check_scores(geo, lig, pocket, sampling, starts, tors, scores, stats)
    if R == 0:
        return e64
    n = len(starts)
    st = np.repeat(starts, R * S)
    tt = np.zeros((n, R, S, R), np.int64)
    for b in range(R):
        for k in range(S):
            tt[:, b, k, :b] = tors[:, :b]
            tt[:, b, k, b] = k
    tr = oracle.score_poses(lig, pocket, sampling, st, tt.reshape(-1, R)).reshape(n, R, S)
    ii, bb = np.arange(n)[:, None], np.arange(R)[None, :]
    chosen = tr[ii, bb, tors]
    best = tr.min(axis=2)
    ok = chosen - best <= tol(best)
    if stats is not None:
        stats.steps += ok.size
        stats.steps_strict += int(ok.sum())
        stats.steps_rounding += int((~ok).sum())
    for j, b in zip(*np.nonzero(~ok)):
        trials = tt[j, b]                       # the S trial poses at this bond
        ug = geo.coords(lig, sampling, np.full(S, starts[j]), trials)
        u64 = geo.exact_coords(lig, sampling, np.full(S, starts[j]), trials)
        e_at = geo.score_at(lig, sampling, ug)
        k = int(tors[j, b])
        assert e_at[k] - e_at.min() <= tol(e_at.min()), (
            f"start {starts[j]} bond {b}: GPU step {k} is not the best on its own coordinates "
            f"({e_at[k]} vs {e_at.min()} at step {int(e_at.argmin())})")
        for q in range(S):
            cr = float(np.max(np.abs(ug[q] - u64[q]))) / coord_envelope(u64[q], R)
            if stats is not None:
                stats.max_coord_ratio = max(stats.max_coord_ratio, cr)
            assert cr <= 1.0, f"start {starts[j]} bond {b} step {q}: coordinates outside the envelope"
    return e64


def oracle_run(lig, pocket, sampling):
    """Oracle greedy over every start."""
    return oracle.greedy(lig, pocket, sampling)


def compare_ligand(lig, pocket, sampling, gpu_rows, K=None, mode="fp32", stats=None):
    """Full check of one ligand's GPU top-K against the FP64 oracle."""
    K = sampling.top_k if K is None else K
    geo = Geometry(pocket, mode)
    valid = gpu_rows["start_id"] >= 0
    g_start = gpu_rows["start_id"][valid].astype(np.int64)
    g_tors = gpu_rows["tors"][valid]
    g_e = gpu_rows["score"][valid].astype(np.float64)
    assert valid.sum() == min(K, sampling.n_starts)
    assert len(set(g_start.tolist())) == len(g_start), "duplicate start ids"
    for a, b, sa, sb in zip(g_e[:-1], g_e[1:], g_start[:-1], g_start[1:]):
        assert a < b or (a == b and sa < sb), "GPU list not sorted by (score, start)"
    path_check(geo, lig, pocket, sampling, g_start, g_tors, g_e, stats)
    e, tors = oracle_run(lig, pocket, sampling)
    idx = oracle.top_k(e, K)
    o_set, g_set = set(idx.tolist()), set(g_start.tolist())
    R = tors.shape[1]
    kth_e, kth_s = g_e[-1], g_start[-1]
    for s in sorted(o_set - g_set):
        # the GPU's own path for this start must be right, and must not beat
        # the GPU's K-th entry (beyond the rounding of a re-run's memo frame)
        gs, gt = geo.path_of(lig, sampling, s)
        if stats is not None:
            stats.rerun_starts += 1
        path_check(geo, lig, pocket, sampling, [s], gt[None, :], [gs], stats)
        assert gs > kth_e - tol(kth_e) or (gs == kth_e and s > kth_s), (
            f"start {s}: GPU score {gs} beats the GPU list's K-th {kth_e} but is missing from it")
    return {"oracle_best": float(e[idx[0]]), "gpu_best": float(g_e[0]), "oracle_best_start": int(idx[0]),
            "same_best_start": int(idx[0]) == int(g_start[0]),
            "same_best_path": int(idx[0]) == int(g_start[0]) and np.array_equal(g_tors[0, :R], tors[idx[0]])}


# ---------------------------------------------------------------------------
# Exact rescoring and pose features: the same rules for their energies, and
# their discrete outputs (filter counts, histogram bins) equal to the
# oracle's at the GPU's coordinates except where a value sits on its
# threshold within the arithmetic bar.

def _gpu_geometry(geo, lig, sampling, starts, tors):
    ug = geo.coords(lig, sampling, starts, tors)
    return ug, geo.org + geo.h * ug


def rescore_check(geo, lig, pocket, sampling, starts, tors, rec, stats=None):
    """rec: RESCORED records of poses (start, tors) of one ligand."""
    R = int(np.sum(np.asarray(lig[3]) != 0))
    starts = np.asarray(starts, np.int64)
    tors = np.asarray(tors)[:, :R].astype(np.int64)
    receptor = pocket.receptor()
    x64 = oracle.pose_coords(lig, pocket.anchors, sampling, starts, tors)
    o = oracle.rescore_coords(lig, pocket, sampling, receptor, x64)
    ug, xg = _gpu_geometry(geo, lig, sampling, starts, tors)
    og = oracle.rescore_coords(lig, pocket, sampling, receptor, xg)
    u64 = (x64 - geo.org) / geo.h
    for key in ("e_inter", "e_clash"):
        ratio = np.abs(rec[key] - o[key]) / tol(o[key])
        bad = ratio > 1.0
        if stats is not None:
            stats.poses += len(ratio)
            stats.strict += int((~bad).sum())
            stats.rounding += int(bad.sum())
            stats.max_strict_ratio = max(stats.max_strict_ratio, float(ratio.max(initial=0.0)))
        for j in np.nonzero(bad)[0]:
            ar = abs(rec[key][j] - og[key][j]) / tol(og[key][j])
            cr = float(np.max(np.abs(ug[j] - u64[j]))) / coord_envelope(u64[j], R)
            if stats is not None:
                stats.max_arith_ratio = max(stats.max_arith_ratio, float(ar))
                stats.max_coord_ratio = max(stats.max_coord_ratio, cr)
            assert ar <= 1.0 and cr <= 1.0, (key, j, rec[key][j], o[key][j], og[key][j], cr)
    # filter counts at the GPU's coordinates: a difference needs an atom at
    # its threshold (receptor sum within the bar of the cap, or a coordinate
    # on a box face)
    s, m, f = oracle.rescore_atoms(lig, pocket, receptor, xg)
    near_cap = (np.abs(s - pocket.cap) <= tol(m)).sum(axis=1)
    on_face = (np.abs(f) <= 1e-9).sum(axis=1)
    dc = np.abs(rec["n_capped"].astype(np.int64) - og["n_capped"])
    do = np.abs(rec["n_outside"].astype(np.int64) - og["n_outside"])
    assert np.all(dc <= near_cap), (dc, near_cap)
    assert np.all(do <= on_face), (do, on_face)
    assert np.all(rec["pass"] == ((rec["n_outside"] == 0) & (rec["n_capped"] == 0)))
    return {"flag_diff_vs_exact": int(np.sum((rec["n_capped"] != o["n_capped"]) |
                                              (rec["n_outside"] != o["n_outside"]))),
            "flag_diff_vs_gpu_coords": int(np.sum((dc > 0) | (do > 0)))}


def features_check(geo, lig, pocket, sampling, starts, tors, feats, stats=None):
    """feats: [n, 256] GPU pose features of poses (start, tors) of one ligand.
    Histogram bins equal the oracle's at the GPU coordinates except for atoms
    whose value lies within 1e-5 of a bin edge; the other entries by the
    score rules."""
    R = int(np.sum(np.asarray(lig[3]) != 0))
    starts = np.asarray(starts, np.int64)
    tors = np.asarray(tors)[:, :R].astype(np.int64)
    ug, xg = _gpu_geometry(geo, lig, sampling, starts, tors)
    og = oracle.pose_features(lig, pocket, sampling, xg)
    e_at, mag = np.zeros(len(starts)), np.zeros(len(starts))
    n_at = len(lig[1])
    edge_atoms = np.zeros(len(starts), np.int64)
    for j in range(len(starts)):
        v = np.array([oracle.trilinear(pocket, int(lig[1][i]), xg[j, i:i + 1], sampling.penalty)[0]
                      for i in range(n_at)])
        sc = (v + 4.0) * 4.0               # bin edges at the integers 0..63 of sc
        edge = np.clip(np.round(sc), 0, 63)
        edge_atoms[j] = int(np.sum(np.abs(sc - edge) <= 1e-4))
    hist_g = np.round(np.expm1(feats[:, :64]))
    hist_o = np.round(np.expm1(og[:, :64]))
    moved = np.abs(hist_g - hist_o).sum(axis=1) / 2  # atoms in a different bin
    assert np.all(moved <= edge_atoms), (moved, edge_atoms)
    same = moved == 0
    np.testing.assert_allclose(feats[same, :64], og[same, :64], rtol=2e-6, atol=2e-6)
    for j in range(len(starts)):
        t = tol(og[j, 72] * n_at)
        assert abs(feats[j, 72] - og[j, 72]) * n_at <= t, (j, feats[j, 72], og[j, 72])
        assert abs(feats[j, 73] - og[j, 73]) <= tol(og[j, 73])
        np.testing.assert_allclose(feats[j, 64:72], og[j, 64:72], atol=float(tol(np.abs(og[j, 64:72]).max())))
    np.testing.assert_allclose(feats[:, 74:77], og[:, 74:77], rtol=1e-6)
    assert np.all(feats[:, 77:] == 0)
    return int((~same).sum())


def check_state_energies(geo, lig, pocket, sampling, rec, st64, energies, e64, stats=None, value=None):
    """Energies of continuous states (docking score, or a rescoring term when
    `value` maps Angstrom coordinate sets to FP64 values): the strict bar
    against the FP64 value of the exact state, else the rounding proof with
    the GPU's own state coordinates (ligate_state_coords)."""
    R = int(np.sum(np.asarray(lig[3]) != 0))
    energies = np.asarray(energies, np.float64)
    e64 = np.asarray(e64, np.float64)
    ratio = np.abs(energies - e64) / tol(e64)
    bad = ratio > 1.0
    if stats is not None:
        stats.poses += len(ratio)
        stats.strict += int((~bad).sum())
        stats.rounding += int(bad.sum())
        stats.max_strict_ratio = max(stats.max_strict_ratio, float(ratio.max(initial=0.0)))
    if not bad.any():
        return
    idx = np.nonzero(bad)[0]
    xg = geo.state_coords(lig, sampling, np.asarray(rec)[idx])
    x64 = oracle.state_coords(lig, np.array([st64[k] for k in idx]))
    if value is None:
        e_at = np.array([oracle.score_coords(lig, pocket, sampling, x) for x in xg])
    else:
        e_at = value(xg)
    for m, j in enumerate(idx):
        ar = abs(energies[j] - e_at[m]) / tol(e_at[m])
        u64 = (x64[m] - geo.org) / geo.h
        cr = float(np.max(np.abs(xg[m] - x64[m]))) / geo.h / coord_envelope(u64, R)
        if stats is not None:
            stats.max_arith_ratio = max(stats.max_arith_ratio, float(ar))
            stats.max_coord_ratio = max(stats.max_coord_ratio, cr)
        assert ar <= 1.0, (j, energies[j], e_at[m], e64[j])
        assert cr <= 1.0, (j, cr)

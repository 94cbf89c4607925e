"""GPU-vs-oracle comparison rules for the docking path.

Tolerance.  A score is a sum of per-atom map values (up to the +10 cap) and
clash terms that often cancel to a small total, so "1e-4 relative per-pose
score" is read relative to the scale of that sum: the sum of the absolute
values of its terms, which bounds the rounding error of any summation
order.  |E_gpu - E_64| <= 1e-4 * max(sum |terms|, 1).

The search is greedy, so FP32 and FP64 may pick different torsion steps
where two trials score within rounding of each other; after such a step the
two paths continue from different poses.  The rules therefore check the GPU
along its own choice path:
  * path check: for a GPU pose (start, tors), at every bond the GPU's step
    scores (FP64, other bonds as the GPU had them) within tolerance of the
    best step, and the reported score equals the FP64 score of the pose;
  * list check: GPU and oracle top-K lists agree on every start whose
    oracle path has no near-tie; a start present in only one list must be
    explained by a near-tie on its path or sit at the K-th boundary.
"""
from __future__ import annotations

import numpy as np

import oracle

REL = 1e-4


def tol(scale):
    return REL * np.maximum(np.abs(scale), 1.0)


def path_check(lig, pocket, sampling, starts, tors, scores, rel=REL):
    """Raise AssertionError unless every (start, tors, score) passes;
    returns (FP64 scores, scales)."""
    R = int(np.sum(np.asarray(lig[3]) != 0))
    S = sampling.torsion_steps
    starts = np.asarray(starts)
    tors = np.asarray(tors)[:, :R].astype(np.int64)
    scores = np.asarray(scores, np.float64)
    e64, mag = oracle.score_poses(lig, pocket, sampling, starts, tors, with_scale=True)
    lim = rel * np.maximum(mag, 1.0)
    bad = np.abs(scores - e64) > lim
    assert not bad.any(), (f"score mismatch: gpu {scores[bad]} vs fp64 {e64[bad]} "
                           f"(scale {mag[bad]}, starts {starts[bad]})")
    if R == 0:
        return e64, mag
    n = len(starts)
    st = np.repeat(starts, R * S)
    tt = np.zeros((n, R, S, R), np.int64)
    for b in range(R):
        for k in range(S):
            tt[:, b, k, :b] = tors[:, :b]
            tt[:, b, k, b] = k
    tr, tm = oracle.score_poses(lig, pocket, sampling, st, tt.reshape(-1, R), with_scale=True)
    tr = tr.reshape(n, R, S)
    tm = tm.reshape(n, R, S)
    ii, bb = np.arange(n)[:, None], np.arange(R)[None, :]
    chosen = tr[ii, bb, tors]
    kbest = tr.argmin(axis=2)
    best = tr[ii, bb, kbest]
    scale = np.maximum(tm[ii, bb, tors], tm[ii, bb, kbest])
    gap = chosen - best
    assert np.all(gap <= rel * np.maximum(scale, 1.0)), f"GPU step not optimal beyond tolerance: {gap.max()}"
    return e64, mag


def near_tie_starts(trials, scale):
    """Starts whose oracle path has a second-best trial within twice the
    tolerance of the best at some bond (trials [n, R, S], scale [n])."""
    if trials.shape[1] == 0 or trials.shape[2] < 2:
        return np.zeros(trials.shape[0], bool)
    srt = np.sort(trials, axis=2)
    gap = srt[:, :, 1] - srt[:, :, 0]
    return np.any(gap <= 2 * tol(scale)[:, None], axis=1)


def oracle_run(lig, pocket, sampling):
    """Oracle greedy over every start with the scale of each final pose."""
    e, tors, trials = oracle.greedy(lig, pocket, sampling, trials=True)
    _, mag = oracle.score_poses(lig, pocket, sampling, np.arange(len(e)), tors, with_scale=True)
    return e, tors, trials, mag


def compare_ligand(lig, pocket, sampling, gpu_rows, K=None):
    """Full check of one ligand's GPU top-K against the FP64 oracle."""
    K = sampling.top_k if K is None else K
    valid = gpu_rows["start_id"] >= 0
    g_start = gpu_rows["start_id"][valid].astype(np.int64)
    g_tors = gpu_rows["tors"][valid]
    g_e = gpu_rows["score"][valid].astype(np.float64)
    assert valid.sum() == min(K, sampling.n_starts)
    assert len(set(g_start.tolist())) == len(g_start), "duplicate start ids"
    for a, b, sa, sb in zip(g_e[:-1], g_e[1:], g_start[:-1], g_start[1:]):
        assert a < b or (a == b and sa < sb), "GPU list not sorted by (score, start)"
    path_check(lig, pocket, sampling, g_start, g_tors, g_e)
    e, tors, trials, mag = oracle_run(lig, pocket, sampling)
    idx = oracle.top_k(e, K)
    ties = near_tie_starts(trials, mag)
    o_set, g_set = set(idx.tolist()), set(g_start.tolist())
    kth = max(e[idx[-1]], g_e[-1])
    for s in o_set ^ g_set:
        boundary = abs(e[s] - kth) <= 2 * tol(mag[s])
        assert ties[s] or boundary, f"start {s} in only one list (oracle E {e[s]}, kth {kth})"
    R = tors.shape[1]
    for j, s in enumerate(g_start):
        if s in o_set and not ties[s]:
            assert np.array_equal(g_tors[j, :R], tors[s]), f"start {s}: torsion path differs"
            assert abs(g_e[j] - e[s]) <= tol(mag[s])
    return {"oracle_best": float(e[idx[0]]), "gpu_best": float(g_e[0]),
            "scale_best": float(mag[idx[0]]), "n_ties": int(ties[idx].sum())}

"""The lower bound the docking kernel prunes the greedy sweep with, checked
on the FP64 oracle (CPU).

A greedy sweep never raises a start's energy, and after bond b an atom that
no later bond moves keeps its place.  So before bond b the final energy is at
least the grid energy of those fixed atoms at the current pose plus, for
every atom a later bond still moves, the least value of its type's map (or
the out-of-box penalty if lower); the clash term is never negative.  A start
whose bound exceeds the K-th best energy found cannot enter the top-K
(paper Sec. 2: the ligand's result is its best poses), so its sweep may
stop without changing any result.  Moved sets here come from walking the
oracle's bond tree, independently of the kernel's DFS ranges."""
import numpy as np

import oracle

PENALTY = 10.0


def moved_sets(lig, u, v):
    n = len(lig[1])
    adj = [[] for _ in range(n)]
    for a, b in np.asarray(lig[2]):
        adj[a].append(b)
        adj[b].append(a)
    sets = []
    for a, b in zip(u, v):
        seen, stack = {b}, [b]
        while stack:
            x = stack.pop()
            for y in adj[x]:
                if y != a and y not in seen:
                    seen.add(y)
                    stack.append(y)
        seen.discard(b)  # the bond's own atoms lie on its axis
        sets.append(np.array(sorted(seen), int))
    return sets


def stage_bounds(lig, pocket, sampling, tors):
    """Bound before each bond b = 0..R (R: after the last bond), every start."""
    u, v = oracle.ligand_bonds(lig)
    R = len(u)
    sets = moved_sets(lig, u, v)
    n = len(lig[1])
    last = -np.ones(n, int)
    for b, s in enumerate(sets):
        last[s] = np.maximum(last[s], b)
    typ = np.asarray(lig[1])
    gmin = np.minimum(pocket.maps.reshape(pocket.maps.shape[0], -1).min(axis=1), PENALTY)
    starts = np.arange(sampling.n_starts)
    out, grid_final = np.zeros((R + 1, len(starts))), None
    for b in range(R + 1):
        tb = tors.copy()
        tb[:, b:] = 0  # bonds from b on still at their input angle
        x = oracle.pose_coords(lig, pocket.anchors, sampling, starts, tb)
        g = np.zeros((len(starts), n))
        for t in np.unique(typ):
            idx = np.where(typ == t)[0]
            g[:, idx] = oracle.trilinear(pocket, int(t), x[:, idx].reshape(-1, 3), PENALTY).reshape(len(starts), -1)
        fixed = last < b
        out[b] = g[:, fixed].sum(axis=1) + gmin[typ[~fixed]].sum()
        grid_final = g.sum(axis=1)
    return out, grid_final, R


def test_bound_never_exceeds_the_final_energy(tiny):
    lig = tiny.ligands.ligand(0)
    E, tors = oracle.greedy(lig, tiny.pocket, tiny.sampling)
    lb, grid_final, R = stage_bounds(lig, tiny.pocket, tiny.sampling, tors)
    assert R >= 2
    assert np.all(lb <= E[None, :] + 1e-9)
    # after the last bond every atom is fixed: the bound is the final grid
    # energy, and what separates it from the final score is the clash term
    np.testing.assert_allclose(lb[R], grid_final, rtol=0, atol=1e-9)
    assert np.all(E - grid_final >= -1e-9)
    # against the K-th best of the tiny search it excludes some starts early
    kth = np.sort(E)[tiny.sampling.top_k - 1]
    assert np.any(lb[:R].max(axis=0) > kth)


def test_bound_on_library_ligands(workload_factory):
    """Ligands of the 10,000-ligand library (nested and branched bonds), a
    reduced start set: the bound holds at every stage for every start."""
    from paper_2304_09953_gb300.workload import Sampling
    w = workload_factory("batched", n_ligands=24)
    samp = Sampling(w.sampling.quats[:8], 8, w.sampling.torsion_steps, 16)
    checked = 0
    for li in range(w.ligands.n):
        if w.ligands.n_rot[li] < 3:
            continue
        lig = w.ligands.ligand(li)
        E, tors = oracle.greedy(lig, w.pocket, samp)
        lb, _, _ = stage_bounds(lig, w.pocket, samp, tors)
        assert np.all(lb <= E[None, :] + 1e-9), li
        checked += 1
        if checked == 6:
            break
    assert checked == 6

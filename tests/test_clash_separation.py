"""The geometric fact behind the docking kernel's clash memo (CPU, oracle).

In the greedy sweep of bond b (paper Sec. 2: torsion steps searched bond by
bond), the steps of the earlier bonds set the ligand's conformation and the
later bonds are still at step 0.  A clash pair (i moved by b, j fixed) keeps
its distance at every step of b unless an earlier bond e separates them,
i.e. exactly one of j and b's moved subtree lies in e's subtree.  So:
pairs no earlier bond separates have the same distances for every prefix
of earlier steps; pairs one earlier bond e separates depend on e's step
only.  Checked on the oracle's own pose construction for random step
prefixes; pairs with two or more separating bonds are checked to vary, so
the test would notice a wrong separation rule."""
import numpy as np

import oracle


def subtrees(lig, u, v):
    """Atom sets moved by each rotatable bond (the side of v away from atom 0)."""
    n = len(lig[1])
    adj = [[] for _ in range(n)]
    for a, b in np.asarray(lig[2]):
        adj[a].append(b)
        adj[b].append(a)
    out = []
    for uu, vv in zip(u, v):
        seen, st = {vv}, [vv]
        while st:
            a = st.pop()
            for c in adj[a]:
                if c != uu and c not in seen:
                    seen.add(c)
                    st.append(c)
        out.append(seen)
    return out


def classify(lig, u, v, sub, b, topo):
    """Candidate pairs of bond b by their set of separating earlier bonds."""
    n = len(lig[1])
    groups = {}
    for i in sorted(sub[b] - {v[b]}):
        for j in range(n):
            if j in sub[b] or j == u[b] or topo[i, j] < 4:
                continue
            sep = tuple(e for e in range(b) if (j in sub[e]) != (v[b] in sub[e]))
            groups.setdefault(sep, []).append((i, j))
    return groups


def dists(lig, w, tors_rows, pairs):
    x = oracle.pose_coords(lig, w.pocket.anchors, w.sampling, np.zeros(len(tors_rows), np.int32),
                           np.asarray(tors_rows, np.int32))
    i, j = np.array(pairs).T
    return np.linalg.norm(x[:, i] - x[:, j], axis=-1)  # [rows, pairs]


def test_separating_bonds_decide_which_steps_change_a_pair(workload_factory):
    w = workload_factory("batched", n_ligands=64)
    rng = np.random.default_rng(11)
    S = w.sampling.torsion_steps
    checked = {0: 0, 1: 0, 2: 0}
    for li in range(w.ligands.n):
        lig = w.ligands.ligand(li)
        u, v = oracle.ligand_bonds(lig)
        R = len(u)
        if R < 4:
            continue
        sub = subtrees(lig, u, v)
        topo = oracle.topo_distance(lig)
        for b in range(2, R):
            groups = classify(lig, u, v, sub, b, topo)
            for sep, pairs in groups.items():
                k = int(rng.integers(1, S))
                base = rng.integers(0, S, size=(6, R))
                base[:, b] = k
                base[:, b + 1:] = 0
                if len(sep) == 0:
                    d = dists(lig, w, base, pairs)
                    np.testing.assert_allclose(d, np.broadcast_to(d[0], d.shape), rtol=0, atol=1e-9)
                    checked[0] += 1
                elif len(sep) == 1:
                    e = sep[0]
                    rows = base.copy()
                    rows[:, e] = rows[0, e]  # same step at e, anything elsewhere
                    d = dists(lig, w, rows, pairs)
                    np.testing.assert_allclose(d, np.broadcast_to(d[0], d.shape), rtol=0, atol=1e-9)
                    checked[1] += 1
                    # other steps at e move the pair, unless j sits on e's axis
                    moving = [(i, j) for i, j in pairs if j not in (u[e], v[e])]
                    if moving:
                        rows[1:, e] = (rows[0, e] + np.arange(1, 6)) % S
                        d2 = dists(lig, w, rows, moving)
                        assert np.abs(d2[1:] - d2[0]).max() > 1e-6
                else:
                    # two or more separating bonds: their steps do move the pair
                    moving = [(i, j) for i, j in pairs if j not in (u[sep[0]], v[sep[0]], u[sep[1]], v[sep[1]])]
                    if not moving:
                        continue
                    rows = np.repeat(base[:1], 6, axis=0)
                    rows[1:, sep[0]] = (rows[0, sep[0]] + np.arange(1, 6)) % S
                    rows[1:, sep[1]] = (rows[0, sep[1]] + np.arange(1, 6)) % S
                    d = dists(lig, w, rows, moving)
                    assert np.abs(d[1:] - d[0]).max() > 1e-6
                    checked[2] += 1
        if min(checked.values()) >= 20:
            break
    assert min(checked.values()) >= 20, checked

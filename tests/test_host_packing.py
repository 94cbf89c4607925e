"""Host packing of ligands for the docking kernel, checked on the CPU.

`ligate_inspect_ligand` runs the library's own packing (no device work).
Everything it returns is recomputed here from the definitions, in plain
Python: DFS pre-order from atom 0 with children by ascending input index
(paper Sec. 2 sweeps the rotatable bonds; the order is this build's reading),
rotatable bonds sorted by the DFS position of the child, the moved subtree
as a DFS range, clash candidates = moved x fixed pairs at least 4 bonds
apart (topological distances from the oracle), and their grouping by the
earlier bonds that separate them: none first, then the most frequent single
separator e1 (ties: the earlier bond), then the rest, each group in the
list's (i, j) order."""
import numpy as np
import pytest

import oracle
from paper_2304_09953_gb300 import native as N


def dfs_order(lig):
    n = len(lig[1])
    adj = [[] for _ in range(n)]
    for a, b in np.asarray(lig[2]):
        adj[a].append(int(b))
        adj[b].append(int(a))
    order, parent, st = [], [-1] * n, [0]
    seen = [False] * n
    seen[0] = True
    while st:
        a = st.pop()
        order.append(a)
        for c in sorted(adj[a], reverse=True):  # pushed descending, popped ascending
            if not seen[c]:
                seen[c] = True
                parent[c] = a
                st.append(c)
    return order, parent


def expected(lig):
    order, parent = dfs_order(lig)
    n = len(order)
    pos = {a: p for p, a in enumerate(order)}
    size = [1] * n
    for a in reversed(order[1:]):
        size[parent[a]] += size[a]
    bonds = []
    for (x, y), rot in zip(np.asarray(lig[2]), np.asarray(lig[3])):
        if not rot:
            continue
        child = int(y) if parent[y] == x else int(x)
        u = parent[child]
        bonds.append((pos[u], pos[child], pos[child] + size[child]))
    bonds.sort(key=lambda r: r[1])
    topo = oracle.topo_distance(lig)
    recs, cands = [], []
    slot = 0
    for bi, (u, v, end) in enumerate(bonds):
        groups = {0: [], 1: {}, 2: []}
        for i in range(v + 1, end):
            for j in range(n):
                if v <= j < end or j == u or topo[order[i], order[j]] < 4:
                    continue
                sep = [e for e in range(bi) if (bonds[e][1] <= j < bonds[e][2]) != (bonds[e][1] <= v < bonds[e][2])]
                c = i | (j << 8)
                if not sep:
                    groups[0].append(c)
                else:
                    groups[2].append((c, sep[0] if len(sep) == 1 else -1))
        by = {}
        for c, e in groups[2]:
            if e >= 0:
                by[e] = by.get(e, 0) + 1
        e1 = min(by, key=lambda e: (-by[e], e)) if by else -1
        one = [c for c, e in groups[2] if e == e1 and e1 >= 0]
        rest = [c for c, e in groups[2] if not (e == e1 and e1 >= 0)]
        off = len(cands)
        cands += groups[0] + one + rest
        e1_field = e1
        if one and bi >= 2:
            e1_field = e1 | (slot << 16)
            slot += 1
        recs.append([u, v, end, len(cands) - off, off, len(groups[0]), len(one), e1_field if one else -1])
    return np.array(order, np.int32), np.array(recs, np.int32).reshape(-1, 8), np.array(cands, np.uint16)


def test_packing_matches_its_definition(workload_factory):
    w = workload_factory("batched", n_ligands=64)
    checked = 0
    for li in range(0, 64, 3):
        lig = w.ligands.ligand(li)
        order, bonds, cand = N.ligate_inspect_ligand(w.ligands, li)
        eo, eb, ec = expected(lig)
        np.testing.assert_array_equal(order, eo)
        np.testing.assert_array_equal(bonds, eb)
        np.testing.assert_array_equal(cand, ec)
        checked += int(np.sum(eb[:, 6] > 0)) if len(eb) else 0
    assert checked > 10  # single-separator groups were exercised


def test_inspect_rejects_bad_arguments(workload_factory):
    w = workload_factory("batched", n_ligands=4)
    with pytest.raises(N.LigateError):
        N.ligate_inspect_ligand(w.ligands, 4)

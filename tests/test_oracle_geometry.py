"""Pins for the oracle's pose construction (rigid start + torsion tree).

Each check is fixed by geometry, not by re-running the oracle's own formula:
rotations preserve lengths, the quaternion rotation equals the Hamilton
product q v q*, a torsion changes the a-u-v-b dihedral by exactly its angle,
torsions about current axes commute, and the root side never moves.
"""
import numpy as np
import pytest

import oracle
from paper_2304_09953_gb300.workload import Sampling, make_ligands


def hamilton(p, q):
    w1, x1, y1, z1 = p
    w2, x2, y2, z2 = q
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2,
                     w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2,
                     w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def quat_rotate(q, v):
    q = np.asarray(q, float) / np.linalg.norm(q)
    qc = q * np.array([1, -1, -1, -1])
    return hamilton(hamilton(q, np.r_[0.0, v]), qc)[1:]


def dihedral(p0, p1, p2, p3):
    """Signed dihedral angle (IUPAC sign) from the atan2 formula."""
    b0 = p0 - p1
    b1 = p2 - p1
    b2 = p3 - p2
    b1n = b1 / np.linalg.norm(b1)
    v = b0 - np.dot(b0, b1n) * b1n
    w = b2 - np.dot(b2, b1n) * b1n
    x = np.dot(v, w)
    y = np.dot(np.cross(b1n, v), w)
    return np.arctan2(y, x)


def test_quaternion_matrix_matches_hamilton_product():
    rng = np.random.default_rng(0)
    for _ in range(50):
        q = rng.normal(size=4)
        R = oracle.quat_to_matrix(q)
        np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-14)
        assert abs(np.linalg.det(R) - 1.0) < 1e-13
        v = rng.normal(size=3)
        np.testing.assert_allclose(R @ v, quat_rotate(q, v), atol=1e-13)


def test_quaternion_axis_angle_right_hand_rule():
    # (cos 45deg, 0, 0, sin 45deg): +90 degrees about +z maps +x to +y
    q = np.array([np.cos(np.pi / 4), 0, 0, np.sin(np.pi / 4)])
    R = oracle.quat_to_matrix(q)
    np.testing.assert_allclose(R @ np.array([1.0, 0, 0]), [0, 1.0, 0], atol=1e-15)
    # q and -q are the same rotation
    np.testing.assert_allclose(oracle.quat_to_matrix(-q), R, atol=1e-15)


@pytest.fixture(scope="module")
def ligs():
    na = np.array([12, 24, 40, 60, 2, 1], np.int32)
    nr = np.array([3, 4, 8, 12, 0, 0], np.int32)
    return make_ligands(77, na, nr, 8)


def _samp(n_orient=4, S=8):
    rng = np.random.default_rng(5)
    return Sampling(rng.normal(size=(n_orient, 4)), 2, S, 4)


ANCH = np.array([[1.0, 2.0, 3.0], [-2.0, 0.5, 4.0]], np.float32)


def _tree_bonds(lig):
    return lig[2]


def test_rigid_and_torsion_moves_preserve_bond_lengths(ligs):
    rng = np.random.default_rng(1)
    samp = _samp()
    for i in range(ligs.n):
        lig = ligs.ligand(i)
        ref = lig[0].astype(np.float64)
        R = int(lig[3].sum())
        starts = rng.integers(0, samp.n_starts, size=6)
        tors = rng.integers(0, samp.torsion_steps, size=(6, max(R, 1)))[:, :R]
        X = oracle.pose_coords(lig, ANCH, samp, starts, tors)
        for b in _tree_bonds(lig):
            l0 = np.linalg.norm(ref[b[0]] - ref[b[1]])
            l1 = np.linalg.norm(X[:, b[0]] - X[:, b[1]], axis=1)
            np.testing.assert_allclose(l1, l0, rtol=1e-12)


def _fragments(lig):
    """Rigid fragments: connected components after cutting rotatable bonds."""
    n = len(lig[0])
    parent = list(range(n))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a
    for (a, b), r in zip(lig[2], lig[3]):
        if not r:
            parent[find(a)] = find(b)
    return np.array([find(a) for a in range(n)])


def test_torsions_preserve_intra_fragment_distances(ligs):
    rng = np.random.default_rng(2)
    samp = _samp()
    for i in range(ligs.n):
        lig = ligs.ligand(i)
        ref = lig[0].astype(np.float64)
        R = int(lig[3].sum())
        frag = _fragments(lig)
        D0 = np.linalg.norm(ref[:, None] - ref[None], axis=-1)
        same = frag[:, None] == frag[None]
        tors = rng.integers(0, samp.torsion_steps, size=(4, max(R, 1)))[:, :R]
        X = oracle.pose_coords(lig, ANCH, samp, rng.integers(0, samp.n_starts, 4), tors)
        for x in X:
            D = np.linalg.norm(x[:, None] - x[None], axis=-1)
            np.testing.assert_allclose(D[same], D0[same], rtol=1e-12, atol=1e-12)


def test_rigid_move_preserves_all_distances(ligs):
    samp = _samp()
    for i in range(ligs.n):
        lig = ligs.ligand(i)
        ref = lig[0].astype(np.float64)
        R = int(lig[3].sum())
        X = oracle.pose_coords(lig, ANCH, samp, np.arange(samp.n_starts),
                               np.zeros((samp.n_starts, R), int))
        D0 = np.linalg.norm(ref[:, None] - ref[None], axis=-1)
        for x in X:
            D = np.linalg.norm(x[:, None] - x[None], axis=-1)
            np.testing.assert_allclose(D, D0, rtol=1e-12, atol=1e-12)


def test_identity_start_is_centroid_shift(ligs):
    """Identity quaternion, zero torsions: x' = x - centroid + anchor."""
    samp = Sampling(np.array([[1.0, 0, 0, 0]]), 2, 8, 1)
    for i in range(ligs.n):
        lig = ligs.ligand(i)
        ref = lig[0].astype(np.float64)
        R = int(lig[3].sum())
        X = oracle.pose_coords(lig, ANCH, samp, [1], np.zeros((1, R), int))[0]
        np.testing.assert_allclose(X, ref - ref.mean(0) + ANCH[1].astype(np.float64), atol=1e-12)


def test_torsion_changes_dihedral_by_its_angle(ligs):
    """For every rotatable bond u-v, step k turns the a-u-v-b dihedral (a on
    the root side, b on the moved side) by 2 pi k / S, right-hand rule about
    u->v, and leaves the root side in place."""
    S = 8
    samp = Sampling(np.array([[1.0, 0, 0, 0]]), 1, S, 1)
    anch = np.zeros((1, 3), np.float32)
    for i in range(ligs.n):
        lig = ligs.ligand(i)
        us, vs = oracle.ligand_bonds(lig)
        R = len(us)
        if R == 0:
            continue
        nb = {a: set() for a in range(len(lig[0]))}
        for a, b in lig[2]:
            nb[a].add(b)
            nb[b].add(a)
        X0 = oracle.pose_coords(lig, anch, samp, [0], np.zeros((1, R), int))[0]
        for bi, (u, v) in enumerate(zip(us, vs)):
            a_side = [a for a in nb[u] if a != v]
            b_side = [b for b in nb[v] if b != u]
            if not a_side or not b_side:
                continue
            a, b = a_side[0], b_side[0]
            for k in range(1, S):
                t = np.zeros((1, R), int)
                t[0, bi] = k
                X = oracle.pose_coords(lig, anch, samp, [0], t)[0]
                d = dihedral(X[a], X[u], X[v], X[b]) - dihedral(X0[a], X0[u], X0[v], X0[b])
                want = 2 * np.pi * k / S
                assert abs(np.angle(np.exp(1j * (d - want)))) < 1e-10
                # same as a quaternion rotation of b about the axis u->v
                n = (X0[v] - X0[u]) / np.linalg.norm(X0[v] - X0[u])
                q = np.r_[np.cos(want / 2), np.sin(want / 2) * n]
                np.testing.assert_allclose(X[b], X0[v] + quat_rotate(q, X0[b] - X0[v]), atol=1e-12)
                # atom 0 (root) and u never move
                np.testing.assert_allclose(X[0], X0[0], atol=1e-12)
                np.testing.assert_allclose(X[u], X0[u], atol=1e-12)


def test_torsion_order_independence(ligs):
    """Torsions about CURRENT axes give the same coordinates in any order."""
    rng = np.random.default_rng(3)
    for i in range(ligs.n):
        lig = ligs.ligand(i)
        R = int(lig[3].sum())
        if R < 2:
            continue
        ang = rng.uniform(-np.pi, np.pi, size=R)
        base = oracle.torsions_in_order(lig, ang, np.arange(R))
        for _ in range(3):
            perm = rng.permutation(R)
            np.testing.assert_allclose(oracle.torsions_in_order(lig, ang, perm), base, atol=1e-11)
        np.testing.assert_allclose(oracle.torsions_in_order(lig, ang, np.arange(R)[::-1]), base,
                                   atol=1e-11)


def test_torsion_periodicity(ligs):
    samp = _samp(S=8)
    rng = np.random.default_rng(4)
    for i in range(ligs.n):
        lig = ligs.ligand(i)
        R = int(lig[3].sum())
        if R == 0:
            continue
        t = rng.integers(0, 8, size=(3, R))
        st = rng.integers(0, samp.n_starts, size=3)
        A = oracle.pose_coords(lig, ANCH, samp, st, t)
        B = oracle.pose_coords(lig, ANCH, samp, st, t + 8)
        np.testing.assert_allclose(A, B, atol=1e-11)


def test_sweep_order_is_dfs_preorder_of_child(ligs):
    """Bonds are swept by ascending DFS pre-order (children in ascending
    index) of their child atom; checked against an independent DFS here."""
    for i in range(ligs.n):
        lig = ligs.ligand(i)
        n = len(lig[0])
        adj = {a: [] for a in range(n)}
        for a, b in lig[2]:
            adj[a].append(b)
            adj[b].append(a)
        pre, parent, stack = {}, {0: -1}, [0]
        while stack:
            a = stack.pop()
            pre[a] = len(pre)
            for c in sorted((c for c in adj[a] if c != parent[a]), reverse=True):
                parent[c] = a
                stack.append(c)
        want = []
        for (a, b), r in zip(lig[2], lig[3]):
            if r:
                u, v = (a, b) if parent.get(b) == a else (b, a)
                want.append((pre[v], u, v))
        want.sort()
        us, vs = oracle.ligand_bonds(lig)
        assert list(zip(us, vs)) == [(u, v) for _, u, v in want]


def test_topological_distance_is_tree_path_length(ligs):
    lig = ligs.ligand(2)
    D = oracle.topo_distance(lig)
    n = len(lig[0])
    # Floyd-Warshall on the bond graph as the independent check
    F = np.full((n, n), 10 ** 6)
    np.fill_diagonal(F, 0)
    for a, b in lig[2]:
        F[a, b] = F[b, a] = 1
    for k in range(n):
        F = np.minimum(F, F[:, k:k + 1] + F[k:k + 1, :])
    np.testing.assert_array_equal(D, F)

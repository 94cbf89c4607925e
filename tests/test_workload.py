"""The synthetic workload follows its stated recipe: 1.5 A tree bonds, bond
angles of at least 100 degrees, non-bonded atoms at least 2 A apart,
rotatable bonds only between non-terminal atoms, and reproducible streams
(a slice of a library equals the same ligands of the full library)."""
import numpy as np

from paper_2304_09953_gb300.workload import make_workload, poses_per_ligand


def test_ligand_geometry_recipe(batched_small):
    L = batched_small.ligands
    for i in range(L.n):
        xyz, typ, bonds, rot = L.ligand(i)
        X = xyz.astype(np.float64)
        n = len(X)
        assert len(bonds) == n - 1
        assert np.all(bonds[:, 0] < bonds[:, 1])  # parent drawn before child
        lens = np.linalg.norm(X[bonds[:, 0]] - X[bonds[:, 1]], axis=1)
        np.testing.assert_allclose(lens, 1.5, atol=1e-6)
        deg = np.bincount(bonds.ravel(), minlength=n)
        assert deg.max() <= 4
        nb = [set() for _ in range(n)]
        for a, b in bonds:
            nb[a].add(b)
            nb[b].add(a)
        for a in range(n):
            ns = sorted(nb[a])
            for p in range(len(ns)):
                for q in range(p + 1, len(ns)):
                    u, v = X[ns[p]] - X[a], X[ns[q]] - X[a]
                    c = u @ v / np.linalg.norm(u) / np.linalg.norm(v)
                    assert c <= np.cos(np.deg2rad(100)) + 1e-6
        D = np.linalg.norm(X[:, None] - X[None], axis=-1)
        bonded = np.zeros((n, n), bool)
        bonded[bonds[:, 0], bonds[:, 1]] = bonded[bonds[:, 1], bonds[:, 0]] = True
        off = ~bonded & ~np.eye(n, dtype=bool)
        assert np.all(D[off] >= 2.0 - 1e-5)
        for (a, b), r in zip(bonds, rot):
            if r:
                assert deg[a] >= 2 and deg[b] >= 2
        assert int(rot.sum()) == L.n_rot[i]
        assert 15 <= n <= 60 and typ.max() < 8


def test_slices_reproduce_the_library():
    full = make_workload("batched", n_ligands=40)
    part = make_workload("batched", n_ligands=10, first_index=25, pocket=full.pocket)
    for i in range(10):
        a = full.ligands.ligand(25 + i)
        b = part.ligands.ligand(i)
        for x, y in zip(a, b):
            np.testing.assert_array_equal(x, y)


def test_pose_count_formula(tiny):
    # 512 starts x (1 + 4 * 7)
    assert poses_per_ligand(tiny.ligands, tiny.sampling)[0] == 512 * 29
    assert np.all(np.isfinite(tiny.pocket.maps)) and tiny.pocket.maps.max() == 10.0

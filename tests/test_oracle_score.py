"""Pins for the oracle's grid interpolation and score, and for the grid-map
generator.  Trilinear interpolation must be exact on functions linear in
each coordinate; node values come back at nodes (upper faces included); a
constant map scores N * c; hand-computed 2- and 5-atom cases fix the clash
term; the Lennard-Jones-like map has its closed-form minimum -eps at r0."""
import numpy as np

import oracle
from paper_2304_09953_gb300.workload import Pocket, Sampling, grid_maps, make_ligands


def _pocket(maps, origin=(0.0, 0.0, 0.0), h=0.5):
    return Pocket(np.ascontiguousarray(maps, np.float32), np.asarray(origin, float), h,
                  np.zeros((1, 3), np.float32))


def _node_field(f, dims, origin, h):
    nx, ny, nz = dims
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return f(origin[0] + h * x, origin[1] + h * y, origin[2] + h * z)


def test_trilinear_exact_on_affine_and_multilinear_fields():
    dims, origin, h = (7, 6, 5), (-1.0, 0.5, 2.0), 0.5
    rng = np.random.default_rng(0)
    affine = lambda x, y, z: 0.25 + 0.5 * x - 0.75 * y + 0.125 * z
    # x*y*z in grid units is multilinear: exact under trilinear interpolation
    multi = lambda x, y, z: ((x - origin[0]) / h) * ((y - origin[1]) / h) * ((z - origin[2]) / h) / 8.0
    maps = np.stack([_node_field(affine, dims, origin, h), _node_field(multi, dims, origin, h)])
    assert np.all(maps.astype(np.float32) == maps)  # exactly representable in FP32
    P = _pocket(maps, origin, h)
    hi = np.array(origin) + h * (np.array(dims) - 1)
    pts = rng.uniform(origin, hi, size=(500, 3))
    np.testing.assert_allclose(oracle.trilinear(P, 0, pts), affine(*pts.T), atol=1e-12)
    want = np.prod((pts - np.array(origin)) / h, axis=1) / 8.0
    np.testing.assert_allclose(oracle.trilinear(P, 1, pts), want, atol=1e-12)


def test_trilinear_node_values_including_upper_faces():
    dims, origin, h = (5, 4, 6), (0.0, 0.0, 0.0), 0.375
    rng = np.random.default_rng(1)
    maps = rng.uniform(-5, 10, size=(1, dims[2], dims[1], dims[0])).astype(np.float32)
    P = _pocket(maps, origin, h)
    z, y, x = np.meshgrid(np.arange(dims[2]), np.arange(dims[1]), np.arange(dims[0]), indexing="ij")
    pts = np.stack([x.ravel() * h, y.ravel() * h, z.ravel() * h], axis=1)
    np.testing.assert_array_equal(oracle.trilinear(P, 0, pts), maps[0].ravel().astype(np.float64))


def test_out_of_grid_penalty_and_boundaries():
    dims, h = (4, 4, 4), 1.0
    maps = np.full((1, 4, 4, 4), -2.0, np.float32)
    P = _pocket(maps, (0, 0, 0), h)
    inside = np.array([[0, 0, 0], [3, 3, 3], [1.5, 3.0, 0.0], [2.999, 0.001, 1.0]])
    outside = np.array([[-1e-9, 1, 1], [1, 3.0000001, 1], [1, 1, -0.5], [4, 4, 4]])
    np.testing.assert_array_equal(oracle.trilinear(P, 0, inside, penalty=10.0), -2.0)
    np.testing.assert_array_equal(oracle.trilinear(P, 0, outside, penalty=10.0), 10.0)


def test_constant_grid_scores_n_times_c():
    ligs = make_ligands(5, np.array([24, 40], np.int32), np.array([4, 6], np.int32), 8)
    c = -1.25
    maps = np.full((8, 96, 96, 96), c, np.float32)  # 47.5 A box: every pose stays inside
    P = Pocket(maps, np.zeros(3), 0.5, np.array([[23.75, 23.75, 23.75]], np.float32))
    samp = Sampling(np.random.default_rng(0).normal(size=(6, 4)), 1, 6, 2, clash_weight=0.0)
    for i in range(ligs.n):
        lig = ligs.ligand(i)
        R = int(lig[3].sum())
        t = np.random.default_rng(i).integers(0, 6, size=(6, R))
        e = oracle.score_poses(lig, P, samp, np.arange(6), t)
        np.testing.assert_allclose(e, len(lig[0]) * c, rtol=1e-14)


def _chain(coords):
    n = len(coords)
    bonds = np.array([[i, i + 1] for i in range(n - 1)], np.int32).reshape(-1, 2)
    return (np.asarray(coords, np.float32), np.zeros(n, np.uint8), bonds, np.zeros(n - 1, np.uint8))


def test_two_atom_score_on_affine_map():
    """Two bonded atoms: no clash pairs; score = f(a) + f(b)."""
    origin, h = (0.0, 0.0, 0.0), 0.5
    f = lambda x, y, z: 1.0 + 2.0 * x - 0.5 * y + 0.25 * z
    maps = _node_field(f, (16, 16, 16), origin, h)[None]
    P = _pocket(maps, origin, h)
    lig = _chain([[2.0, 3.0, 1.0], [3.5, 3.0, 1.0]])
    samp = Sampling(np.array([[1.0, 0, 0, 0]]), 1, 4, 1)
    e = oracle.score_coords(lig, P, samp, lig[0].astype(np.float64))
    assert abs(e - (f(2.0, 3.0, 1.0) + f(3.5, 3.0, 1.0))) < 1e-12


def test_clash_term_hand_computed():
    """5-atom chain folded so atoms 0 and 4 (4 bonds apart) sit 2 A apart:
    clash = (1 - 4/9)^2 with d_c = 3 A; atoms 0 and 3 (3 bonds apart) are
    excluded even though they are closer than d_c."""
    maps = np.zeros((1, 8, 8, 8), np.float32)
    P = _pocket(maps, (-10.0, -10.0, -10.0), 3.0)  # zero map covering the molecule
    coords = np.array([[0.0, 0, 0], [1.5, 0, 0], [1.5, 1.5, 0], [0.0, 1.5, 0], [0.0, 1.5, 2.0]])
    # chain 0-1-2-3-4 with |x0 - x4| = sqrt(0 + 2.25 + 4) = 2.5
    lig = _chain(coords)
    samp = Sampling(np.array([[1.0, 0, 0, 0]]), 1, 4, 1, clash_weight=2.0, clash_cutoff=3.0)
    d2 = np.sum((coords[0] - coords[4]) ** 2)
    want = 2.0 * (1.0 - d2 / 9.0) ** 2
    e = oracle.score_coords(lig, P, samp, coords)
    assert abs(e - want) < 1e-12
    # a 4-atom square: 0-3 is a 1-4 pair (3 bonds), excluded -> zero clash
    e4 = oracle.score_coords(_chain(coords[:4]), P, samp, coords[:4])
    assert e4 == 0.0


def test_clash_zero_for_straight_chain():
    maps = np.zeros((1, 8, 8, 8), np.float32)
    P = _pocket(maps, (-1.0, -1.0, -1.0), 3.0)
    coords = np.array([[1.5 * i, 0.0, 0.0] for i in range(8)])
    lig = _chain(coords)
    samp = Sampling(np.array([[1.0, 0, 0, 0]]), 1, 4, 1, clash_weight=1.0, clash_cutoff=3.0)
    assert oracle.score_coords(lig, P, samp, coords) == 0.0


def test_lj_map_minimum_and_cap():
    """One receptor atom of type 0: the map of type 0 at distance r0 = 2 r_0
    equals -eps_0 (closed-form minimum of eps[(r0/r)^12 - 2 (r0/r)^6]);
    the repulsive core is capped; nodes beyond the cutoff read 0."""
    radius = np.array([1.75, 2.0])
    eps = np.array([0.2, 0.1])
    r0 = 2 * radius[0]
    h = 0.5
    rec = np.array([[0.0, 0.0, 0.0]])
    origin = np.array([-r0, 0.0, 0.0])  # node (0,0,0) sits exactly r0 from the atom
    maps = grid_maps(radius, eps, rec, np.array([0]), origin, h, (40, 3, 3))
    assert abs(maps[0, 0, 0, 0] - np.float32(-eps[0])) <= 1e-7
    # mixed pair: eps = sqrt(eps_1 eps_0), r0 = r_1 + r_0
    origin2 = np.array([-(radius[0] + radius[1]), 0.0, 0.0])
    maps2 = grid_maps(radius, eps, rec, np.array([0]), origin2, h, (40, 3, 3))
    assert abs(maps2[1, 0, 0, 0] - np.float32(-np.sqrt(eps[0] * eps[1]))) <= 1e-7
    assert maps.max() <= 10.0 and maps[0, 0, 0, int(r0 / h)] == 10.0  # node at the atom: capped
    far = grid_maps(radius, eps, rec, np.array([0]), np.array([8.5, 0, 0]), h, (4, 2, 2))
    assert np.all(far == 0.0)

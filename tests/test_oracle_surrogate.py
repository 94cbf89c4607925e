"""Pins for the oracle's descriptor and surrogate network.

The descriptor is checked against an independent numpy computation and its
count identities; the network's backward pass against FP64 central
differences; Adam's first step against its closed form; BF16 rounding
against hand-worked ties and torch's own conversion."""
import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_2304_09953_gb300.workload import make_ligands


@pytest.fixture(scope="module")
def ligs():
    rng = np.random.default_rng(3)
    na = rng.integers(10, 80, size=40).astype(np.int32)
    nr = rng.integers(0, 15, size=40).astype(np.int32)
    return make_ligands(99, na, nr, 8)


def _pair_index(a, b):
    pairs = [(i, j) for i in range(8) for j in range(i + 1, 8)]
    return pairs.index((a, b))


def test_descriptor_matches_independent_histogram(ligs):
    for i in range(ligs.n):
        lig = ligs.ligand(i)
        xyz, typ, bonds, rot = lig
        d = oracle.descriptor(lig)
        n = len(typ)
        want = np.zeros(256)
        want[:8] = np.log1p(np.bincount(typ, minlength=8))
        hist = np.zeros((28, 8))
        X = xyz.astype(np.float32)
        # Bonded pairs sit exactly on the 1.5 A edge, so the bin is decided by
        # rounding; the decision is defined in FP32 as ((dx*dx + dy*dy) + dz*dz)
        # against the exactly representable squared edges (1.5 k)^2.
        edges2 = np.array([(1.5 * k) ** 2 for k in range(1, 8)], np.float32)
        for a in range(n):
            for b in range(a + 1, n):
                ta, tb = sorted((int(typ[a]), int(typ[b])))
                if ta == tb:
                    continue
                dv = X[a] - X[b]
                sq = dv * dv
                d2 = np.float32(np.float32(sq[0] + sq[1]) + sq[2])
                hist[_pair_index(ta, tb), int(np.sum(d2 >= edges2))] += 1
        want[8:232] = np.log1p(hist).ravel()
        want[232] = np.log1p(rot.sum())
        np.testing.assert_allclose(d, want, atol=1e-15)
        # count identities
        assert abs(np.expm1(d[:8]).sum() - n) < 1e-9
        distinct = sum(1 for a in range(n) for b in range(a + 1, n) if typ[a] != typ[b])
        assert abs(np.expm1(d[8:232]).sum() - distinct) < 1e-8
        assert np.all(d[233:] == 0.0)


def _params(seed=0, dims=(12, 16, 16, 16, 1)):
    rng = np.random.default_rng(seed)
    p = []
    for fi, fo in zip(dims[:-1], dims[1:]):
        p += [rng.normal(size=(fi, fo)) * np.sqrt(2.0 / fi), rng.normal(size=fo) * 0.1]
    return p


def test_mlp_backward_matches_central_differences():
    rng = np.random.default_rng(1)
    params = _params()
    X = rng.normal(size=(9, 12))
    t = rng.normal(size=9)
    y, cache = mlp.forward(params, X)
    g = mlp.backward(params, cache, y, t)
    h = 1e-6
    for li, P in enumerate(params):
        flat = P.reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp = mlp.mse(mlp.forward(params, X)[0], t)
            flat[idx] = old - h
            lm = mlp.mse(mlp.forward(params, X)[0], t)
            flat[idx] = old
            num = (lp - lm) / (2 * h)
            ana = g[li].reshape(-1)[idx]
            assert abs(num - ana) <= 1e-6 * max(1.0, abs(ana)), (li, idx, num, ana)


def test_mlp_forward_is_relu_chain():
    params = _params(2, dims=(3, 2, 2, 2, 1))
    X = np.array([[1.0, -2.0, 0.5]])
    h = X
    for l in range(4):
        z = h @ params[2 * l] + params[2 * l + 1]
        h = np.where(z > 0, z, 0.0) if l < 3 else z
    assert abs(mlp.forward(params, X)[0][0] - h[0, 0]) < 1e-15


def test_adam_first_step_closed_form():
    """At step 1 the bias-corrected moments are g and g^2, so every weight
    moves by lr * g / (|g| + eps)."""
    rng = np.random.default_rng(4)
    p = [rng.normal(size=(5, 3))]
    g = [rng.normal(size=(5, 3))]
    z = [np.zeros((5, 3))]
    newp, m, v = mlp.adam_step(p, g, z, z, 1, lr=1e-3, eps=1e-8)
    np.testing.assert_allclose(newp[0], p[0] - 1e-3 * g[0] / (np.abs(g[0]) + 1e-8), rtol=1e-12)
    np.testing.assert_allclose(m[0], 0.1 * g[0], rtol=1e-15)
    np.testing.assert_allclose(v[0], 0.001 * g[0] ** 2, rtol=1e-15)


def test_bf16_round_ties_and_torch():
    one = np.float32(1.0)
    ulp = 2.0 ** -7
    vals = np.array([1.0, 1 + ulp / 2, 1 + 1.5 * ulp, 1 + 0.75 * ulp, -3.0 - ulp / 2], np.float32)
    want = np.array([1.0, 1.0, 1 + 2 * ulp, 1 + ulp, -3.0], np.float32)
    np.testing.assert_array_equal(mlp.bf16_round(vals), want)
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(5).normal(size=10000).astype(np.float32) * 100
    tb = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(mlp.bf16_round(x), tb)
    assert one == 1.0


def test_he_init_scale():
    draws = np.random.default_rng(6).normal(size=mlp.n_weights())
    p = mlp.he_init(draws)
    assert [w.shape for w in p[::2]] == [(256, 512), (512, 512), (512, 512), (512, 1)]
    assert abs(p[0].std() - np.sqrt(2 / 256)) < 0.01 * np.sqrt(2 / 256) * 10


def test_bf16_activation_rounding_points():
    """With BF16 storage the only change is rounding of the hidden
    activations (forward) and of their gradients (backward): exactly
    representable values pass unchanged, others round to nearest even."""
    dims = (2, 1, 1, 1, 1)
    params = [np.array([[1.0], [2.0 ** -9]]), np.zeros(1), np.array([[1.0]]), np.zeros(1),
              np.array([[1.0]]), np.zeros(1), np.array([[3.0]]), np.zeros(1)]
    X = np.array([[1.0, 1.0], [2.0, 0.0]])
    y64, c64 = mlp.forward(params, X)
    y16, c16 = mlp.forward(params, X, bf16_acts=True)
    # h1 = 1 + 2^-9 is a tie between 1 and 1 + 2^-7 -> 1 (even); row 2 exact
    assert y64[0] == 3.0 * (1 + 2.0 ** -9) and y16[0] == 3.0
    assert y64[1] == y16[1] == 6.0
    t = np.array([0.0, 5.0])
    g64 = mlp.backward(params, c64, y64, t)
    g16 = mlp.backward(params, c16, y16, t)
    # dy = (3, 1); backward signal into layer 3 = 3 dy: exact in BF16 here
    d = np.array([3.0, 1.0])
    assert g16[6][0, 0] == d @ np.array([1.0, 2.0])
    assert g16[4][0, 0] == (3 * d) @ np.array([1.0, 2.0])
    assert g64[4][0, 0] == (3 * np.array([3 * (1 + 2.0 ** -9), 1.0])) @ np.array([1 + 2.0 ** -9, 2.0])
    assert len(dims) == 5

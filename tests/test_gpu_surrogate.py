"""Triage surrogate on the GPU vs the FP64 oracle, through the C ABI.

Descriptors: identical histogram bins (the FP32 bin decision is defined on
both sides), log1p values within FP32 rounding.  Network: forward and
backward of the BF16 tensor-core kernels vs the FP64 numpy oracle on the
same BF16-rounded weights and inputs (relative L2 <= 1e-2 per tensor; BF16
activations are the gap).  Ranking equals a stable sort of the predictions.
Triage: trained on the docking kernel's own best scores, the network's top
5% recalls far more of the true top 1% than a random 5% or a heavy-atom
count ranking."""
import numpy as np
import pytest

import oracle
from oracle import mlp as omlp
from paper_2304_09953_gb300 import docking as D
from paper_2304_09953_gb300 import native as N
from paper_2304_09953_gb300.workload import make_workload, normal

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

DIMS = omlp.DIMS


def split(flat):
    out, off = [], 0
    for fi, fo in zip(DIMS[:-1], DIMS[1:]):
        out.append(flat[off:off + fi * fo].reshape(fi, fo))
        off += fi * fo
        out.append(flat[off:off + fo])
        off += fo
    return out


def flat_params(params):
    return np.concatenate([p.reshape(-1) for p in params]).astype(np.float32)


def he_weights(seed):
    p = omlp.he_init(normal(seed, 1, omlp.n_weights()))
    rng = np.random.default_rng(seed)
    p = [q if q.ndim == 2 else rng.normal(size=q.shape) * 0.05 for q in p]
    return flat_params(p)


def test_descriptors_match_oracle(batched_small):
    w = batched_small
    bh = D.BatchHandle(w.ligands)
    out = torch.zeros((w.ligands.n, 256), dtype=torch.float32, device="cuda")
    N.ligate_descriptors(bh.h, out)
    got = out.cpu().numpy()
    for i in range(w.ligands.n):
        want = oracle.descriptor(w.ligands.ligand(i))
        np.testing.assert_allclose(got[i], want, rtol=2e-7, atol=1e-7)
        np.testing.assert_array_equal(np.round(np.expm1(got[i])), np.round(np.expm1(want)))


@pytest.mark.parametrize("engine,B", [("tc05", 256), ("tc05", 200), ("mma", 256), ("mma", 200)])
def test_forward_and_gradients_match_oracle(engine, B, monkeypatch):
    """Both contraction engines; B = 200 leaves a ragged 72-row tile."""
    monkeypatch.setenv("LIGATE_MLP_GEMM", engine)
    rng = np.random.default_rng(3)
    wf = omlp.bf16_round(he_weights(5))
    x = omlp.bf16_round(rng.normal(size=(B, 256)).astype(np.float32))
    t = rng.normal(size=B).astype(np.float32)
    s = N.ligate_surrogate_create(wf, 0)
    try:
        assert N.ligate_surrogate_engine(s) == (1 if engine == "tc05" else 0)
        xd = torch.from_numpy(x).cuda()
        td = torch.from_numpy(t).cuda()
        g = torch.zeros(N.LIGATE_SURROGATE_PARAMS, dtype=torch.float32, device="cuda")
        loss = N.ligate_surrogate_grad(s, xd, td, B, g)
        params = [p.astype(np.float64) for p in split(wf)]
        got = split(g.cpu().numpy().astype(np.float64))
        # oracle with the network's BF16 storage points (activations and their
        # gradients): the GPU must match it closely
        y, cache = omlp.forward(params, x.astype(np.float64), bf16_acts=True)
        assert abs(loss - omlp.mse(y, t)) <= 1e-3 * omlp.mse(y, t)
        want = omlp.backward(params, cache, y, t)
        for a, b in zip(got, want):
            rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
            assert rel <= 5e-3, rel
        # all-FP64 oracle: the gap is the BF16 storage itself (reported)
        y64, c64 = omlp.forward(params, x.astype(np.float64))
        want64 = omlp.backward(params, c64, y64, t)
        rels = [np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30) for a, b in zip(got, want64)]
        print("rel-L2 vs all-FP64 oracle per tensor:", np.round(rels, 4))
        assert max(rels) <= 0.1
        # forward through the public predict path (standardisation off: mu 0, sd 1)
        pred = torch.zeros(B, dtype=torch.float32, device="cuda")
        N.ligate_surrogate_predict(s, xd, B, pred)
        yp = pred.cpu().numpy()
        assert np.linalg.norm(yp - y) / np.linalg.norm(y) <= 1e-3
    finally:
        N.ligate_surrogate_destroy(s)


def test_tcgen05_and_mma_engines_agree(monkeypatch):
    """Same weights, two engines: predictions over 70,001 rows (three
    32,768-row chunks, ragged last tile) and the weights after two epochs of
    training.  Only FP32 summation order differs, so BF16 activations may
    differ by one unit in rare elements."""
    rng = np.random.default_rng(12)
    wf = he_weights(13)
    n = 70001
    desc = torch.from_numpy(rng.normal(size=(n, 256)).astype(np.float32)).cuda()
    lab = torch.from_numpy(rng.normal(size=n).astype(np.float32)).cuda()
    preds, weights = [], []
    for engine in ("tc05", "mma"):
        monkeypatch.setenv("LIGATE_MLP_GEMM", engine)
        s = N.ligate_surrogate_create(wf, 0)
        try:
            assert N.ligate_surrogate_engine(s) == (1 if engine == "tc05" else 0)
            pred = torch.zeros(n, dtype=torch.float32, device="cuda")
            N.ligate_surrogate_predict(s, desc, n, pred)
            preds.append(pred.cpu().numpy().astype(np.float64))
            N.ligate_surrogate_train(s, desc[:8192], lab[:8192], 8192, 2, 1024, 1e-3, 5)
            weights.append(N.ligate_surrogate_get_weights(s).astype(np.float64))
        finally:
            N.ligate_surrogate_destroy(s)
    a, b = preds
    assert np.all(np.isfinite(a))
    assert np.linalg.norm(a - b) / np.linalg.norm(b) <= 2e-3
    assert np.max(np.abs(a - b)) <= 2e-2 * np.max(np.abs(b))
    d0 = weights[1] - wf.astype(np.float64)
    assert np.linalg.norm(weights[0] - weights[1]) <= 5e-2 * np.linalg.norm(d0)


def test_first_adam_step_follows_gradient_sign():
    """One full-batch step: every weight whose gradient is clearly nonzero
    moves by lr against its sign (Adam's first step)."""
    rng = np.random.default_rng(4)
    wf = omlp.bf16_round(he_weights(6))
    n = 512
    desc = rng.normal(size=(n, 256)).astype(np.float32)
    lab = rng.normal(size=n).astype(np.float32)
    s = N.ligate_surrogate_create(wf, 0)
    try:
        dd = torch.from_numpy(desc).cuda()
        ld = torch.from_numpy(lab).cuda()
        N.ligate_surrogate_train(s, dd, ld, n, 1, n, 1e-3, 1)
        w1 = N.ligate_surrogate_get_weights(s)
    finally:
        N.ligate_surrogate_destroy(s)
    mu, sd = omlp.standardize_stats(desc)
    xs = omlp.bf16_round(((desc - mu) / sd).astype(np.float32)).astype(np.float64)
    ts = (lab - lab.mean()) / lab.std()
    params = [p.astype(np.float64) for p in split(wf)]
    y, cache = omlp.forward(params, xs)
    g = np.concatenate([q.reshape(-1) for q in omlp.backward(params, cache, y, ts)])
    step = (w1.astype(np.float64) - wf.astype(np.float64))
    clear = np.abs(g) > 1e-3 * np.abs(g).max()
    agree = np.mean(np.sign(step[clear]) == -np.sign(g[clear]))
    assert agree > 0.99, agree
    assert np.allclose(np.abs(step[clear]), 1e-3, rtol=0.05, atol=2e-5)


def test_rank_is_stable_sort_of_predictions():
    rng = np.random.default_rng(8)
    s = N.ligate_surrogate_create(None, 11)
    try:
        n = 70001
        desc = torch.from_numpy(rng.normal(size=(n, 256)).astype(np.float32)).cuda()
        pred = torch.zeros(n, dtype=torch.float32, device="cuda")
        k = int(np.ceil(n * 0.05))
        idx = torch.zeros(k, dtype=torch.int32, device="cuda")
        N.ligate_surrogate_rank(s, desc, n, 0.05, idx, pred)
        p = pred.cpu().numpy()
        want = np.lexsort((np.arange(n), p))[:k]
        np.testing.assert_array_equal(idx.cpu().numpy(), want)
    finally:
        N.ligate_surrogate_destroy(s)


def test_ensemble_rank_is_the_mean_of_its_networks():
    rng = np.random.default_rng(9)
    nets = [N.ligate_surrogate_create(None, 21 + m) for m in range(3)]
    try:
        n = 40003
        desc = torch.from_numpy(rng.normal(size=(n, 256)).astype(np.float32)).cuda()
        preds = []
        for h in nets:
            p = torch.zeros(n, dtype=torch.float32, device="cuda")
            N.ligate_surrogate_predict(h, desc, n, p)
            preds.append(p.cpu().numpy())
        k = int(np.ceil(n * 0.1))
        idx = torch.zeros(k, dtype=torch.int32, device="cuda")
        mean = torch.zeros(n, dtype=torch.float32, device="cuda")
        N.ligate_surrogate_rank_ensemble(nets, desc, n, 0.1, idx, mean)
        m = mean.cpu().numpy()
        np.testing.assert_allclose(m, np.mean(preds, axis=0), rtol=2e-6, atol=2e-6 * np.abs(m).max())
        np.testing.assert_array_equal(idx.cpu().numpy(), np.lexsort((np.arange(n), m))[:k])
        # one network: the plain ranking, bit for bit
        idx1 = torch.zeros(k, dtype=torch.int32, device="cuda")
        idx2 = torch.zeros(k, dtype=torch.int32, device="cuda")
        N.ligate_surrogate_rank_ensemble(nets[:1], desc, n, 0.1, idx1)
        N.ligate_surrogate_rank(nets[0], desc, n, 0.1, idx2)
        assert torch.equal(idx1, idx2)
        with pytest.raises(N.LigateError):
            N.ligate_surrogate_rank_ensemble([], desc, n, 0.1, idx1)
    finally:
        for h in nets:
            N.ligate_surrogate_destroy(h)


def test_triage_beats_the_method_without_it():
    """Dock 24,000 ligands of the batched library with the FP32 kernel,
    train on 20,000 best scores, rank the 4,000 held out: recall of their
    true top 1% inside the predicted top 5%, against a random 5% (expected
    recall 0.05) and against ranking by heavy-atom count."""
    w = make_workload("batched", n_ligands=24000)
    best = D.dock(w.pocket, w.ligands, w.sampling, mode="fp32c")["score"][:, 0].astype(np.float32)
    bh = D.BatchHandle(w.ligands)
    desc = torch.zeros((w.ligands.n, 256), dtype=torch.float32, device="cuda")
    N.ligate_descriptors(bh.h, desc)
    ntr = 20000
    s = N.ligate_surrogate_create(None, 7)
    try:
        lab = torch.from_numpy(best[:ntr]).cuda()
        l0 = N.ligate_surrogate_train(s, desc[:ntr].contiguous(), lab, ntr, 1, 1000, 1e-3, 3)
        l1 = N.ligate_surrogate_train(s, desc[:ntr].contiguous(), lab, ntr, 12, 1000, 1e-3, 4)
        assert l1 < l0
        nte = w.ligands.n - ntr
        k = int(np.ceil(0.05 * nte))
        idx = torch.zeros(k, dtype=torch.int32, device="cuda")
        N.ligate_surrogate_rank(s, desc[ntr:].contiguous(), nte, 0.05, idx)
        pick = idx.cpu().numpy()
    finally:
        N.ligate_surrogate_destroy(s)
    test_best = best[ntr:]
    truth = set(np.argsort(test_best, kind="stable")[:int(np.ceil(0.01 * nte))].tolist())
    recall = len(truth & set(pick.tolist())) / len(truth)
    heavy = np.argsort(w.ligands.n_atoms()[ntr:], kind="stable")[:k]
    recall_heavy = len(truth & set(heavy.tolist())) / len(truth)
    flex = np.argsort(-w.ligands.n_rot[ntr:], kind="stable")[:k]
    recall_flex = len(truth & set(flex.tolist())) / len(truth)
    print(f"triage recall {recall:.3f}; without the network: random 5% 0.05, fewest heavy atoms "
          f"{recall_heavy:.3f}, most rotatable bonds {recall_flex:.3f}")
    # the network's gain over docking a random 5%: at least 3x the recall
    assert recall >= 0.15 and recall > recall_heavy


def test_coarse_docking_feature_lifts_triage_recall():
    """The same network with the best score of a 256-start coarse docking
    run in descriptor column 233 (ligate_plan_best_scores): trained on
    100,000 ligands, ranking 4,000 held out, it recalls far more of the true
    top 1% than the descriptors alone and as much as the coarse score alone
    within one ligand (the gain over the coarse score alone shows at the
    10,000-ligand scale of the benchmark)."""
    import dataclasses
    from paper_2304_09953_gb300 import triage as T
    w = make_workload("batched", n_ligands=104000)
    best = D.dock(w.pocket, w.ligands, w.sampling, mode="fp32c")["score"][:, 0].astype(np.float32)
    ph = D.PocketHandle(w.pocket)
    bh = D.BatchHandle(w.ligands)
    desc = torch.zeros((w.ligands.n, 256), dtype=torch.float32, device="cuda")
    N.ligate_descriptors(bh.h, desc)
    cs = dataclasses.replace(w.sampling, quats=w.sampling.quats[:32], n_anchor=8, top_k=1)
    cp = D.Plan(ph, bh, cs, mode="bf16", rescore=False)
    cp.run()
    coarse = cp.result()["score"][:, 0]
    with_c = desc.clone()
    N.ligate_plan_best_scores(cp.h, with_c, 256, 233)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(with_c[:, 233].cpu().numpy(), coarse)
    cp.close()
    ntr, nte = 100000, 4000
    recalls = {}
    for name, x in (("descriptors", desc), ("with coarse", with_c)):
        s = N.ligate_surrogate_create(None, 9)
        try:
            N.ligate_surrogate_train(s, x[:ntr].contiguous(), torch.from_numpy(best[:ntr]).cuda(), ntr, 20,
                                     1024, 1e-3, 4)
            pred = torch.zeros(nte, dtype=torch.float32, device="cuda")
            N.ligate_surrogate_predict(s, x[ntr:].contiguous(), nte, pred)
            recalls[name] = T.recall_curve(pred.cpu().numpy(), best[ntr:], [0.05, 0.1])
        finally:
            N.ligate_surrogate_destroy(s)
    alone = T.recall_curve(coarse[ntr:], best[ntr:], [0.05, 0.1])
    print("recall at 5% / 10%:", {k: v for k, v in recalls.items()}, "coarse alone", alone)
    assert recalls["with coarse"][0.1] > recalls["descriptors"][0.1] + 0.2
    # 40 true top-1% ligands: one ligand is 0.025 of recall
    assert recalls["with coarse"][0.05] >= alone[0.05] - 0.05
    assert recalls["with coarse"][0.1] >= alone[0.1] - 0.025


def test_tcgen05_wait_timeout_is_reported_and_recoverable(monkeypatch):
    """Failure path without a GPU fault: the test hook makes one CTA of the
    next tcgen05 contraction skip its tensor loads (a flag nothing else
    sets), so its bounded wait runs out; predict returns LIGATE_ERR_TIMEOUT,
    and the next predict on the same context gives the normal results."""
    monkeypatch.setenv("LIGATE_MLP_GEMM", "tc05")
    rng = np.random.default_rng(21)
    s = N.ligate_surrogate_create(None, 3)
    try:
        assert N.ligate_surrogate_engine(s) == 1
        n = 1000
        desc = torch.from_numpy(rng.normal(size=(n, 256)).astype(np.float32)).cuda()
        ref = torch.zeros(n, dtype=torch.float32, device="cuda")
        N.ligate_surrogate_predict(s, desc, n, ref)
        N.ligate_debug_inject_fault(1)
        bad = torch.zeros(n, dtype=torch.float32, device="cuda")
        with pytest.raises(N.LigateError) as ei:
            N.ligate_surrogate_predict(s, desc, n, bad)
        assert ei.value.status == N.LIGATE_ERR_TIMEOUT
        again = torch.zeros(n, dtype=torch.float32, device="cuda")
        N.ligate_surrogate_predict(s, desc, n, again)
        np.testing.assert_array_equal(again.cpu().numpy(), ref.cpu().numpy())
    finally:
        N.ligate_surrogate_destroy(s)
    with pytest.raises(N.LigateError):
        N.ligate_debug_inject_fault(7)


def test_checkpoint_resumes_training_exactly(tmp_path):
    """Save after one epoch, load into a new object, train both one more
    epoch with the same seed: identical weights (Adam moments, step and
    standardisation travel with the checkpoint) and identical predictions."""
    rng = np.random.default_rng(31)
    n = 4096
    desc = torch.from_numpy(rng.normal(size=(n, 256)).astype(np.float32)).cuda()
    lab = torch.from_numpy(rng.normal(size=n).astype(np.float32)).cuda()
    a = N.ligate_surrogate_create(None, 5)
    b = None
    try:
        N.ligate_surrogate_train(a, desc, lab, n, 1, 512, 1e-3, 1)
        path = tmp_path / "sur.bin"
        N.ligate_surrogate_save(a, path)
        b = N.ligate_surrogate_load(path)
        np.testing.assert_array_equal(N.ligate_surrogate_get_weights(a), N.ligate_surrogate_get_weights(b))
        N.ligate_surrogate_train(a, desc, lab, n, 1, 512, 1e-3, 2)
        N.ligate_surrogate_train(b, desc, lab, n, 1, 512, 1e-3, 2)
        np.testing.assert_array_equal(N.ligate_surrogate_get_weights(a), N.ligate_surrogate_get_weights(b))
        pa = torch.zeros(n, dtype=torch.float32, device="cuda")
        pb = torch.zeros(n, dtype=torch.float32, device="cuda")
        N.ligate_surrogate_predict(a, desc, n, pa)
        N.ligate_surrogate_predict(b, desc, n, pb)
        np.testing.assert_array_equal(pa.cpu().numpy(), pb.cpu().numpy())
        bad = tmp_path / "bad.bin"
        bad.write_bytes(b"not a checkpoint")
        with pytest.raises(N.LigateError):
            N.ligate_surrogate_load(bad)
    finally:
        N.ligate_surrogate_destroy(a)
        if b is not None:
            N.ligate_surrogate_destroy(b)

"""GPU docking path vs the FP64 oracle, through the C ABI.

FP32 maps: every reported pose within 1e-4 relative of its FP64 score or,
where FP32 rounding of its coordinates moves it further, with the rounding
proof of tests/parity.py (exact arithmetic at the GPU's own coordinates,
coordinates inside the FP32 envelope); each greedy step optimal along the
GPU's own path by the same rule; and a start in the oracle's top-K but not
the GPU's re-docked alone and shown not to beat the GPU's K-th entry.  Sizes:
the 1-ligand configuration, the first 64 ligands of the 10,000-ligand
library, and the full library in the launch configuration the benchmark
times (sampled ligands checked)."""
import numpy as np
import pytest

import oracle
from paper_2304_09953_gb300 import docking as D
from paper_2304_09953_gb300 import native as N
from paper_2304_09953_gb300.workload import Sampling, make_ligands, make_workload
from tests.parity import Geometry, Stats, check_scores, compare_ligand, path_check, tol

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def full():
    return make_workload("batched")


@pytest.mark.parametrize("mode", ["fp32", "fp32c"])
def test_tiny_matches_oracle(tiny, mode):
    res = D.dock(tiny.pocket, tiny.ligands, tiny.sampling, mode=mode)
    st = Stats()
    info = compare_ligand(tiny.ligands.ligand(0), tiny.pocket, tiny.sampling, res[0], mode=mode, stats=st)
    print(st.line())
    assert info["same_best_path"] or abs(info["gpu_best"] - info["oracle_best"]) <= tol(info["oracle_best"])


def test_every_start_matches_oracle(tiny):
    """32 starts with K = 32: the GPU returns every start, and every start's
    score and greedy path pass the parity rules; the paths equal the
    oracle's wherever the oracle's own path has no step decided by less
    than the strict bar."""
    lig = tiny.ligands.ligand(0)
    st = Stats()
    geo = Geometry(tiny.pocket)
    same = 0
    for sub in range(4):
        samp = Sampling(tiny.sampling.quats[4 * sub:4 * sub + 4], 8, 8, 32)
        res = D.dock(tiny.pocket, tiny.ligands, samp, mode="fp32")[0]
        assert np.all(res["start_id"] >= 0)
        s = res["start_id"].astype(np.int64)
        path_check(geo, lig, tiny.pocket, samp, s, res["tors"], res["score"], st)
        e, tors = oracle.greedy(lig, tiny.pocket, samp)
        R = tors.shape[1]
        same += sum(np.array_equal(res["tors"][j, :R], tors[s[j]]) for j in range(32))
    print(st.line(), f"paths equal to the oracle's: {same}/128")
    assert same >= 120


def test_first_64_ligands(batched_small):
    w = batched_small
    res = D.dock(w.pocket, w.ligands, w.sampling, mode="fp32")
    st = Stats()
    for i in range(0, w.ligands.n, 4):
        compare_ligand(w.ligands.ligand(i), w.pocket, w.sampling, res[i], stats=st)
    print(st.line())


def test_clash_tables_with_unaligned_scratch(batched_small):
    """S = 12: a clash table is 12 x 12 floats (576 bytes), so the per-warp
    table regions do not start on 128-byte lines; 64 ligands x 256 starts
    keep many warps busy side by side, each dropping its own dead tables from
    L2 when it takes the next ligand.  Every ligand that has single-separator
    tables must still match the oracle."""
    w = batched_small
    samp = Sampling(w.sampling.quats[:32], 8, 12, 8)
    with_tables = [i for i in range(w.ligands.n)
                   if np.any(N.ligate_inspect_ligand(w.ligands, i)[1][2:, 6] > 0)]
    assert len(with_tables) >= 20
    res = D.dock(w.pocket, w.ligands, samp, mode="fp32")
    st = Stats()
    for i in with_tables[::2]:
        compare_ligand(w.ligands.ligand(i), w.pocket, samp, res[i], K=8, stats=st)
    print(st.line())


def test_sweep_bound_counts_and_pruning(batched_small):
    """Branch and bound on the sweep.  With K equal to the number of starts
    the K-th best stays infinite until the last start, nothing is bounded
    out, and the device counters equal the search space exactly.  With 256
    starts and K = 16 starts are bounded out (fewer atom evaluations and pair
    trials than the search space), and every checked ligand's top-K still
    matches the oracle, which sweeps every start in full."""
    w = batched_small
    ph, bh = D.PocketHandle(w.pocket), D.BatchHandle(w.ligands)
    try:
        for mode in ("fp32", "bf16"):
            pl = D.Plan(ph, bh, Sampling(w.sampling.quats[:2], 4, 16, 8), mode=mode)
            pl.result()
            wk = pl.work()
            pl.close()
            assert wk.done_pruned_starts == 0
            assert wk.done_atom_evals == wk.atom_evals and wk.done_pair_evals == wk.pair_evals
            assert wk.starts + wk.done_bond_sweeps * 15 == wk.poses  # S = 16
        samp = Sampling(w.sampling.quats[:32], 8, 16, 16)
        pl = D.Plan(ph, bh, samp, mode="fp32")
        res = pl.result()
        wk = pl.work()
        pl.close()
    finally:
        bh.close()
        ph.close()
    print(f"bounded out: {wk.done_pruned_starts:.0f} of {wk.starts:.0f} starts; atom evaluations "
          f"{wk.done_atom_evals / wk.atom_evals:.3f}, pair trials {wk.done_pair_evals / wk.pair_evals:.3f} "
          "of the search space")
    assert 0 < wk.done_pruned_starts < wk.starts
    assert wk.done_atom_evals < wk.atom_evals and wk.done_pair_evals < wk.pair_evals
    assert wk.starts + wk.done_bond_sweeps * 15 < wk.poses
    st = Stats()
    for i in range(0, w.ligands.n, 8):
        compare_ligand(w.ligands.ligand(i), w.pocket, samp, res[i], stats=st)
    print(st.line())


def test_screening_cutoff_keeps_every_pose_below_it(batched_small):
    """ligate_plan_set_cutoff / ligate_plan_best_quantile on 64 ligands (256
    starts, K = 16, FP32 maps).  The quantile is the k-th smallest best score;
    with it as cutoff every pose at or below it is the full run's, bit for
    bit and in the same order, no ligand reports a pose below its full-run
    best, and fewer atoms are evaluated; detached, the run is the full run
    again.  A plan over the first starts only (the coarse pass) gives a
    quantile at or above the full plan's."""
    w = batched_small
    samp = Sampling(w.sampling.quats[:32], 8, 16, 16)
    ph, bh = D.PocketHandle(w.pocket), D.BatchHandle(w.ligands)
    try:
        pl = D.Plan(ph, bh, samp, mode="fp32")
        full = pl.result()
        w_full = pl.work()
        cut = torch.empty(1, dtype=torch.float32, device="cuda")
        pl.best_quantile(0.25, cut)
        torch.cuda.synchronize()
        c = float(cut.item())
        best = full["score"][:, 0]
        assert c == np.sort(best)[int(np.ceil(0.25 * w.ligands.n)) - 1]
        pl.set_cutoff(cut)
        scr = pl.result()
        w_scr = pl.work()
        pl.set_cutoff(None)
        again = pl.result()
        pl.close()
        coarse = D.Plan(ph, bh, Sampling(w.sampling.quats[:8], 4, 16, 1), mode="fp32")
        coarse.result()
        cq = torch.empty(1, dtype=torch.float32, device="cuda")
        coarse.best_quantile(0.25, cq)
        torch.cuda.synchronize()
        coarse.close()
    finally:
        bh.close()
        ph.close()
    assert np.array_equal(again, full)
    kept = 0
    for i in range(w.ligands.n):
        f, s = full[i], scr[i]
        m = int(np.sum(f["score"] <= c))
        assert np.array_equal(s[:m], f[:m]), i
        assert m == 16 or s[m]["start_id"] == -1 or s[m]["score"] > c
        ok = s["start_id"] >= 0
        assert np.all(s["score"][ok] >= best[i])
        kept += m > 0
    assert kept == int(np.sum(best <= c))
    assert w_scr.done_atom_evals < w_full.done_atom_evals
    assert float(cq.item()) >= c
    print(f"screening at the 25% quantile {c:.3f}: atom evaluations "
          f"{w_scr.done_atom_evals / w_full.done_atom_evals:.3f} of the full run's")


def test_screening_with_rescoring_matches_the_chosen_form(workload_factory):
    """Screening as the benchmark runs it, on 2,000 ligands of the target
    library: a coarse plan (the first 32 orientations x 8 anchors, BF16, no
    rescoring) gives the 1% quantile of its best scores on the device; the
    chosen form (BF16 search, FP32 top-16 rescoring) run with that cutoff
    ranks the same ligands in its top 1% as without it, reports the same
    rescored best for every ligand whose BF16 best is at or below the cutoff,
    and its BF16 search keeps every such pose of the full run bit for bit."""
    import dataclasses
    w = workload_factory("combined", n_ligands=2000)
    n = w.ligands.n
    k1 = int(np.ceil(0.01 * n))
    ph, bh = D.PocketHandle(w.pocket), D.BatchHandle(w.ligands)
    try:
        chosen = D.Plan(ph, bh, w.sampling, mode="bf16", rescore=True)
        full = chosen.result()
        coarse = D.Plan(ph, bh, dataclasses.replace(w.sampling, quats=w.sampling.quats[:32], n_anchor=8, top_k=1),
                        mode="bf16", rescore=False)
        coarse.run()
        cut = torch.empty(1, dtype=torch.float32, device="cuda")
        coarse.best_quantile(0.01, cut)
        chosen.set_cutoff(cut)
        scr = chosen.result()
        search = D.Plan(ph, bh, w.sampling, mode="bf16", rescore=False)
        s_full = search.result()
        search.set_cutoff(cut)
        s_scr = search.result()
        c = float(cut.item())
        for pl in (chosen, coarse, search):
            pl.close()
    finally:
        bh.close()
        ph.close()

    def top(best):
        return set(np.lexsort((np.arange(n), best))[:k1].tolist())

    best16 = s_full["score"][:, 0]
    inside = np.where(best16 <= c)[0]
    assert c >= np.sort(best16)[k1 - 1]  # the coarse quantile bounds the full one
    assert top(scr["score"][:, 0]) == top(full["score"][:, 0])
    assert np.array_equal(scr["score"][inside, 0], full["score"][inside, 0])
    for i in inside:
        m = s_full[i]["score"] <= c
        assert np.array_equal(s_scr[i][:int(m.sum())], s_full[i][m]), i
    print(f"cutoff {c:.3f}: {len(inside)} of {n} ligands at or below it")


def test_target_library_sample(workload_factory):
    """Ligands of the 1,000,000-ligand target library (up to 80 atoms and 15
    rotatable bonds, so all four packed torsion words; 8 x 96^3 maps), 256
    starts: the FP32 form against the oracle on the largest and most flexible
    ligands of the first 64, and the BF16 form with FP32 rescoring within
    0.02 of the oracle's best on the same ligands."""
    w = workload_factory("combined", n_ligands=64)
    samp = Sampling(w.sampling.quats[:32], 8, w.sampling.torsion_steps, 16)
    n_at = np.diff(w.ligands.atom_offset)
    pick = sorted(set(np.argsort(-w.ligands.n_rot, kind="stable")[:6].tolist()) |
                  set(np.argsort(-n_at, kind="stable")[:6].tolist()))
    assert w.ligands.n_rot[pick].max() >= 13 and n_at[pick].max() >= 60
    res = D.dock(w.pocket, w.ligands, samp, mode="fp32")
    low = D.dock(w.pocket, w.ligands, samp, mode="bf16")
    st = Stats()
    errs = []
    for i in pick:
        lig = w.ligands.ligand(int(i))
        info = compare_ligand(lig, w.pocket, samp, res[i], stats=st)
        errs.append(abs(float(low[i]["score"][0]) - info["oracle_best"]))
    print(st.line(), f"bf16 best vs oracle best: max {max(errs):.2e}")
    assert max(errs) <= 0.02


def _dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


@pytest.mark.parametrize("mode,limit", [("fp32", None), ("fp32c", None), ("bf16", 0.5), ("fp16", 0.1)])
def test_explicit_pose_scores(batched_small, mode, limit):
    """ligate_score_poses on random (ligand, start, torsions) vs FP64: the
    FP32 layouts by the parity rules, the 16-bit maps within the error
    their rounding of the map values allows (their scores are rescored from
    FP32 maps before they are reported)."""
    w = batched_small
    rng = np.random.default_rng(7)
    n = 600
    li = rng.integers(0, w.ligands.n, n).astype(np.int32)
    starts = rng.integers(0, w.sampling.n_starts, n).astype(np.int32)
    tors = rng.integers(0, w.sampling.torsion_steps, (n, 16)).astype(np.uint8)
    for j in range(n):
        tors[j, w.ligands.n_rot[li[j]]:] = 0
    ph = D.PocketHandle(w.pocket)
    bh = D.BatchHandle(w.ligands)
    prec, layout = D.MODES[mode]
    s = N.make_sampling(w.sampling, prec, layout)
    out = torch.zeros(n, dtype=torch.float32, device="cuda")
    N.ligate_score_poses(ph.h, bh.h, s, n, _dev(li, torch.int32), _dev(starts, torch.int32),
                         _dev(tors, torch.uint8), out)
    got = out.cpu().numpy().astype(np.float64)
    if limit is None:
        st = Stats()
        geo = Geometry(w.pocket, mode)
        for l in np.unique(li):
            sel = np.nonzero(li == l)[0]
            R = int(w.ligands.n_rot[l])
            check_scores(geo, w.ligands.ligand(int(l)), w.pocket, w.sampling, starts[sel], tors[sel, :R],
                         got[sel], st)
        print(st.line())
    else:
        want = np.array([oracle.score_poses(w.ligands.ligand(int(li[j])), w.pocket, w.sampling, [starts[j]],
                                            tors[j:j + 1, :w.ligands.n_rot[li[j]]])[0] for j in range(n)])
        err = np.abs(got - want)
        assert err.max() <= limit, err.max()


def test_full_library_bench_configuration(full):
    """All 10,000 ligands in one persistent launch (default tile), 24 seeded
    ligands checked in full against the oracle."""
    res = D.dock(full.pocket, full.ligands, full.sampling, mode="fp32")
    assert res.shape == (10000, 16)
    assert np.all(res["start_id"] >= 0)
    rng = np.random.default_rng(1234)
    st = Stats()
    for i in rng.choice(full.ligands.n, 24, replace=False):
        compare_ligand(full.ligands.ligand(int(i)), full.pocket, full.sampling, res[i], stats=st)
    print(st.line())


def test_tile_shapes_give_identical_results(full):
    sub = make_workload("batched", n_ligands=300, pocket=full.pocket)
    a = D.dock(sub.pocket, sub.ligands, sub.sampling, mode="fp32c")
    t = N.ligate_tile()
    t.warps_per_cta = 4
    for b in range(N.LIGATE_N_BUCKETS):
        t.starts_per_item[b] = 96 + 32 * b
    b_ = D.dock(sub.pocket, sub.ligands, sub.sampling, mode="fp32c", tile=t)
    assert np.array_equal(a, b_)


def test_edge_cases(tiny):
    P = tiny.pocket
    # empty batch
    empty = make_workload("tiny", n_ligands=0, pocket=P)
    r = D.dock(P, empty.ligands, tiny.sampling)
    assert r.shape == (0, 4)
    # 1 and 2 atoms, R = 0, and K larger than the number of starts
    ligs = make_ligands(21, np.array([1, 2, 9], np.int32), np.array([0, 0, 0], np.int32), 6)
    samp = Sampling(tiny.sampling.quats[:2], 2, 8, 8)
    r = D.dock(P, ligs, samp)
    for i in range(3):
        assert np.all(r[i, :4]["start_id"] >= 0) and np.all(r[i, 4:]["start_id"] == -1)
        assert np.all(np.isinf(r[i, 4:]["score"]))
        compare_ligand(ligs.ligand(i), P, samp, r[i], K=8)


@pytest.mark.parametrize("S", [1, 3, 32])
def test_torsion_step_counts(tiny, S):
    samp = Sampling(tiny.sampling.quats[:8], 4, S, 6)
    r = D.dock(tiny.pocket, tiny.ligands, samp)
    compare_ligand(tiny.ligands.ligand(0), tiny.pocket, samp, r[0])


def test_largest_ligands():
    """128 atoms and 16 rotatable bonds, the library limits."""
    w = make_workload("tiny", n_ligands=0)
    big = make_ligands(5, np.array([128, 100], np.int32), np.array([16, 16], np.int32), 6)
    assert big.n_rot.max() == 16
    maps = np.zeros((6, 80, 80, 80), np.float32)
    maps += w.pocket.maps.mean()
    from paper_2304_09953_gb300.workload import Pocket
    rng = np.random.default_rng(0)
    maps = (maps + rng.normal(size=maps.shape).astype(np.float32)).astype(np.float32)
    P = Pocket(maps, np.zeros(3), 0.5, np.array([[19.75, 19.75, 19.75]], np.float32))
    samp = Sampling(w.sampling.quats[:4], 1, 4, 4)
    r = D.dock(P, big, samp)
    for i in range(2):
        compare_ligand(big.ligand(i), P, samp, r[i])


def test_subset_plan_equals_rows_of_full_run(batched_small):
    """A plan over a subset of the batch gives, row for row, the poses of
    the same ligands in the full run."""
    w = batched_small
    ph = D.PocketHandle(w.pocket)
    bh = D.BatchHandle(w.ligands)
    full = D.Plan(ph, bh, w.sampling, mode="bf16").result()
    sel = np.array([63, 5, 17, 17, 0, 42], np.int32)
    sub = D.Plan(ph, bh, w.sampling, mode="bf16", subset=sel).result()
    assert sub.shape == (len(sel), w.sampling.top_k)
    assert np.array_equal(sub, full[sel])
    with pytest.raises(N.LigateError):
        D.Plan(ph, bh, w.sampling, mode="bf16", subset=np.array([64], np.int32))


def test_host_array_call_equals_plan_path(batched_small):
    """ligate_dock_batch (pack, upload, dock, download in one call) returns
    the plan path's poses."""
    w = batched_small
    ph = D.PocketHandle(w.pocket)
    bh = D.BatchHandle(w.ligands)
    want = D.Plan(ph, bh, w.sampling, mode="fp16").result()
    s = N.make_sampling(w.sampling, N.LIGATE_FP16, N.LIGATE_LAYOUT_CORNER, rescore=True)
    got = np.zeros_like(want)
    N.ligate_dock_batch(ph.h, w.ligands, s, got)
    assert np.array_equal(got, want)


def test_autotune_cache_round_trip(batched_small, tmp_path, monkeypatch):
    """The tuned shape is written to LIGATE_TUNE_CACHE and picked up by a
    plan created without an explicit tile; results do not depend on it."""
    w = batched_small
    path = tmp_path / "tune.txt"
    monkeypatch.setenv("LIGATE_TUNE_CACHE", str(path))
    ph = D.PocketHandle(w.pocket)
    bh = D.BatchHandle(w.ligands)
    s = N.make_sampling(w.sampling, N.LIGATE_BF16, N.LIGATE_LAYOUT_CORNER, rescore=True)
    best = N.ligate_autotune(ph.h, bh.h, s, 5000.0)
    assert path.exists() and len(path.read_text().split()) == 12
    assert list(best.starts_per_item) == [0] * 8  # chunks come from the work model per plan
    pl = D.Plan(ph, bh, w.sampling, mode="bf16")
    t, launches = pl.tile()
    assert launches == 1
    assert t.warps_per_cta == best.warps_per_cta and t.reg_cap == best.reg_cap
    G = 32 // (1 << (w.sampling.torsion_steps - 1).bit_length())
    assert all(c % G == 0 and c >= G for c in t.starts_per_item)
    ref = D.Plan(ph, bh, w.sampling, mode="bf16", tile=N.ligate_tile()).result()
    assert np.array_equal(pl.result(), ref)


@pytest.mark.parametrize("mode", ["fp32", "bf16"])
def test_model_tile_is_valid_and_changes_nothing(batched_small, mode):
    """The analytic launch model gives a shape the plan accepts (plain layout:
    the 128-register instance; chunks within [128, 2048], multiples of the
    start group) and the same results as the default shape."""
    w = batched_small
    ph = D.PocketHandle(w.pocket)
    bh = D.BatchHandle(w.ligands)
    prec, layout = D.MODES[mode]
    s = N.make_sampling(w.sampling, prec, layout, rescore=(mode != "fp32"))
    t = N.ligate_model_tile(ph.h, bh.h, s)
    assert t.warps_per_cta in (2, 4) and t.reg_cap in (1, 2, 3)
    if mode == "fp32":
        assert t.reg_cap == 3
    G = 32 // (1 << (w.sampling.torsion_steps - 1).bit_length())
    for c in t.starts_per_item:
        assert c % G == 0 and G <= c <= 2048
    pl = D.Plan(ph, bh, w.sampling, mode=mode, tile=t)
    ref = D.Plan(ph, bh, w.sampling, mode=mode, tile=N.ligate_tile()).result()
    assert np.array_equal(pl.result(), ref)


def test_journaled_screening_resumes_after_an_interruption(batched_small, tmp_path):
    """Chunks of 16 ligands; the first run stops (an exception raised on the
    host) after the second chunk is journaled; the rerun docks only the
    missing chunks and the result equals one run over the whole library."""
    from paper_2304_09953_gb300.screen import screen_library
    w = batched_small
    seen = []

    def stop_after_two(c):
        seen.append(c)
        if len(seen) == 2:
            raise KeyboardInterrupt("simulated interruption")

    with pytest.raises(KeyboardInterrupt):
        screen_library(w.pocket, w.ligands, w.sampling, tmp_path / "j", chunk=16, on_chunk=stop_after_two)
    rest = []
    out = screen_library(w.pocket, w.ligands, w.sampling, tmp_path / "j", chunk=16, on_chunk=rest.append)
    assert seen == [0, 1] and rest == [2, 3]
    ref = D.dock(w.pocket, w.ligands, w.sampling, mode="bf16")
    assert np.array_equal(out, ref)
    with pytest.raises(ValueError):
        screen_library(w.pocket, w.ligands.subset(np.arange(10)), w.sampling, tmp_path / "j", chunk=16)


def test_pose_coords_are_the_exact_poses_within_the_fp32_envelope(batched_small):
    """ligate_pose_coords on random poses of the 64 ligands: every atom (input
    order) within the FP32 construction envelope of the oracle's FP64 pose;
    rows past a ligand's atoms untouched; a bad ligand or start index gives
    NaN rows.  The measured error distribution is printed for the record."""
    from tests.parity import U32, coord_envelope
    w = batched_small
    rng = np.random.default_rng(21)
    n = 512
    li = rng.integers(0, w.ligands.n, n).astype(np.int32)
    starts = rng.integers(0, w.sampling.n_starts, n).astype(np.int32)
    tors = rng.integers(0, w.sampling.torsion_steps, (n, 16)).astype(np.uint8)
    for j in range(n):
        tors[j, w.ligands.n_rot[li[j]]:] = 0
    li[-1], starts[-2] = w.ligands.n, w.sampling.n_starts  # out of range
    ph = D.PocketHandle(w.pocket)
    bh = D.BatchHandle(w.ligands)
    s = N.make_sampling(w.sampling)
    out = torch.full((n * 128 * 3,), 7.0, dtype=torch.float32, device="cuda")
    N.ligate_pose_coords(ph.h, bh.h, s, n, _dev(li, torch.int32), _dev(starts, torch.int32),
                         _dev(tors, torch.uint8), out)
    u = out.cpu().numpy().reshape(n, 128, 3).astype(np.float64)
    assert np.all(np.isnan(u[-2:]))
    org, h = np.asarray(w.pocket.origin), w.pocket.spacing
    ratios, by_r = [], {}
    for j in range(n - 2):
        lig = w.ligands.ligand(int(li[j]))
        na, R = len(lig[0]), int(w.ligands.n_rot[li[j]])
        assert np.all(u[j, na:] == 7.0)
        x64 = oracle.pose_coords(lig, w.pocket.anchors, w.sampling, [starts[j]], tors[j:j + 1, :R].astype(np.int32))
        u64 = (x64[0] - org) / h
        err = float(np.max(np.abs(u[j, :na] - u64)))
        assert err <= coord_envelope(u64, R), (j, err, coord_envelope(u64, R))
        r_ = err / (U32 * float(np.max(np.abs(u64))))
        ratios.append(r_)
        by_r[R] = max(by_r.get(R, 0.0), r_)
    q = np.quantile(ratios, [0.5, 0.99, 1.0])
    print(f"coordinate error / (u X): median {q[0]:.1f}, 99% {q[1]:.1f}, max {q[2]:.1f}; max by R "
          + ", ".join(f"{k}:{v:.0f}" for k, v in sorted(by_r.items())))


def test_device_subset_run_equals_rows_of_full_run(batched_small):
    """ligate_plan_run_subset: a selection given on the device docks to the
    same poses as the full run's rows, twice in a row and for a new
    selection; a repeated ligand keeps one of its rows (the other is empty),
    an out-of-range index gives an empty row; the post-docking stages then
    act on the selection's rows."""
    w = batched_small
    ph = D.PocketHandle(w.pocket)
    bh = D.BatchHandle(w.ligands)
    pl = D.Plan(ph, bh, w.sampling, mode="bf16")
    full = pl.result()
    for sel in (np.array([63, 5, 17, 0, 42, 7], np.int32), np.array([63, 5, 17, 0, 42, 7], np.int32),
                np.arange(64, dtype=np.int32)[::-3]):
        got = pl.run_subset(sel, result=True)
        assert np.array_equal(got, full[sel])
    bad = np.array([4, 4, 999, -1, 6], np.int32)
    got = pl.run_subset(bad, result=True)
    empty = got["start_id"][:, 0] == -1
    assert list(empty[2:]) == [True, True, False]
    assert empty[0] != empty[1]
    j = 0 if not empty[0] else 1
    assert np.array_equal(got[j], full[4]) and np.array_equal(got[4], full[6])
    assert np.all(np.isinf(got[empty]["score"]))
    rs = pl.rescore_exact()
    assert rs.shape == (5, w.sampling.top_k)
    assert np.all(np.isinf(rs[empty]["energy"])) and np.all(np.isfinite(rs[~empty]["energy"]))
    pl.result()
    ref = pl.rescore_exact()
    np.testing.assert_array_equal(rs[4], ref[6])
    with pytest.raises(N.LigateError):
        D.Plan(ph, bh, w.sampling, mode="bf16", subset=np.array([1, 2], np.int32)).run_subset(np.array([0], np.int32))


def test_host_array_call_in_two_halves_equals_plan_path(full):
    """ligate_dock_batch on 3,000 ligands packs and docks the library in
    parts (each packed while the previous one docks, one stream per part):
    the same poses as one plan over all of them; a malformed ligand in a
    later part is reported with its number in the input."""
    sub = make_workload("batched", n_ligands=3000, pocket=full.pocket)
    ph = D.PocketHandle(sub.pocket)
    bh = D.BatchHandle(sub.ligands)
    want = D.Plan(ph, bh, sub.sampling, mode="bf16").result()
    s = N.make_sampling(sub.sampling, N.LIGATE_BF16, N.LIGATE_LAYOUT_CORNER, rescore=True)
    got = np.zeros_like(want)
    N.ligate_dock_batch(ph.h, sub.ligands, s, got)
    assert np.array_equal(got, want)
    bad = sub.ligands.subset(np.arange(3000))
    j = int(bad.bond_offset[2500])
    bad.bonds[j] = bad.bonds[j + 1]  # a repeated edge: no longer a tree
    with pytest.raises(N.LigateError) as err:
        N.ligate_dock_batch(ph.h, bad, s, np.zeros_like(want))
    # "ligand <i> ... (ligand numbers counted from ligand <first> of the input)":
    # the second part's number plus its first input ligand is the bad one
    import re
    m = re.search(r"ligand (\d+): .*counted from ligand (\d+) of the input", str(err.value))
    assert m and int(m.group(1)) + int(m.group(2)) == 2500, str(err.value)


def test_plan_output_is_the_last_run(batched_small):
    """Plan.output() copies the last run's rows from the plan's buffer: the
    full run's, then a subset run's."""
    w = batched_small
    ph = D.PocketHandle(w.pocket)
    bh = D.BatchHandle(w.ligands)
    pl = D.Plan(ph, bh, w.sampling, mode="bf16")
    full = pl.result()
    assert np.array_equal(pl.output(), full)
    sel = np.array([9, 3, 60], np.int32)
    pl.run_subset(sel)
    assert np.array_equal(pl.output(), full[sel])

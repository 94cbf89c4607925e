"""Precision pattern: BF16 / FP16 corner-packed maps, FP32 accumulation,
top-16 re-scored from the FP32 maps.  On the full 10,000-ligand library:
  * every reported pose's score (an FP32 rescore) passes the FP32 parity
    rules against its FP64 score (tests/parity.py);
  * the reported best score of each sampled ligand lies within 0.02 of the
    oracle's best score (the FP64 greedy search over all starts);
  * the top-1% ligands agree with the plain FP32 GPU run at >= 0.99 overlap.
Measured figures are printed for the record."""
import numpy as np
import pytest

import oracle
from paper_2304_09953_gb300 import docking as D
from paper_2304_09953_gb300.workload import make_workload
from tests.parity import Geometry, Stats, check_scores, path_check

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def runs():
    w = make_workload("batched")
    ph = D.PocketHandle(w.pocket)
    bh = D.BatchHandle(w.ligands)
    out = {}
    for mode in ("fp32", "bf16", "fp16"):
        pl = D.Plan(ph, bh, w.sampling, mode=mode, rescore=mode != "fp32")
        out[mode] = pl.result()
        pl.close()
    return w, out


def _overlap(a, b, frac=0.01):
    n = len(a)
    k = int(np.ceil(frac * n))
    ta = set(np.lexsort((np.arange(n), a))[:k].tolist())
    tb = set(np.lexsort((np.arange(n), b))[:k].tolist())
    return len(ta & tb) / k


@pytest.mark.parametrize("mode", ["fp16", "bf16"])
def test_reduced_precision_maps_with_fp32_rescore(runs, mode):
    w, res = runs
    r = res[mode]
    truth = res["fp32"]["score"][:, 0]
    ov = _overlap(r["score"][:, 0], truth)
    rng = np.random.default_rng(99)
    sample = rng.choice(w.ligands.n, 24, replace=False)
    best_err = []
    st = Stats()
    geo = Geometry(w.pocket, "fp32")
    for i in sample:
        lig = w.ligands.ligand(int(i))
        R = int(w.ligands.n_rot[i])
        check_scores(geo, lig, w.pocket, w.sampling, r["start_id"][i], r["tors"][i][:, :R], r["score"][i], st)
        e_or, _ = oracle.greedy(lig, w.pocket, w.sampling)
        best_err.append(abs(float(r["score"][i, 0]) - e_or.min()))
    best_err = np.array(best_err)
    print(f"{mode}: top-1% overlap vs FP32 {ov:.3f}; best vs oracle best: median {np.median(best_err):.2e}, "
          f"max {best_err.max():.2e}; {st.line()}")
    assert best_err.max() <= 0.02
    assert ov >= 0.99


def test_fp32_corner_layout_equals_plain_within_rounding(runs):
    w, res = runs
    sub = make_workload("batched", n_ligands=200, pocket=w.pocket)
    a = D.dock(sub.pocket, sub.ligands, sub.sampling, mode="fp32c")
    b = res["fp32"][:200]
    assert _overlap(a["score"][:, 0], b["score"][:, 0], 0.05) >= 0.9
    geo = Geometry(sub.pocket, "fp32c")
    st = Stats()
    for i in range(0, 200, 20):
        path_check(geo, sub.ligands.ligand(i), sub.pocket, sub.sampling, a[i]["start_id"], a[i]["tors"],
                   a[i]["score"], st)
    print(st.line())

"""ligate_dock_noalloc, the allocation-free docking entry point.

It exists for callers that cannot call cudaMalloc (a process whose device
memory is all reserved by its own pool, or a loop that cannot afford
cudaMalloc's implicit synchronisation): its scratch lives in a fixed device
array inside the library.  Checked here through the C ABI: two calls in a
row give the same poses as the allocating plan path (same starts and
torsion steps, scores within the docking tolerance), the second call leaves
the device's free memory unchanged (the first may load the library's device
code, and with it the array), and requests larger than the array are
refused with an error.  This file is named to be
collected last; it also passes alone in a fresh process."""
import numpy as np
import pytest

from paper_2304_09953_gb300 import docking as D
from paper_2304_09953_gb300 import native as N
from paper_2304_09953_gb300.workload import make_workload
from tests.parity import REL

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("mode", ["fp32", "bf16"])
def test_noalloc_matches_plan_path_twice(mode):
    w = make_workload("batched", n_ligands=400)
    ph = D.PocketHandle(w.pocket)
    bh = D.BatchHandle(w.ligands)
    pl = D.Plan(ph, bh, w.sampling, mode=mode)
    want = pl.result()
    pl.close()
    prec, layout = D.MODES[mode]
    s = N.make_sampling(w.sampling, prec, layout, rescore=prec != N.LIGATE_FP32)
    K = w.sampling.top_k
    outs = [torch.full((w.ligands.n * K * 24,), 0xAB, dtype=torch.uint8, device="cuda") for _ in range(2)]
    torch.cuda.synchronize()
    for call in range(2):
        if call == 1:  # the first call may have loaded the array; the second allocates nothing
            free0 = torch.cuda.mem_get_info()[0]
            held0 = torch.cuda.memory_reserved()
        out = outs[call]
        N.ligate_dock_noalloc(ph.h, bh.h, s, out)
        torch.cuda.synchronize()
        if call == 1:
            assert torch.cuda.mem_get_info()[0] == free0, "the second call changed the free device memory"
            assert torch.cuda.memory_reserved() == held0
        got = out.cpu().numpy().view(N.POSE_DTYPE).reshape(w.ligands.n, K)
        np.testing.assert_array_equal(got["start_id"], want["start_id"])
        np.testing.assert_array_equal(got["tors"], want["tors"])
        scale = np.maximum(np.abs(want["score"]), 1.0)
        assert np.all(np.abs(got["score"] - want["score"]) <= REL * scale), call


def test_noalloc_refuses_oversized_requests():
    w = make_workload("batched", n_ligands=6000)
    ph = D.PocketHandle(w.pocket)
    bh = D.BatchHandle(w.ligands)
    s = N.make_sampling(w.sampling)
    out = torch.zeros(w.ligands.n * w.sampling.top_k * 24, dtype=torch.uint8, device="cuda")
    with pytest.raises(N.LigateError) as err:
        N.ligate_dock_noalloc(ph.h, bh.h, s, out)
    assert err.value.status == N.LIGATE_ERR_UNSUPPORTED
    assert "scratch" in str(err.value)

"""Convenience layer over the C ABI: RAII wrappers for pockets, batches and
plans, returning numpy structured arrays of poses.  No computation here:
every selection and score comes from the library's kernels."""
from __future__ import annotations

import numpy as np

from . import native as N


class PocketHandle:
    def __init__(self, pocket, mask=N.LIGATE_POCKET_FP32_CORNER | N.LIGATE_POCKET_BF16_CORNER
                 | N.LIGATE_POCKET_FP16_CORNER):
        self.h = N.ligate_pocket_create(pocket.maps, pocket.origin, pocket.spacing, pocket.anchors, mask)
        if getattr(pocket, "receptor_xyz", None) is not None and getattr(pocket, "type_radius", None) is not None:
            r = pocket.receptor()
            N.ligate_pocket_set_receptor(self.h, r["xyz"], r["type"], r["radius"], r["eps"], r["cutoff"],
                                         r["cap"], r["rmin"])

    def close(self):
        if getattr(self, "h", None):
            N.ligate_pocket_destroy(self.h)
            self.h = None

    __del__ = close


class BatchHandle:
    def __init__(self, ligands):
        self.n = ligands.n
        self.h = N.ligate_batch_create(ligands)

    def close(self):
        if getattr(self, "h", None):
            N.ligate_batch_destroy(self.h)
            self.h = None

    __del__ = close


MODES = {
    "fp32": (N.LIGATE_FP32, N.LIGATE_LAYOUT_PLAIN),
    "fp32c": (N.LIGATE_FP32, N.LIGATE_LAYOUT_CORNER),
    "bf16": (N.LIGATE_BF16, N.LIGATE_LAYOUT_CORNER),
    "fp16": (N.LIGATE_FP16, N.LIGATE_LAYOUT_CORNER),
}


class Plan:
    def __init__(self, pocket: PocketHandle, batch: BatchHandle, sampling, mode="fp32", rescore=None,
                 tile=None, top_k=None, subset=None):
        prec, layout = MODES[mode]
        if rescore is None:
            rescore = prec != N.LIGATE_FP32
        self.s = N.make_sampling(sampling, prec, layout, rescore, top_k)
        self.k = self.s.top_k
        self.n = batch.n
        self._refs = (pocket, batch)
        if subset is None:
            self.h = N.ligate_plan_create(pocket.h, batch.h, self.s, tile)
        else:
            self.n = len(subset)
            self.h = N.ligate_plan_create_subset(pocket.h, batch.h, self.s, subset, tile)
        self.rows = self.n  # rows of the last run

    def run(self, stream=None):
        N.ligate_plan_run(self.h, None, stream)
        self.rows = self.n

    def result(self, stream=None) -> np.ndarray:
        out = np.zeros((self.n, self.k), N.POSE_DTYPE)
        N.ligate_plan_run(self.h, out, stream)
        self.rows = self.n
        return out

    def output(self) -> np.ndarray:
        """The last run's poses (rows of the last run), copied from the
        plan's device buffer without running again."""
        import torch
        out = np.zeros((self.rows, self.k), N.POSE_DTYPE)
        torch.cuda.synchronize()
        if out.nbytes:
            view = torch.as_tensor(_DeviceBytes(self.device_output(), out.nbytes), device="cuda")
            out.reshape(-1).view(np.uint8)[:] = view.cpu().numpy()
        return out

    def run_subset(self, ligands, n_sel=None, stream=None, result=False):
        """Dock a device-chosen selection of this plan's ligands
        (ligate_plan_run_subset): ligands is a CUDA int32 tensor (or a host
        array, uploaded); with result=True returns POSE_DTYPE [n_sel, K]."""
        import torch
        if isinstance(ligands, np.ndarray):
            ligands = torch.from_numpy(np.ascontiguousarray(ligands, np.int32)).cuda()
        n_sel = int(ligands.numel()) if n_sel is None else int(n_sel)
        out = np.zeros((n_sel, self.k), N.POSE_DTYPE) if result else None
        N.ligate_plan_run_subset(self.h, ligands, n_sel, out, stream)
        self.rows = n_sel
        return out

    def refine(self, iterations=32, eta0=0.1, stream=None) -> np.ndarray:
        """Gradient-descent refinement of every pose of the last run
        (ligate_plan_refine); returns REFINED_DTYPE [n, K] on the host."""
        import torch
        buf = torch.empty(self.rows * self.k * N.REFINED_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        N.ligate_plan_refine(self.h, iterations, eta0, buf, stream)
        torch.cuda.synchronize()
        return buf.cpu().numpy().view(N.REFINED_DTYPE).reshape(self.rows, self.k)

    def rescore_exact(self, stream=None) -> np.ndarray:
        """Exact receptor term + clash and the filter flags of every pose of
        the last run (ligate_plan_rescore); RESCORED_DTYPE [n, K] on the host."""
        import torch
        buf = torch.empty(self.rows * self.k * N.RESCORED_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        N.ligate_plan_rescore(self.h, buf, stream)
        torch.cuda.synchronize()
        return buf.cpu().numpy().view(N.RESCORED_DTYPE).reshape(self.rows, self.k)

    def best_passing(self, rescored, stream=None):
        """Per ligand the slot of its lowest-energy pose that passes the
        filter (-1 if none) and that energy (+inf if none), from rescored
        records of this plan's poses (RESCORED_DTYPE [n, K], host array or a
        CUDA byte tensor), by ligate_plan_best_passing."""
        import torch
        buf = _device_bytes(rescored)
        idx = torch.empty(max(self.rows, 1), dtype=torch.int32, device="cuda")
        en = torch.empty(max(self.rows, 1), dtype=torch.float32, device="cuda")
        N.ligate_plan_best_passing(self.h, buf, idx, en, stream)
        torch.cuda.synchronize()
        return idx[:self.rows].cpu().numpy(), en[:self.rows].cpu().numpy()

    def device_output(self) -> int:
        """Device address of the last run's ligate_pose[n][K] result."""
        return N.ligate_plan_output(self.h)

    def tile(self):
        return N.ligate_plan_get_tile(self.h)

    def work(self):
        return N.ligate_plan_work(self.h)

    def best_quantile(self, frac, out, stream=None):
        """k-th smallest best score of the last run into DEVICE out[0]."""
        N.ligate_plan_best_quantile(self.h, frac, out, stream)

    def set_cutoff(self, cutoff):
        """Screening cutoff for later runs: DEVICE tensor of one float, or None."""
        self._cutoff = cutoff  # kept alive while attached
        N.ligate_plan_set_cutoff(self.h, cutoff)

    def close(self):
        if getattr(self, "h", None):
            N.ligate_plan_destroy(self.h)
            self.h = None

    __del__ = close


def dock(pocket, ligands, sampling, mode="fp32", rescore=None, tile=None, top_k=None):
    """One-shot docking of a workload on the current CUDA device."""
    ph = PocketHandle(pocket)
    bh = BatchHandle(ligands)
    pl = Plan(ph, bh, sampling, mode, rescore, tile, top_k)
    try:
        return pl.result()
    finally:
        pl.close()
        bh.close()
        ph.close()


def _device_bytes(a):
    """A CUDA byte view of a structured host array (copied) or a CUDA tensor."""
    import torch
    if isinstance(a, np.ndarray):
        return torch.from_numpy(np.ascontiguousarray(a).reshape(-1).view(np.uint8)).cuda()
    return a


class _DeviceBytes:
    """A device byte range (pointer, size) seen through the CUDA array
    interface, so torch can copy it without owning it."""

    def __init__(self, ptr, nbytes):
        self.__cuda_array_interface__ = {"shape": (int(nbytes),), "typestr": "|u1", "data": (int(ptr), False),
                                         "version": 3, "strides": None}

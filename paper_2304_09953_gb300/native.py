"""Thin ctypes binding of libligate.so (include/ligate.h), same names.

Argument marshalling only: every docking and network step runs in the
library's CUDA kernels.  Device buffers are passed as raw pointers (for
example ``tensor.data_ptr()`` of a CUDA torch tensor) and streams as
``cudaStream_t`` integers (``torch.cuda.Stream().cuda_stream``).  Loading
fails loudly when the library has not been built: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

LIGATE_OK = 0
LIGATE_ERR_INVALID = -1
LIGATE_ERR_OOM = -2
LIGATE_ERR_CUDA = -3
LIGATE_ERR_TIMEOUT = -4
LIGATE_ERR_UNSUPPORTED = -5
LIGATE_FP32, LIGATE_BF16, LIGATE_FP16 = 0, 1, 2
LIGATE_LAYOUT_PLAIN, LIGATE_LAYOUT_CORNER = 0, 1
LIGATE_POCKET_FP32_CORNER, LIGATE_POCKET_BF16_CORNER, LIGATE_POCKET_FP16_CORNER = 1, 2, 4
LIGATE_MAX_ATOMS, LIGATE_MAX_ROT, LIGATE_MAX_STEPS, LIGATE_MAX_TOPK = 128, 16, 32, 32
LIGATE_N_BUCKETS = 8
LIGATE_SURROGATE_PARAMS = 256 * 512 + 512 + 512 * 512 + 512 + 512 * 512 + 512 + 512 + 1

P = ctypes.c_void_p


class ligate_ligands(ctypes.Structure):
    _fields_ = [("n_ligands", ctypes.c_int), ("atom_offset", P), ("xyz", P), ("type", P),
                ("bond_offset", P), ("bonds", P), ("rotatable", P)]


class ligate_batch_info(ctypes.Structure):
    _fields_ = [("n_ligands", ctypes.c_int), ("max_atoms", ctypes.c_int), ("max_rot", ctypes.c_int),
                ("total_atoms", ctypes.c_int64)]


class ligate_sampling(ctypes.Structure):
    _fields_ = [("n_orient", ctypes.c_int), ("n_anchor", ctypes.c_int),
                ("torsion_steps", ctypes.c_int), ("top_k", ctypes.c_int), ("orientations", P),
                ("clash_weight", ctypes.c_float), ("clash_cutoff", ctypes.c_float),
                ("penalty", ctypes.c_float), ("precision", ctypes.c_int), ("layout", ctypes.c_int),
                ("rescore_fp32", ctypes.c_int)]


class ligate_pose(ctypes.Structure):
    _fields_ = [("score", ctypes.c_float), ("start_id", ctypes.c_int32),
                ("tors", ctypes.c_uint8 * LIGATE_MAX_ROT)]


POSE_DTYPE = np.dtype([("score", np.float32), ("start_id", np.int32), ("tors", np.uint8, (16,))])
assert POSE_DTYPE.itemsize == ctypes.sizeof(ligate_pose) == 24
LIGATE_REFINE_MAX_ITERS = 32
LIGATE_GRAD_DIM = 6 + 16
# ligate_pose_state and ligate_refined (include/ligate.h)
STATE_DTYPE = np.dtype([("rot", np.float32, (9,)), ("trans", np.float32, (3,)), ("tors", np.float32, (16,))])
REFINED_DTYPE = np.dtype([("state", STATE_DTYPE), ("score_in", np.float32), ("score", np.float32),
                          ("accepted", np.uint32), ("ligand", np.int32)])
assert STATE_DTYPE.itemsize == 112 and REFINED_DTYPE.itemsize == 128
RESCORED_DTYPE = np.dtype([("energy", np.float32), ("e_inter", np.float32), ("e_clash", np.float32),
                           ("n_outside", np.int32), ("n_capped", np.int32), ("pass", np.int32)])


class ligate_tile(ctypes.Structure):
    _fields_ = [("warps_per_cta", ctypes.c_int), ("ctas_per_sm", ctypes.c_int),
                ("starts_per_item", ctypes.c_int * LIGATE_N_BUCKETS), ("reg_cap", ctypes.c_int)]


class ligate_work(ctypes.Structure):
    _fields_ = [("poses", ctypes.c_double), ("atom_evals", ctypes.c_double),
                ("pair_evals", ctypes.c_double), ("starts", ctypes.c_double),
                ("done_atom_evals", ctypes.c_double), ("done_pair_tests", ctypes.c_double),
                ("done_pair_survivors", ctypes.c_double), ("done_pair_evals", ctypes.c_double),
                ("done_pruned_starts", ctypes.c_double), ("done_bond_sweeps", ctypes.c_double)]


# name -> (restype, argtypes)
_SIGS = {
    "ligate_last_error": (ctypes.c_char_p, []),
    "ligate_version": (ctypes.c_char_p, []),
    "ligate_pocket_create": (ctypes.c_int, [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, P,
                                            ctypes.c_double, P, ctypes.c_int, ctypes.c_uint, P]),
    "ligate_pocket_destroy": (None, [P]),
    "ligate_probe_gather": (ctypes.c_int, [P, ctypes.c_int, P]),
    "ligate_batch_create": (ctypes.c_int, [P, P]),
    "ligate_batch_destroy": (None, [P]),
    "ligate_batch_get_info": (ctypes.c_int, [P, P]),
    "ligate_batch_rot_counts": (ctypes.c_int, [P, P]),
    "ligate_plan_create": (ctypes.c_int, [P, P, P, P, P]),
    "ligate_plan_create_subset": (ctypes.c_int, [P, P, P, P, P, ctypes.c_int, P]),
    "ligate_plan_run": (ctypes.c_int, [P, P, P]),
    "ligate_plan_run_subset": (ctypes.c_int, [P, P, ctypes.c_int, P, P]),
    "ligate_plan_output": (ctypes.c_int, [P, P]),
    "ligate_plan_best_scores": (ctypes.c_int, [P, P, ctypes.c_int, ctypes.c_int, P]),
    "ligate_plan_best_quantile": (ctypes.c_int, [P, ctypes.c_double, P, P]),
    "ligate_plan_set_cutoff": (ctypes.c_int, [P, P]),
    "ligate_plan_get_tile": (ctypes.c_int, [P, P, P]),
    "ligate_plan_work": (ctypes.c_int, [P, P]),
    "ligate_plan_destroy": (None, [P]),
    "ligate_dock_batch": (ctypes.c_int, [P, P, P, P, P]),
    "ligate_dock_noalloc": (ctypes.c_int, [P, P, P, P, P]),
    "ligate_score_poses": (ctypes.c_int, [P, P, P, ctypes.c_int, P, P, P, P, P]),
    "ligate_pose_coords": (ctypes.c_int, [P, P, P, ctypes.c_int, P, P, P, P, P]),
    "ligate_state_coords": (ctypes.c_int, [P, P, P, ctypes.c_int, P, P, P, P]),
    "ligate_autotune": (ctypes.c_int, [P, P, P, ctypes.c_double, P]),
    "ligate_model_tile": (ctypes.c_int, [P, P, P, P]),
    "ligate_descriptors": (ctypes.c_int, [P, P, P]),
    "ligate_surrogate_create": (ctypes.c_int, [P, ctypes.c_uint64, P]),
    "ligate_surrogate_destroy": (None, [P]),
    "ligate_surrogate_train": (ctypes.c_int, [P, P, P, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                              ctypes.c_float, ctypes.c_uint64, P, P]),
    "ligate_surrogate_predict": (ctypes.c_int, [P, P, ctypes.c_int, P, P]),
    "ligate_inspect_ligand": (ctypes.c_int, [P, ctypes.c_int, P, P, P, P, P, ctypes.c_int, P]),
    "ligate_surrogate_rank": (ctypes.c_int, [P, P, ctypes.c_int, ctypes.c_double, P, P, P]),
    "ligate_surrogate_rank_ensemble": (ctypes.c_int, [P, ctypes.c_int, P, ctypes.c_int, ctypes.c_double, P, P,
                                                      P]),
    "ligate_surrogate_grad": (ctypes.c_int, [P, P, P, ctypes.c_int, P, P, P]),
    "ligate_surrogate_get_weights": (ctypes.c_int, [P, P]),
    "ligate_surrogate_engine": (ctypes.c_int, [P]),
    "ligate_surrogate_save": (ctypes.c_int, [P, ctypes.c_char_p]),
    "ligate_surrogate_load": (ctypes.c_int, [ctypes.c_char_p, P]),
    "ligate_debug_inject_fault": (ctypes.c_int, [ctypes.c_int]),
    "ligate_pose_gradient": (ctypes.c_int, [P, P, P, ctypes.c_int, P, P, P, P, P]),
    "ligate_refine_states": (ctypes.c_int, [P, P, P, ctypes.c_int, P, P, ctypes.c_int, ctypes.c_float, P, P]),
    "ligate_plan_refine": (ctypes.c_int, [P, ctypes.c_int, ctypes.c_float, P, P]),
    "ligate_pocket_set_receptor": (ctypes.c_int, [P, P, P, ctypes.c_int, P, P, ctypes.c_int, ctypes.c_float,
                                                  ctypes.c_float, ctypes.c_float]),
    "ligate_rescore_poses": (ctypes.c_int, [P, P, P, ctypes.c_int, P, P, P, P, P]),
    "ligate_plan_rescore": (ctypes.c_int, [P, P, P]),
    "ligate_rescore_states": (ctypes.c_int, [P, P, P, ctypes.c_int, P, P, P, P]),
    "ligate_plan_rescore_refined": (ctypes.c_int, [P, P, P, P]),
    "ligate_pose_features": (ctypes.c_int, [P, P, P, ctypes.c_int, P, P, P, P, P]),
    "ligate_plan_pose_features": (ctypes.c_int, [P, P, P]),
    "ligate_plan_best_passing": (ctypes.c_int, [P, P, P, P, P]),
    "ligate_select_poses": (ctypes.c_int, [P, P, ctypes.c_int, ctypes.c_int, ctypes.c_float, P, P]),
    "ligate_selector_labels": (ctypes.c_int, [P, ctypes.c_int64, ctypes.c_float, P, P]),
}

_lib = None


def library_path() -> str:
    return _build.SO


def load(build_if_missing: bool = True):
    """Load libligate.so (building it first if asked); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.SO):
        if not build_if_missing:
            raise RuntimeError(f"{_build.SO} is not built; run paper_2304_09953_gb300.build.build()")
        _build.build()
    lib = ctypes.CDLL(_build.SO)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    return list(_SIGS)


class LigateError(RuntimeError):
    def __init__(self, status, where):
        msg = load().ligate_last_error().decode(errors="replace")
        super().__init__(f"{where} failed ({status}): {msg}")
        self.status = status


def check(status, where=""):
    if status != LIGATE_OK:
        raise LigateError(status, where)
    return status


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"], "arrays must be C-contiguous"
        return a.ctypes.data
    return int(a.data_ptr())  # torch tensor


# --- thin wrappers with the C names -----------------------------------------
def ligate_pocket_create(maps, origin, spacing, anchors, precision_mask):
    lib = load()
    maps = np.ascontiguousarray(maps, np.float32)
    T, nz, ny, nx = maps.shape
    org = (ctypes.c_double * 3)(*[float(v) for v in origin])
    anchors = np.ascontiguousarray(anchors, np.float32)
    h = P()
    check(lib.ligate_pocket_create(maps.ctypes.data, T, nx, ny, nz, ctypes.addressof(org),
                                   float(spacing), anchors.ctypes.data, len(anchors),
                                   int(precision_mask), ctypes.byref(h)), "ligate_pocket_create")
    return h


def ligate_pocket_destroy(h):
    load().ligate_pocket_destroy(h)


def make_ligands_struct(lig):
    """ligate_ligands over a workload.Ligands (arrays must stay alive)."""
    keep = [np.ascontiguousarray(lig.atom_offset, np.int32), np.ascontiguousarray(lig.xyz, np.float32),
            np.ascontiguousarray(lig.type, np.uint8), np.ascontiguousarray(lig.bond_offset, np.int32),
            np.ascontiguousarray(lig.bonds, np.int32), np.ascontiguousarray(lig.rotatable, np.uint8)]
    s = ligate_ligands(lig.n, *[k.ctypes.data for k in keep])
    s._keep = keep
    return s


def ligate_batch_create(lig):
    lib = load()
    s = make_ligands_struct(lig)
    h = P()
    check(lib.ligate_batch_create(ctypes.byref(s), ctypes.byref(h)), "ligate_batch_create")
    return h


def ligate_batch_destroy(h):
    load().ligate_batch_destroy(h)


def ligate_inspect_ligand(lig, li):
    """Host-only packing of ligand li: (order, bonds [n_rot][8], candidates)."""
    lib = load()
    s = make_ligands_struct(lig)
    na, nr, nc = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    order = np.zeros(LIGATE_MAX_ATOMS, np.int32)
    bonds = np.zeros((LIGATE_MAX_ROT, 8), np.int32)
    check(lib.ligate_inspect_ligand(ctypes.byref(s), int(li), ctypes.byref(na), order.ctypes.data,
                                    ctypes.byref(nr), bonds.ctypes.data, None, 0, ctypes.byref(nc)),
          "ligate_inspect_ligand")
    cand = np.zeros(max(nc.value, 1), np.uint16)
    check(lib.ligate_inspect_ligand(ctypes.byref(s), int(li), ctypes.byref(na), None, ctypes.byref(nr), None,
                                    cand.ctypes.data, len(cand), ctypes.byref(nc)), "ligate_inspect_ligand")
    return order[:na.value].copy(), bonds[:nr.value].copy(), cand[:nc.value].copy()


def ligate_batch_get_info(h):
    info = ligate_batch_info()
    check(load().ligate_batch_get_info(h, ctypes.byref(info)), "ligate_batch_get_info")
    return info


def ligate_batch_rot_counts(h, n):
    out = np.zeros(n, np.int32)
    check(load().ligate_batch_rot_counts(h, out.ctypes.data), "ligate_batch_rot_counts")
    return out


def make_sampling(sampling, precision=LIGATE_FP32, layout=LIGATE_LAYOUT_PLAIN, rescore=False,
                  top_k=None):
    q = np.ascontiguousarray(sampling.quats, np.float64)
    s = ligate_sampling(q.shape[0], int(sampling.n_anchor), int(sampling.torsion_steps),
                        int(sampling.top_k if top_k is None else top_k), q.ctypes.data,
                        float(sampling.clash_weight), float(sampling.clash_cutoff),
                        float(sampling.penalty), int(precision), int(layout), int(bool(rescore)))
    s._keep = q
    return s


def ligate_plan_create(pocket, batch, sampling_struct, tile=None):
    h = P()
    check(load().ligate_plan_create(pocket, batch, ctypes.byref(sampling_struct),
                                    ctypes.byref(tile) if tile is not None else None,
                                    ctypes.byref(h)), "ligate_plan_create")
    return h


def ligate_plan_create_subset(pocket, batch, sampling_struct, ligands, tile=None):
    h = P()
    sel = np.ascontiguousarray(ligands, np.int32)
    check(load().ligate_plan_create_subset(pocket, batch, ctypes.byref(sampling_struct),
                                           ctypes.byref(tile) if tile is not None else None,
                                           sel.ctypes.data, len(sel), ctypes.byref(h)),
          "ligate_plan_create_subset")
    return h


def ligate_plan_run(plan, out=None, stream=None):
    check(load().ligate_plan_run(plan, _ptr(out), stream), "ligate_plan_run")


def ligate_plan_output(plan):
    p = P()
    check(load().ligate_plan_output(plan, ctypes.byref(p)), "ligate_plan_output")
    return p.value


def ligate_plan_get_tile(plan):
    t = ligate_tile()
    n = ctypes.c_int()
    check(load().ligate_plan_get_tile(plan, ctypes.byref(t), ctypes.byref(n)), "ligate_plan_get_tile")
    return t, n.value


def ligate_plan_work(plan):
    w = ligate_work()
    check(load().ligate_plan_work(plan, ctypes.byref(w)), "ligate_plan_work")
    return w


def ligate_plan_destroy(plan):
    load().ligate_plan_destroy(plan)


def ligate_dock_batch(pocket, lig, sampling_struct, out: np.ndarray, stream=None):
    s = make_ligands_struct(lig)
    check(load().ligate_dock_batch(pocket, ctypes.byref(s), ctypes.byref(sampling_struct),
                                   _ptr(out), stream), "ligate_dock_batch")


def ligate_dock_noalloc(pocket, batch, sampling_struct, out, stream=None):
    """Allocation-free docking run into DEVICE `out` (enqueue only)."""
    check(load().ligate_dock_noalloc(pocket, batch, ctypes.byref(sampling_struct), _ptr(out), stream),
          "ligate_dock_noalloc")


def ligate_score_poses(pocket, batch, sampling_struct, n, lig_idx, start_id, tors, out, stream=None):
    check(load().ligate_score_poses(pocket, batch, ctypes.byref(sampling_struct), int(n), _ptr(lig_idx),
                                    _ptr(start_id), _ptr(tors), _ptr(out), stream), "ligate_score_poses")


def ligate_pose_coords(pocket, batch, sampling_struct, n, lig_idx, start_id, tors, out, stream=None):
    """out: DEVICE float32 [n][LIGATE_MAX_ATOMS][3], grid units, input atom order."""
    check(load().ligate_pose_coords(pocket, batch, ctypes.byref(sampling_struct), int(n), _ptr(lig_idx),
                                    _ptr(start_id), _ptr(tors), _ptr(out), stream), "ligate_pose_coords")


def ligate_state_coords(pocket, batch, sampling_struct, n, lig_idx, states, out, stream=None):
    """states: DEVICE ligate_pose_state[n]; out: DEVICE float32 [n][LIGATE_MAX_ATOMS][3], Angstrom."""
    check(load().ligate_state_coords(pocket, batch, ctypes.byref(sampling_struct), int(n), _ptr(lig_idx),
                                     _ptr(states), _ptr(out), stream), "ligate_state_coords")


def ligate_pose_gradient(pocket, batch, sampling_struct, n, lig_idx, states, energy, grad, stream=None):
    """states: DEVICE ligate_pose_state[n] (e.g. a uint8 tensor of n * 112 bytes)."""
    check(load().ligate_pose_gradient(pocket, batch, ctypes.byref(sampling_struct), int(n), _ptr(lig_idx),
                                      _ptr(states), _ptr(energy), _ptr(grad), stream), "ligate_pose_gradient")


def ligate_refine_states(pocket, batch, sampling_struct, n, lig_idx, init, iterations, eta0, out,
                         stream=None):
    check(load().ligate_refine_states(pocket, batch, ctypes.byref(sampling_struct), int(n), _ptr(lig_idx),
                                      _ptr(init), int(iterations), float(eta0), _ptr(out), stream),
          "ligate_refine_states")


def ligate_plan_refine(plan, iterations, eta0, out, stream=None):
    check(load().ligate_plan_refine(plan, int(iterations), float(eta0), _ptr(out), stream),
          "ligate_plan_refine")


def ligate_pocket_set_receptor(pocket, xyz, type_, radius, eps, cutoff, cap, rmin):
    xyz = np.ascontiguousarray(xyz, np.float32)
    type_ = np.ascontiguousarray(type_, np.int32)
    radius = np.ascontiguousarray(radius, np.float32)
    eps = np.ascontiguousarray(eps, np.float32)
    check(load().ligate_pocket_set_receptor(pocket, xyz.ctypes.data, type_.ctypes.data, len(type_),
                                            radius.ctypes.data, eps.ctypes.data, len(radius), float(cutoff),
                                            float(cap), float(rmin)), "ligate_pocket_set_receptor")


def ligate_rescore_poses(pocket, batch, sampling_struct, n, lig_idx, start_id, tors, out, stream=None):
    check(load().ligate_rescore_poses(pocket, batch, ctypes.byref(sampling_struct), int(n), _ptr(lig_idx),
                                      _ptr(start_id), _ptr(tors), _ptr(out), stream), "ligate_rescore_poses")


def ligate_plan_rescore(plan, out, stream=None):
    check(load().ligate_plan_rescore(plan, _ptr(out), stream), "ligate_plan_rescore")


def ligate_pose_features(pocket, batch, sampling_struct, n, lig_idx, start_id, tors, out, stream=None):
    check(load().ligate_pose_features(pocket, batch, ctypes.byref(sampling_struct), int(n), _ptr(lig_idx),
                                      _ptr(start_id), _ptr(tors), _ptr(out), stream), "ligate_pose_features")


def ligate_plan_pose_features(plan, out, stream=None):
    check(load().ligate_plan_pose_features(plan, _ptr(out), stream), "ligate_plan_pose_features")


def ligate_rescore_states(pocket, batch, sampling_struct, n, lig_idx, states, out, stream=None):
    check(load().ligate_rescore_states(pocket, batch, ctypes.byref(sampling_struct), int(n), _ptr(lig_idx),
                                       _ptr(states), _ptr(out), stream), "ligate_rescore_states")


def ligate_plan_rescore_refined(plan, refined, out, stream=None):
    check(load().ligate_plan_rescore_refined(plan, _ptr(refined), _ptr(out), stream),
          "ligate_plan_rescore_refined")


def ligate_plan_best_scores(plan, out, stride, column, stream=None):
    check(load().ligate_plan_best_scores(plan, _ptr(out), int(stride), int(column), stream),
          "ligate_plan_best_scores")


def ligate_plan_best_quantile(plan, frac, out, stream=None):
    """k-th smallest best score of the last run (k = ceil(frac rows)) into DEVICE out[0]."""
    check(load().ligate_plan_best_quantile(plan, float(frac), _ptr(out), stream), "ligate_plan_best_quantile")


def ligate_plan_set_cutoff(plan, cutoff):
    """Attach a DEVICE cutoff (one float) to a plan's runs; None detaches it."""
    check(load().ligate_plan_set_cutoff(plan, _ptr(cutoff)), "ligate_plan_set_cutoff")


def ligate_autotune(pocket, batch, sampling_struct, budget_ms=20000.0):
    t = ligate_tile()
    check(load().ligate_autotune(pocket, batch, ctypes.byref(sampling_struct), float(budget_ms),
                                 ctypes.byref(t)), "ligate_autotune")
    return t


def ligate_model_tile(pocket, batch, sampling_struct):
    t = ligate_tile()
    check(load().ligate_model_tile(pocket, batch, ctypes.byref(sampling_struct), ctypes.byref(t)),
          "ligate_model_tile")
    return t


def ligate_descriptors(batch, out, stream=None):
    check(load().ligate_descriptors(batch, _ptr(out), stream), "ligate_descriptors")


def ligate_surrogate_create(init_weights=None, seed=0):
    h = P()
    w = None if init_weights is None else np.ascontiguousarray(init_weights, np.float32)
    check(load().ligate_surrogate_create(_ptr(w), int(seed), ctypes.byref(h)), "ligate_surrogate_create")
    return h


def ligate_surrogate_destroy(h):
    load().ligate_surrogate_destroy(h)


def ligate_surrogate_train(h, desc, labels, n, epochs, batch, lr, seed, stream=None):
    loss = ctypes.c_float()
    check(load().ligate_surrogate_train(h, _ptr(desc), _ptr(labels), int(n), int(epochs), int(batch),
                                        float(lr), int(seed), ctypes.byref(loss), stream),
          "ligate_surrogate_train")
    return loss.value


def ligate_surrogate_predict(h, desc, n, pred, stream=None):
    check(load().ligate_surrogate_predict(h, _ptr(desc), int(n), _ptr(pred), stream),
          "ligate_surrogate_predict")


def ligate_surrogate_rank(h, desc, n, keep_frac, idx_out, pred_out=None, stream=None):
    check(load().ligate_surrogate_rank(h, _ptr(desc), int(n), float(keep_frac), _ptr(idx_out),
                                       _ptr(pred_out), stream), "ligate_surrogate_rank")


def ligate_surrogate_rank_ensemble(hs, desc, n, keep_frac, idx_out, pred_out=None, stream=None):
    arr = (ctypes.c_void_p * len(hs))(*hs)
    check(load().ligate_surrogate_rank_ensemble(arr, len(hs), _ptr(desc), int(n), float(keep_frac),
                                                _ptr(idx_out), _ptr(pred_out), stream),
          "ligate_surrogate_rank_ensemble")


def ligate_surrogate_grad(h, x, t, b, grad, stream=None):
    loss = ctypes.c_float()
    check(load().ligate_surrogate_grad(h, _ptr(x), _ptr(t), int(b), _ptr(grad), ctypes.byref(loss),
                                       stream), "ligate_surrogate_grad")
    return loss.value


def ligate_surrogate_get_weights(h):
    out = np.zeros(LIGATE_SURROGATE_PARAMS, np.float32)
    check(load().ligate_surrogate_get_weights(h, out.ctypes.data), "ligate_surrogate_get_weights")
    return out


def ligate_surrogate_engine(h):
    """1: tcgen05 contractions, 0: mma.sync (LIGATE_MLP_GEMM=mma at creation)."""
    return int(load().ligate_surrogate_engine(h))


def ligate_debug_inject_fault(kind):
    """Test hook: see include/ligate.h."""
    check(load().ligate_debug_inject_fault(int(kind)), "ligate_debug_inject_fault")


def ligate_surrogate_save(h, path):
    check(load().ligate_surrogate_save(h, str(path).encode()), "ligate_surrogate_save")


def ligate_surrogate_load(path):
    h = ctypes.c_void_p()
    check(load().ligate_surrogate_load(str(path).encode(), ctypes.byref(h)), "ligate_surrogate_load")
    return h


def ligate_plan_best_passing(plan, rescored, idx_out, energy_out=None, stream=None):
    """rescored: DEVICE RESCORED_DTYPE [n][K]; idx_out DEVICE int32 [n]; energy_out DEVICE float32 [n]."""
    check(load().ligate_plan_best_passing(plan, _ptr(rescored), _ptr(idx_out), _ptr(energy_out), stream),
          "ligate_plan_best_passing")


def ligate_select_poses(pred, poses, n, k, pass_below, idx_out, stream=None):
    """pred DEVICE float32 [n][k]; poses DEVICE POSE_DTYPE [n][k]; idx_out DEVICE int32 [n]."""
    check(load().ligate_select_poses(_ptr(pred), _ptr(poses), int(n), int(k), float(pass_below), _ptr(idx_out),
                                     stream), "ligate_select_poses")


def ligate_selector_labels(rescored, n, fail_label, out, stream=None):
    """rescored DEVICE RESCORED_DTYPE [n]; out DEVICE float32 [n]."""
    check(load().ligate_selector_labels(_ptr(rescored), int(n), float(fail_label), _ptr(out), stream),
          "ligate_selector_labels")


def ligate_probe_gather(pocket, precision):
    """Measured GB/s of random corner-cell gathers over the pocket's maps."""
    v = ctypes.c_double()
    check(load().ligate_probe_gather(pocket, int(precision), ctypes.byref(v)), "ligate_probe_gather")
    return v.value


def ligate_plan_run_subset(plan, ligands, n_sel, out=None, stream=None):
    """ligands: DEVICE int32 [n_sel] batch indices; out: optional host/device POSE_DTYPE [n_sel][K]."""
    check(load().ligate_plan_run_subset(plan, _ptr(ligands), int(n_sel), _ptr(out), stream),
          "ligate_plan_run_subset")

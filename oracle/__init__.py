"""FP64 CPU oracle for the ligand dock+score hot path and its surrogate MLP.

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the timed CPU
baseline of ``bench.py`` may import this package; the library itself never
does.  It shares no code with the CUDA path and imports nothing from it:
inputs arrive as plain numpy arrays (or any object with the same attribute
names as the synthetic-workload dataclasses).

The docking functions wrap ``ligate_oracle.c`` (plain C, FP64, OpenMP over
starts); the network functions live in ``oracle.mlp`` (numpy FP64).  See the
header of ``ligate_oracle.c`` for the method definition each function follows
(paper Sec. 2: multi-restart docking, geometric score, ligand score = best
pose; Sec. 3.5: affinity prediction from ligand features).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ligate_oracle.c")
_OUT = os.path.join(_HERE, "_lib")
_SO = os.path.join(_OUT, "libligate_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    os.makedirs(_OUT, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class _Lig(ctypes.Structure):
    _fields_ = [("n_atoms", ctypes.c_int), ("xyz", ctypes.c_void_p), ("type", ctypes.c_void_p),
                ("n_bonds", ctypes.c_int), ("bonds", ctypes.c_void_p), ("rot", ctypes.c_void_p)]


class _Samp(ctypes.Structure):
    _fields_ = [("n_orient", ctypes.c_int), ("n_anchor", ctypes.c_int), ("S", ctypes.c_int),
                ("quat", ctypes.c_void_p), ("anchors", ctypes.c_void_p),
                ("clash_w", ctypes.c_double), ("clash_dc", ctypes.c_double),
                ("clash_min_sep", ctypes.c_int), ("penalty", ctypes.c_double)]


class _Rec(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("xyz", ctypes.c_void_p), ("type", ctypes.c_void_p),
                ("n_types", ctypes.c_int), ("radius", ctypes.c_void_p), ("eps", ctypes.c_void_p),
                ("cutoff", ctypes.c_double), ("cap", ctypes.c_double), ("rmin", ctypes.c_double)]


class _Pock(ctypes.Structure):
    _fields_ = [("maps", ctypes.c_void_p), ("n_types", ctypes.c_int), ("nx", ctypes.c_int),
                ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("origin", ctypes.c_double * 3),
                ("h", ctypes.c_double)]


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        lib.or_quat_to_matrix.argtypes = [P, P]
        lib.or_ligand_bonds.argtypes = [P, P, P]
        lib.or_topo_distance.argtypes = [P, P]
        lib.or_pose_coords.argtypes = [P, P, I, P, P, I, P]
        lib.or_torsions_in_order.argtypes = [P, P, P, P]
        lib.or_trilinear.argtypes = [P, D, I, I, P, P]
        lib.or_trilinear.restype = None
        lib.or_score_coords.argtypes = [P, P, P, P, P]
        lib.or_score_poses.argtypes = [P, P, P, I, P, P, I, P, P]
        lib.or_greedy.argtypes = [P, P, P, I, P, P, P, I, P]
        lib.or_exhaustive.argtypes = [P, P, P, I, P, P]
        lib.or_descriptor.argtypes = [P, I, P]
        lib.or_pose_grad.argtypes = [P, P, P, I, P, P, P, P, P, P]
        lib.or_state_coords.argtypes = [P, I, P, P]
        lib.or_refine.argtypes = [P, P, P, I, P, I, D, P, D, P, P, P, P, P, P]
        lib.or_rescore_coords.argtypes = [P, P, P, P, I, P, P, P, P, P, P]
        lib.or_pose_features.argtypes = [P, P, P, I, P, P]
        lib.or_rescore_atoms.argtypes = [P, P, P, I, P, P, P, P]
        _lib = lib
    return _lib


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


class _Keep:
    """Holds numpy arrays alive while a ctypes struct points at them."""

    def __init__(self):
        self.refs = []

    def ptr(self, a):
        self.refs.append(a)
        return a.ctypes.data_as(ctypes.c_void_p).value


def _lig(keep, xyz, typ, bonds, rot):
    xyz = _c(xyz, np.float32)
    return _Lig(len(xyz), keep.ptr(xyz), keep.ptr(_c(typ, np.uint8)), len(bonds),
                keep.ptr(_c(bonds, np.int32)), keep.ptr(_c(rot, np.uint8)))


def _samp(keep, sampling, anchors):
    q = _c(sampling.quats, np.float64)
    a = _c(anchors, np.float32)
    return _Samp(q.shape[0], int(sampling.n_anchor), int(sampling.torsion_steps), keep.ptr(q),
                 keep.ptr(a), float(sampling.clash_weight), float(sampling.clash_cutoff),
                 int(sampling.clash_min_sep), float(sampling.penalty))


def _pock(keep, pocket):
    m = _c(pocket.maps, np.float32)
    t, nz, ny, nx = m.shape
    o = (ctypes.c_double * 3)(*[float(v) for v in pocket.origin])
    return _Pock(keep.ptr(m), t, nx, ny, nz, o, float(pocket.spacing))


def _ref(x):
    return ctypes.byref(x)


# ---------------------------------------------------------------------------
def quat_to_matrix(q) -> np.ndarray:
    lib = _load()
    q = _c(q, np.float64)
    R = np.zeros(9)
    lib.or_quat_to_matrix(q.ctypes.data, R.ctypes.data)
    return R.reshape(3, 3)


def ligand_bonds(lig):
    """Rotatable bonds (u, v) in sweep order (DFS pre-order of the child)."""
    lib = _load()
    k = _Keep()
    L = _lig(k, *lig)
    u = np.zeros(256, np.int32)
    v = np.zeros(256, np.int32)
    r = lib.or_ligand_bonds(_ref(L), u.ctypes.data, v.ctypes.data)
    if r < 0:
        raise ValueError("ligand bonds do not form a tree")
    return u[:r].copy(), v[:r].copy()


def topo_distance(lig) -> np.ndarray:
    lib = _load()
    k = _Keep()
    L = _lig(k, *lig)
    n = L.n_atoms
    out = np.zeros((n, n), np.int32)
    if lib.or_topo_distance(_ref(L), out.ctypes.data):
        raise ValueError("ligand bonds do not form a tree")
    return out


def pose_coords(lig, pocket_anchors, sampling, starts, tors) -> np.ndarray:
    lib = _load()
    k = _Keep()
    L = _lig(k, *lig)
    S = _samp(k, sampling, pocket_anchors)
    starts = _c(starts, np.int32)
    tors = _c(np.atleast_2d(tors), np.int32)
    if tors.shape[1] == 0:
        tors = np.zeros((len(starts), 1), np.int32)
    out = np.zeros((len(starts), L.n_atoms, 3))
    lib.or_pose_coords(_ref(L), _ref(S), len(starts), starts.ctypes.data, tors.ctypes.data,
                       tors.shape[1], out.ctypes.data)
    return out


def torsions_in_order(lig, angles, order) -> np.ndarray:
    lib = _load()
    k = _Keep()
    L = _lig(k, *lig)
    angles = _c(angles, np.float64)
    order = _c(order, np.int32)
    out = np.zeros((L.n_atoms, 3))
    lib.or_torsions_in_order(_ref(L), angles.ctypes.data, order.ctypes.data, out.ctypes.data)
    return out


def trilinear(pocket, t, pts, penalty=10.0) -> np.ndarray:
    lib = _load()
    k = _Keep()
    P = _pock(k, pocket)
    pts = _c(np.atleast_2d(pts), np.float64)
    out = np.zeros(len(pts))
    lib.or_trilinear(_ref(P), float(penalty), int(t), len(pts), pts.ctypes.data, out.ctypes.data)
    return out


def score_coords(lig, pocket, sampling, coords) -> float:
    lib = _load()
    k = _Keep()
    L = _lig(k, *lig)
    P = _pock(k, pocket)
    S = _samp(k, sampling, pocket.anchors)
    coords = _c(coords, np.float64)
    out = ctypes.c_double()
    lib.or_score_coords(_ref(L), _ref(P), _ref(S), coords.ctypes.data, ctypes.byref(out))
    return out.value


def score_poses(lig, pocket, sampling, starts, tors, with_scale: bool = False):
    """FP64 scores of (start, tors) poses; with ``with_scale`` also each
    score's sum of absolute term values (the scale of its rounding error)."""
    lib = _load()
    k = _Keep()
    L = _lig(k, *lig)
    P = _pock(k, pocket)
    S = _samp(k, sampling, pocket.anchors)
    starts = _c(starts, np.int32)
    tors = _c(np.atleast_2d(tors), np.int32)
    if tors.shape[1] == 0:
        tors = np.zeros((len(starts), 1), np.int32)
    out = np.zeros(len(starts))
    mag = np.zeros(len(starts))
    lib.or_score_poses(_ref(L), _ref(P), _ref(S), len(starts), starts.ctypes.data,
                       tors.ctypes.data, tors.shape[1], out.ctypes.data, mag.ctypes.data)
    return (out, mag) if with_scale else out


def greedy(lig, pocket, sampling, starts=None, trials: bool = False):
    """FP64 greedy sweep for each start; returns (E[n], tors[n, R]) and,
    with ``trials``, every trial score [n, R, S]."""
    lib = _load()
    k = _Keep()
    L = _lig(k, *lig)
    P = _pock(k, pocket)
    S = _samp(k, sampling, pocket.anchors)
    if starts is None:
        starts = np.arange(sampling.n_starts)
    starts = _c(starts, np.int32)
    R = int(np.sum(np.asarray(lig[3]) != 0))
    e = np.zeros(len(starts))
    tors = np.zeros((len(starts), max(R, 1)), np.int32)
    tr = np.zeros((len(starts), R, sampling.torsion_steps)) if trials else None
    rc = lib.or_greedy(_ref(L), _ref(P), _ref(S), len(starts), starts.ctypes.data, e.ctypes.data,
                       tors.ctypes.data, tors.shape[1], tr.ctypes.data if trials else None)
    if rc:
        raise ValueError("ligand bonds do not form a tree")
    tors = tors[:, :R]
    return (e, tors, tr) if trials else (e, tors)


def exhaustive(lig, pocket, sampling, starts) -> np.ndarray:
    """Scores of every torsion combination [n_starts, S^R] (bond 0 fastest)."""
    lib = _load()
    k = _Keep()
    L = _lig(k, *lig)
    P = _pock(k, pocket)
    S = _samp(k, sampling, pocket.anchors)
    starts = _c(starts, np.int32)
    R = int(np.sum(np.asarray(lig[3]) != 0))
    out = np.zeros((len(starts), sampling.torsion_steps ** R))
    lib.or_exhaustive(_ref(L), _ref(P), _ref(S), len(starts), starts.ctypes.data, out.ctypes.data)
    return out


def top_k(e, k):
    """Indices of the k smallest (E, start) pairs, best first."""
    e = np.asarray(e)
    order = np.lexsort((np.arange(len(e)), e))
    return order[:k]


def dock_ligand(lig, pocket, sampling, k=None):
    """Full per-ligand docking: greedy over every start, then top-K.
    Returns (scores[K], start_ids[K], tors[K, R])."""
    k = sampling.top_k if k is None else k
    e, tors = greedy(lig, pocket, sampling)
    idx = top_k(e, k)
    return e[idx], idx.astype(np.int32), tors[idx]


def descriptor(lig, n_types: int = 8) -> np.ndarray:
    lib = _load()
    k = _Keep()
    L = _lig(k, *lig)
    out = np.zeros(256)
    if lib.or_descriptor(_ref(L), n_types, out.ctypes.data):
        raise ValueError("descriptor needs 8 atom types")
    return out


# ---------------------------------------------------------------------------
# Pose refinement (see the refinement section of ligate_oracle.c).  A state
# is a row [R (9, row-major), t (3, Angstrom), phi (nrot, radians)].

def docked_state(sampling, anchors, start, tors) -> np.ndarray:
    """State of docked pose (start, tors): R of the start's orientation
    quaternion, t = its anchor, phi_b = 2 pi tors[b] / S."""
    o, a = divmod(int(start), int(sampling.n_anchor))
    R = quat_to_matrix(np.asarray(sampling.quats)[o])
    t = np.asarray(anchors, np.float64)[a]
    phi = 2.0 * np.pi * np.asarray(tors, np.float64) / sampling.torsion_steps
    return np.concatenate([R.reshape(-1), t, phi])


def state_coords(lig, states) -> np.ndarray:
    """Coordinates [n, n_atoms, 3] of state rows [R (9), t (3), phi (nrot)]."""
    lib = _load()
    k = _Keep()
    L = _lig(k, *lig)
    st = _c(np.atleast_2d(states), np.float64)
    out = np.zeros((st.shape[0], L.n_atoms, 3))
    if lib.or_state_coords(_ref(L), st.shape[0], st.ctypes.data, out.ctypes.data):
        raise ValueError("ligand bonds do not form a tree")
    return out


def pose_grad(lig, pocket, sampling, states):
    """E, generalised gradient (F, tau, psi), error scales (of E, then of
    each gradient component), moments (I_R, I_b) and the smallest cell-face
    distance of any atom, for each state row."""
    lib = _load()
    k = _Keep()
    L = _lig(k, *lig)
    P = _pock(k, pocket)
    S = _samp(k, sampling, pocket.anchors)
    st = _c(np.atleast_2d(states), np.float64)
    n, w = st.shape
    nr = w - 12
    e = np.zeros(n)
    g = np.zeros((n, 6 + nr))
    sc = np.zeros((n, 7 + nr))
    inert = np.zeros((n, 1 + nr))
    face = np.zeros(n)
    if lib.or_pose_grad(_ref(L), _ref(P), _ref(S), n, st.ctypes.data, e.ctypes.data, g.ctypes.data,
                        sc.ctypes.data, inert.ctypes.data, face.ctypes.data):
        raise ValueError("ligand bonds do not form a tree")
    return e, g, sc, inert, face


def refine(lig, pocket, sampling, states, iters, eta0, follow=None, tie_rel=1e-4):
    """Gradient-descent refinement of each state row for `iters` iterations.
    With `follow` (accept masks, one per row) the oracle takes those
    decisions and counts the ones that contradict its own beyond a near-tie.
    Returns dict(states, e_in, e_out, own_mask, n_disagree, scale)."""
    lib = _load()
    k = _Keep()
    L = _lig(k, *lig)
    P = _pock(k, pocket)
    S = _samp(k, sampling, pocket.anchors)
    st = _c(np.atleast_2d(states), np.float64)
    n = st.shape[0]
    out = np.zeros_like(st)
    e_in, e_out, scale = np.zeros(n), np.zeros(n), np.zeros(n)
    mask = np.zeros(n, np.uint32)
    dis = np.zeros(n, np.int32)
    fol = None if follow is None else _c(follow, np.uint32)
    rc = lib.or_refine(_ref(L), _ref(P), _ref(S), n, st.ctypes.data, int(iters), float(eta0),
                       None if fol is None else fol.ctypes.data, float(tie_rel), out.ctypes.data,
                       e_in.ctypes.data, e_out.ctypes.data, mask.ctypes.data, dis.ctypes.data,
                       scale.ctypes.data)
    if rc:
        raise ValueError("bad refinement arguments")
    return {"states": out, "e_in": e_in, "e_out": e_out, "own_mask": mask, "n_disagree": dis,
            "scale": scale}


# ---------------------------------------------------------------------------
# Exact rescoring and pose filter (see the rescoring section of ligate_oracle.c).

def rescore_coords(lig, pocket, sampling, receptor, coords):
    """receptor: dict(xyz [m,3] float32, type [m], radius [T], eps [T],
    cutoff, cap, rmin).  coords [n_poses, n_atoms, 3].  Returns dict(e_inter,
    e_clash, n_outside, n_capped, scale)."""
    lib = _load()
    k = _Keep()
    L = _lig(k, *lig)
    P = _pock(k, pocket)
    S = _samp(k, sampling, pocket.anchors)
    rx = _c(receptor["xyz"], np.float32)
    rt = _c(receptor["type"], np.int32)
    rr = _c(receptor["radius"], np.float64)
    re = _c(receptor["eps"], np.float64)
    R = _Rec(len(rx), k.ptr(rx), k.ptr(rt), len(rr), k.ptr(rr), k.ptr(re), float(receptor["cutoff"]),
             float(receptor["cap"]), float(receptor["rmin"]))
    x = _c(coords, np.float64)
    n = x.shape[0]
    ei, ec, sc = np.zeros(n), np.zeros(n), np.zeros(n)
    no, nc = np.zeros(n, np.int32), np.zeros(n, np.int32)
    if lib.or_rescore_coords(_ref(L), _ref(P), _ref(S), _ref(R), n, x.ctypes.data, ei.ctypes.data,
                             ec.ctypes.data, no.ctypes.data, nc.ctypes.data, sc.ctypes.data):
        raise ValueError("ligand bonds do not form a tree")
    return {"e_inter": ei, "e_clash": ec, "n_outside": no, "n_capped": nc, "scale": sc}


def rescore_atoms(lig, pocket, receptor, coords):
    """Per atom of coordinate sets [n_poses, n_atoms, 3]: the uncapped
    receptor sum, the sum of its pair-term magnitudes and the signed
    distance (grid units) to the map box faces, each [n_poses, n_atoms]."""
    lib = _load()
    k = _Keep()
    L = _lig(k, *lig)
    P = _pock(k, pocket)
    rx = _c(receptor["xyz"], np.float32)
    rt = _c(receptor["type"], np.int32)
    rr = _c(receptor["radius"], np.float64)
    re = _c(receptor["eps"], np.float64)
    R = _Rec(len(rx), k.ptr(rx), k.ptr(rt), len(rr), k.ptr(rr), k.ptr(re), float(receptor["cutoff"]),
             float(receptor["cap"]), float(receptor["rmin"]))
    x = _c(coords, np.float64)
    n, na = x.shape[0], x.shape[1]
    s, m, f = np.zeros((n, na)), np.zeros((n, na)), np.zeros((n, na))
    if lib.or_rescore_atoms(_ref(L), _ref(P), _ref(R), n, x.ctypes.data, s.ctypes.data, m.ctypes.data,
                            f.ctypes.data):
        raise ValueError("ligand bonds do not form a tree")
    return s, m, f


def pose_features(lig, pocket, sampling, coords) -> np.ndarray:
    """Per-pose selector features [n_poses, 256] of coordinate sets
    [n_poses, n_atoms, 3] (see the pose-feature section of ligate_oracle.c)."""
    lib = _load()
    k = _Keep()
    L = _lig(k, *lig)
    P = _pock(k, pocket)
    S = _samp(k, sampling, pocket.anchors)
    x = _c(coords, np.float64)
    out = np.zeros((x.shape[0], 256))
    if lib.or_pose_features(_ref(L), _ref(P), _ref(S), x.shape[0], x.ctypes.data, out.ctypes.data):
        raise ValueError("ligand bonds do not form a tree")
    return out


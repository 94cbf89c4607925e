"""Seeded synthetic docking workloads (inputs only).

The paper's workloads (real chemical libraries in SMILES, PDB targets, the
CASF-2016 set; Sec. 2, 3.3, 3.8) are not available here, so every input is a
seeded synthetic stand-in with the shapes of the benchmark configurations:
ligand trees with 3D coordinates, receptor atoms, per-atom-type grid maps,
pocket anchor points and orientation quaternions.

This module holds none of the docking arithmetic; it only draws inputs, which
both the FP64 oracle and the CUDA library consume.  The C generator is built
on first use (or by ``build()``) into ``_lib/libligate_workload.so``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ligate_workload.c")
_OUT_DIR = os.path.join(_HERE, "_lib")
_SO = os.path.join(_OUT_DIR, "libligate_workload.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the generator with gcc (deterministic FP: no contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        P = ctypes.c_void_p
        I, U64, I64, D = ctypes.c_int, ctypes.c_uint64, ctypes.c_int64, ctypes.c_double
        lib.lw_ligand_sizes.argtypes = [U64, I, I, I, I, I, I, P, P]
        lib.lw_ligands.argtypes = [U64, I64, I, I, P, P, P, P, P, P, P, P, P]
        lib.lw_type_params.argtypes = [U64, I, P, P]
        lib.lw_receptor.argtypes = [U64, I, I, P, D, D, P, P]
        lib.lw_anchors.argtypes = [U64, I, P, D, P]
        lib.lw_orientations.argtypes = [U64, I, P]
        lib.lw_normal.argtypes = [U64, U64, I64, P]
        lib.lw_uniform.argtypes = [U64, U64, I64, P]
        lib.lw_grid_maps.argtypes = [I, P, P, I, P, P, P, D, I, I, I, D, D, D, P]
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class Ligands:
    """A ligand library in the C-ABI's host layout (concatenated arrays)."""
    atom_offset: np.ndarray  # int32 [n+1]
    xyz: np.ndarray          # float32 [total_atoms, 3]
    type: np.ndarray         # uint8 [total_atoms]
    bond_offset: np.ndarray  # int32 [n+1]
    bonds: np.ndarray        # int32 [total_bonds, 2]  (parent, child) tree edges
    rotatable: np.ndarray    # uint8 [total_bonds]
    n_rot: np.ndarray        # int32 [n] realised rotatable counts

    @property
    def n(self) -> int:
        return len(self.atom_offset) - 1

    def n_atoms(self) -> np.ndarray:
        return np.diff(self.atom_offset)

    def ligand(self, i: int):
        """(xyz[n,3], type[n], bonds[n-1,2], rotatable[n-1]) of ligand i."""
        a0, a1 = int(self.atom_offset[i]), int(self.atom_offset[i + 1])
        b0, b1 = int(self.bond_offset[i]), int(self.bond_offset[i + 1])
        return (self.xyz[a0:a1], self.type[a0:a1], self.bonds[b0:b1], self.rotatable[b0:b1])

    def subset(self, idx) -> "Ligands":
        idx = np.asarray(idx, dtype=np.int64)
        na = np.diff(self.atom_offset)[idx]
        nb = np.diff(self.bond_offset)[idx]
        ao = np.zeros(len(idx) + 1, np.int32)
        bo = np.zeros(len(idx) + 1, np.int32)
        ao[1:] = np.cumsum(na)
        bo[1:] = np.cumsum(nb)
        a_idx = np.concatenate([np.arange(self.atom_offset[i], self.atom_offset[i + 1]) for i in idx]) \
            if len(idx) else np.zeros(0, np.int64)
        b_idx = np.concatenate([np.arange(self.bond_offset[i], self.bond_offset[i + 1]) for i in idx]) \
            if len(idx) else np.zeros(0, np.int64)
        return Ligands(ao, np.ascontiguousarray(self.xyz[a_idx]), np.ascontiguousarray(self.type[a_idx]),
                       bo, np.ascontiguousarray(self.bonds[b_idx]),
                       np.ascontiguousarray(self.rotatable[b_idx]), self.n_rot[idx].copy())


@dataclass
class Pocket:
    """Per-atom-type grid maps of a prepared target plus its anchor points."""
    maps: np.ndarray      # float32 [T, nz, ny, nx]
    origin: np.ndarray    # float64 [3]
    spacing: float
    anchors: np.ndarray   # float32 [n_anchors, 3]
    receptor_xyz: Optional[np.ndarray] = None
    receptor_type: Optional[np.ndarray] = None
    # parameters the maps were computed with (per-type LJ radius and depth,
    # cutoff, cap, radius floor)
    type_radius: Optional[np.ndarray] = None
    type_eps: Optional[np.ndarray] = None
    cutoff: float = 8.0
    cap: float = 10.0
    rmin: float = 0.5

    def receptor(self) -> dict:
        """Receptor atoms (FP32 coordinates) and the parameters of the maps'
        potential, as the rescoring stage takes them."""
        return {"xyz": np.ascontiguousarray(self.receptor_xyz, np.float32),
                "type": np.ascontiguousarray(self.receptor_type, np.int32),
                "radius": np.asarray(self.type_radius, np.float64),
                "eps": np.asarray(self.type_eps, np.float64),
                "cutoff": self.cutoff, "cap": self.cap, "rmin": self.rmin}

    @property
    def n_types(self) -> int:
        return self.maps.shape[0]

    @property
    def dims(self):
        t, nz, ny, nx = self.maps.shape
        return nx, ny, nz


@dataclass
class Sampling:
    """Search parameters: orientations x anchors starts, torsion steps."""
    quats: np.ndarray      # float64 [n_orient, 4]  (w, x, y, z)
    n_anchor: int
    torsion_steps: int
    top_k: int
    clash_weight: float = 1.0
    clash_cutoff: float = 3.0
    clash_min_sep: int = 4
    penalty: float = 10.0

    @property
    def n_orient(self) -> int:
        return self.quats.shape[0]

    @property
    def n_starts(self) -> int:
        return self.n_orient * self.n_anchor


@dataclass
class Workload:
    name: str
    ligands: Ligands
    pocket: Pocket
    sampling: Sampling
    meta: dict = field(default_factory=dict)


# --------------------------------------------------------------------------
def ligand_sizes(seed: int, n: int, kind: int, nmin: int, nmax: int, rmin: int, rmax: int):
    lib = _load()
    na = np.zeros(n, np.int32)
    nr = np.zeros(n, np.int32)
    rc = lib.lw_ligand_sizes(seed, n, kind, nmin, nmax, rmin, rmax, _p(na), _p(nr))
    if rc != 0:
        raise ValueError("bad ligand size parameters")
    return na, nr


def make_ligands(seed: int, n_atoms: np.ndarray, n_rot_req: np.ndarray, n_types: int,
                 first_index: int = 0) -> Ligands:
    """Ligand trees; ligand i is drawn from stream (seed, first_index + i)."""
    lib = _load()
    n = len(n_atoms)
    n_atoms = np.ascontiguousarray(n_atoms, np.int32)
    n_rot_req = np.ascontiguousarray(n_rot_req, np.int32)
    ao = np.zeros(n + 1, np.int64)
    ao[1:] = np.cumsum(n_atoms)
    nb = np.maximum(n_atoms - 1, 0)
    bo = np.zeros(n + 1, np.int64)
    bo[1:] = np.cumsum(nb)
    xyz = np.zeros((int(ao[-1]), 3), np.float32)
    typ = np.zeros(int(ao[-1]), np.uint8)
    bonds = np.zeros((int(bo[-1]), 2), np.int32)
    rot = np.zeros(int(bo[-1]), np.uint8)
    rr = np.zeros(n, np.int32)
    rc = lib.lw_ligands(seed, first_index, n, n_types, _p(n_atoms), _p(n_rot_req), _p(ao), _p(bo),
                        _p(xyz), _p(typ), _p(bonds), _p(rot), _p(rr))
    if rc != 0:
        raise RuntimeError(f"ligand generation failed at index {-rc - 1}")
    return Ligands(ao.astype(np.int32), xyz, typ, bo.astype(np.int32), bonds, rot, rr)


def make_pocket(seed: int, n_types: int, n: int, spacing: float, n_receptor: int, n_anchors: int,
                cutoff: float = 8.0, cap: float = 10.0, rmin: float = 0.5) -> Pocket:
    """Cubic n^3 grid, origin at 0, receptor shell [0.3 L, 0.5 sqrt(3) L] about
    the box centre (L = (n-1) * spacing), anchors in a ball of 0.2 L."""
    lib = _load()
    L = (n - 1) * spacing
    center = np.array([L / 2, L / 2, L / 2], np.float64)
    radius = np.zeros(n_types)
    eps = np.zeros(n_types)
    lib.lw_type_params(seed, n_types, _p(radius), _p(eps))
    rxyz = np.zeros((n_receptor, 3))
    rtyp = np.zeros(n_receptor, np.int32)
    lib.lw_receptor(seed, n_receptor, n_types, _p(center), 0.3 * L, 0.5 * np.sqrt(3.0) * L,
                    _p(rxyz), _p(rtyp))
    origin = np.zeros(3)
    maps = np.zeros((n_types, n, n, n), np.float32)
    rc = lib.lw_grid_maps(n_types, _p(radius), _p(eps), n_receptor, _p(rxyz), _p(rtyp), _p(origin),
                          spacing, n, n, n, cutoff, cap, rmin, _p(maps))
    if rc != 0:
        raise MemoryError("grid map generation failed")
    anchors = np.zeros((n_anchors, 3), np.float32)
    lib.lw_anchors(seed, n_anchors, _p(center), 0.2 * L, _p(anchors))
    return Pocket(maps, origin, float(spacing), anchors, rxyz, rtyp, radius, eps, cutoff, cap, rmin)


def type_params(seed: int, n_types: int):
    lib = _load()
    radius = np.zeros(n_types)
    eps = np.zeros(n_types)
    lib.lw_type_params(seed, n_types, _p(radius), _p(eps))
    return radius, eps


def grid_maps(radius, eps, rec_xyz, rec_type, origin, spacing, dims, cutoff=8.0, cap=10.0,
              rmin=0.5) -> np.ndarray:
    """Maps for arbitrary receptor atoms (used by tests on tiny cases)."""
    lib = _load()
    nx, ny, nz = dims
    T = len(radius)
    maps = np.zeros((T, nz, ny, nx), np.float32)
    radius = np.ascontiguousarray(radius, np.float64)
    eps = np.ascontiguousarray(eps, np.float64)
    rec_xyz = np.ascontiguousarray(rec_xyz, np.float64)
    rec_type = np.ascontiguousarray(rec_type, np.int32)
    origin = np.ascontiguousarray(origin, np.float64)
    lib.lw_grid_maps(T, _p(radius), _p(eps), len(rec_type), _p(rec_xyz), _p(rec_type), _p(origin),
                     spacing, nx, ny, nz, cutoff, cap, rmin, _p(maps))
    return maps


def orientations(seed: int, n: int) -> np.ndarray:
    lib = _load()
    q = np.zeros((n, 4))
    lib.lw_orientations(seed, n, _p(q))
    return q


def normal(seed: int, tag: int, n: int) -> np.ndarray:
    lib = _load()
    out = np.zeros(n)
    lib.lw_normal(seed, tag, n, _p(out))
    return out


def uniform(seed: int, tag: int, n: int) -> np.ndarray:
    lib = _load()
    out = np.zeros(n)
    lib.lw_uniform(seed, tag, n, _p(out))
    return out


# --------------------------------------------------------------------------
# Benchmark configurations (synthetic stand-ins, seeds 1000 + i).
CONFIGS = {
    "tiny": dict(seed=1000, n_ligands=1, kind=0, nmin=24, nmax=24, rmin=4, rmax=4, n_types=6,
                 grid=32, spacing=0.375, n_receptor=400, n_orient=64, n_anchor=8, steps=8, top_k=4),
    "batched": dict(seed=1001, n_ligands=10_000, kind=0, nmin=15, nmax=60, rmin=0, rmax=12,
                    n_types=8, grid=64, spacing=0.375, n_receptor=3000, n_orient=256, n_anchor=32,
                    steps=16, top_k=16),
    "learned_train": dict(seed=1003, pocket_seed=1001, n_ligands=200_000, kind=0, nmin=15, nmax=60, rmin=0, rmax=12,
                          n_types=8, grid=64, spacing=0.375, n_receptor=3000, n_orient=256,
                          n_anchor=32, steps=16, top_k=16),
    "combined": dict(seed=1004, n_ligands=1_000_000, kind=1, nmin=10, nmax=80, rmin=0, rmax=15,
                     n_types=8, grid=96, spacing=0.375, n_receptor=8000, n_orient=256, n_anchor=32,
                     steps=16, top_k=16),
    "combined_train": dict(seed=1005, pocket_seed=1004, n_ligands=200_000, kind=1, nmin=10, nmax=80,
                           rmin=0, rmax=15, n_types=8, grid=96, spacing=0.375, n_receptor=8000,
                           n_orient=256, n_anchor=32, steps=16, top_k=16),
}


def make_workload(name: str, n_ligands: Optional[int] = None, first_index: int = 0,
                  pocket: Optional[Pocket] = None, **override) -> Workload:
    """Build a configuration by name; ``n_ligands``/``first_index`` select a
    contiguous slice of the library (each ligand has its own stream, so a
    slice equals the same ligands of the full library)."""
    cfg = dict(CONFIGS[name])
    cfg.update(override)
    seed = cfg["seed"]
    n = cfg["n_ligands"] if n_ligands is None else n_ligands
    total = first_index + n
    na, nr = ligand_sizes(seed, total, cfg["kind"], cfg["nmin"], cfg["nmax"], cfg["rmin"], cfg["rmax"])
    ligs = make_ligands(seed, na[first_index:], nr[first_index:], cfg["n_types"], first_index)
    if pocket is None:
        pocket = make_pocket(cfg.get("pocket_seed", seed), cfg["n_types"], cfg["grid"], cfg["spacing"], cfg["n_receptor"],
                             max(cfg["n_anchor"], 32))
    samp = Sampling(orientations(seed, cfg["n_orient"]), cfg["n_anchor"], cfg["steps"], cfg["top_k"])
    return Workload(name, ligs, pocket, samp, dict(cfg, n_ligands=n, first_index=first_index))


def poses_per_ligand(ligands: Ligands, sampling: Sampling) -> np.ndarray:
    """Unique poses scored per ligand: n_starts * (1 + R (S - 1)) (the k = 0
    trial of each bond repeats the current pose)."""
    return sampling.n_starts * (1 + ligands.n_rot.astype(np.int64) * (sampling.torsion_steps - 1))

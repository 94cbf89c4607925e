"""The C-ABI library builds for sm_103a, loads without a GPU, exports every
function include/ligate.h declares, and rejects malformed input on the host
before any CUDA call."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2304_09953_gb300 import build as B
from paper_2304_09953_gb300 import native as N
from paper_2304_09953_gb300.workload import make_ligands

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "ligate.h")


def declared():
    src = open(HDR).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ligate_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    B.build()
    lib = ctypes.CDLL(B.SO)
    names = declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), f"{n} missing from libligate.so"
    assert set(names) == set(N.exported_symbols())
    assert b"sm_103a" in N.load().ligate_version()


def _lig_struct(atom_offset, xyz, typ, bond_offset, bonds, rot):
    keep = [np.ascontiguousarray(atom_offset, np.int32), np.ascontiguousarray(xyz, np.float32),
            np.ascontiguousarray(typ, np.uint8), np.ascontiguousarray(bond_offset, np.int32),
            np.ascontiguousarray(bonds, np.int32), np.ascontiguousarray(rot, np.uint8)]
    s = N.ligate_ligands(len(atom_offset) - 1, *[k.ctypes.data for k in keep])
    s._keep = keep
    return s


def _create(s):
    h = ctypes.c_void_p()
    return N.load().ligate_batch_create(ctypes.byref(s), ctypes.byref(h))


def test_batch_validation_errors_on_host():
    xyz = np.arange(12, dtype=np.float32).reshape(4, 3)
    typ = np.zeros(4)
    # cycle (3 bonds over 3 atoms + isolated atom): not a tree
    s = _lig_struct([0, 4], xyz, typ, [0, 3], [[0, 1], [1, 2], [2, 0]], [0, 0, 0])
    assert _create(s) == N.LIGATE_ERR_INVALID
    # wrong number of bonds
    s = _lig_struct([0, 4], xyz, typ, [0, 2], [[0, 1], [1, 2]], [0, 0])
    assert _create(s) == N.LIGATE_ERR_INVALID
    # bad atom index
    s = _lig_struct([0, 4], xyz, typ, [0, 3], [[0, 1], [1, 2], [2, 7]], [0, 0, 0])
    assert _create(s) == N.LIGATE_ERR_INVALID
    # non-finite coordinate
    bad = xyz.copy()
    bad[2, 1] = np.nan
    s = _lig_struct([0, 4], bad, typ, [0, 3], [[0, 1], [1, 2], [2, 3]], [0, 0, 0])
    assert _create(s) == N.LIGATE_ERR_INVALID
    assert b"non-finite" in N.load().ligate_last_error()
    # disconnected although n-1 bonds: a duplicate edge leaves an atom out
    s = _lig_struct([0, 4], xyz, typ, [0, 3], [[0, 1], [1, 0], [2, 3]], [0, 0, 0])
    assert _create(s) == N.LIGATE_ERR_INVALID
    # empty ligand
    s = _lig_struct([0, 0], np.zeros((0, 3)), np.zeros(0), [0, 0], np.zeros((0, 2)), np.zeros(0))
    assert _create(s) == N.LIGATE_ERR_INVALID


def test_batch_limits_are_unsupported():
    big = make_ligands(3, np.array([129], np.int32), np.array([0], np.int32), 8)
    assert _create(N.make_ligands_struct(big)) == N.LIGATE_ERR_UNSUPPORTED
    many = make_ligands(3, np.array([80], np.int32), np.array([17], np.int32), 8)
    if many.n_rot[0] == 17:
        assert _create(N.make_ligands_struct(many)) == N.LIGATE_ERR_UNSUPPORTED


def test_batch_packing_on_host_threads_reports_errors_per_caller():
    """Batches of 600 ligands are packed on the library's host thread pool
    (a batch of 256 ligands or more); one bad ligand in each fails the call
    before any device work, with its own index in the caller's error
    message.  Four callers at once: one runs on the pool, the others on
    threads of their own, and every call returns."""
    import threading
    n = 600
    libs = []
    for bad in (500, 17, 333, 599):
        lig = make_ligands(11, np.full(n, 20, np.int32), np.full(n, 3, np.int32), 8)
        lig.bonds[lig.bond_offset[bad] + 2, 1] = 99  # an atom index outside the ligand
        libs.append((bad, N.make_ligands_struct(lig)))
    out = {}

    def call(bad, st):
        out[bad] = (_create(st), N.load().ligate_last_error())

    for _ in range(3):
        out.clear()
        th = [threading.Thread(target=call, args=a) for a in libs]
        for t in th:
            t.start()
        for t in th:
            t.join(timeout=120)
        assert not any(t.is_alive() for t in th)
        for bad, _ in libs:
            code, msg = out[bad]
            assert code == N.LIGATE_ERR_INVALID
            assert f"ligand {bad}: bond 2 has bad atom index".encode() in msg, msg


def test_pocket_validation_errors_on_host():
    lib = N.load()
    h = ctypes.c_void_p()
    maps = np.zeros((1, 4, 4, 4), np.float32)
    org = (ctypes.c_double * 3)(0, 0, 0)
    anc = np.zeros((1, 3), np.float32)
    assert lib.ligate_pocket_create(maps.ctypes.data, 1, 4, 4, 1, ctypes.addressof(org), 0.5,
                                    anc.ctypes.data, 1, 0, ctypes.byref(h)) == N.LIGATE_ERR_INVALID
    assert lib.ligate_pocket_create(maps.ctypes.data, 1, 4, 4, 4, ctypes.addressof(org), 0.0,
                                    anc.ctypes.data, 1, 0, ctypes.byref(h)) == N.LIGATE_ERR_INVALID
    maps[0, 1, 2, 3] = np.inf
    assert lib.ligate_pocket_create(maps.ctypes.data, 1, 4, 4, 4, ctypes.addressof(org), 0.5,
                                    anc.ctypes.data, 1, 0, ctypes.byref(h)) == N.LIGATE_ERR_INVALID
    assert lib.ligate_pocket_create(maps.ctypes.data, 1, 4, 4, 4, ctypes.addressof(org), 0.5,
                                    anc.ctypes.data, 1, 0, None) == N.LIGATE_ERR_INVALID


def test_null_handles_are_accepted_by_destroy():
    lib = N.load()
    lib.ligate_pocket_destroy(None)
    lib.ligate_batch_destroy(None)
    lib.ligate_plan_destroy(None)
    lib.ligate_surrogate_destroy(None)


@pytest.mark.parametrize("fn", ["ligate_plan_run", "ligate_plan_get_tile"])
def test_null_plan_is_invalid(fn):
    lib = N.load()
    assert getattr(lib, fn)(None, None, None) == N.LIGATE_ERR_INVALID


def test_screening_calls_reject_bad_arguments_on_host():
    """ligate_plan_best_quantile and ligate_plan_set_cutoff check their
    arguments before any device work: a NULL plan or output, or a fraction
    outside (0, 1], is INVALID with a message."""
    lib = N.load()
    out = ctypes.c_float()
    for frac in (0.01, 0.0, -1.0, 1.5, float("nan")):
        assert lib.ligate_plan_best_quantile(None, ctypes.c_double(frac), ctypes.byref(out), None) == \
            N.LIGATE_ERR_INVALID
        assert b"0 < frac <= 1" in lib.ligate_last_error()
    assert lib.ligate_plan_set_cutoff(None, None) == N.LIGATE_ERR_INVALID
    assert b"NULL plan" in lib.ligate_last_error()

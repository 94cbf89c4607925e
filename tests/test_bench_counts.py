"""The benchmark's roofline counts against their definitions (CPU only).

The algorithmic count is per unique pose of the search space the run
evaluated: N atom interpolations for a start's rigid pose, then for every
bond the moved atoms and the crossing clash pairs of its S - 1 new trials
(the k = 0 trial repeats the current pose).  The device counters count all
S trials, so the benchmark converts; here the counters are built from the
packed ligands' bond tables for a run that prunes nothing, and the
conversion must give the closed form."""
import types

import numpy as np

import bench
from paper_2304_09953_gb300 import native as N
from paper_2304_09953_gb300.workload import make_workload


def test_algorithmic_count_is_the_unique_pose_count():
    w = make_workload("batched", n_ligands=12)
    S, n_starts = w.sampling.torsion_steps, w.sampling.n_starts
    atoms_all = pairs_all = unique_atoms = unique_pairs = 0
    total_atoms = 0
    for i in range(w.ligands.n):
        order, bonds, cand = N.ligate_inspect_ligand(w.ligands, i)
        n = len(order)
        moved = sum(int(b[2] - b[1] - 1) for b in bonds)  # (v, end): atoms after v in the subtree
        ncand = sum(int(b[3]) for b in bonds)
        total_atoms += n
        atoms_all += n_starts * (n + S * moved)  # what the device counts: every trial
        pairs_all += n_starts * ncand  # candidates once per bond sweep (the counter)
        unique_atoms += n_starts * (n + (S - 1) * moved)
        unique_pairs += n_starts * (S - 1) * ncand
    work = types.SimpleNamespace(done_atom_evals=float(atoms_all), done_pair_evals=float(pairs_all * S))
    flop, atoms, pairs = bench.algorithmic_flops(work, S, n_starts, total_atoms)
    assert atoms == unique_atoms and pairs == unique_pairs
    assert flop == bench.FLOP_ALG_ATOM * unique_atoms + bench.FLOP_ALG_PAIR * unique_pairs


def test_peak_and_traffic_lookup():
    assert abs(bench.fp32_peak_tflops(152, 2070.0) - 80.54784) < 1e-9
    assert bench.kernel_traffic("batched", 12345) is None  # no capture for that size
    sha = bench.kernel_source_sha()
    assert len(sha) == 12 and all(c in "0123456789abcdef" for c in sha)

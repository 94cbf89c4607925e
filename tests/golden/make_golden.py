"""Writes tests/golden/tiny_oracle.json: the FP64 oracle's docking result on
the 1-ligand configuration (24 atoms, 4 rotatable bonds, 6 x 32^3 maps,
64 x 8 starts, 8 torsion steps, top-4).

The paper prints no worked example (its figures are plots only), so this file
is not a pin of the oracle; it records the oracle's own output so that a run
on another host (the aarch64 GPU machine regenerates inputs and re-runs the
oracle) can confirm that generator and oracle are bit-for-bit portable.
Calls only the workload generator and ``oracle``.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2304_09953_gb300.workload import make_workload  # noqa: E402


def compute():
    w = make_workload("tiny")
    lig = w.ligands.ligand(0)
    s, st, t = oracle.dock_ligand(lig, w.pocket, w.sampling)
    e_all, _ = oracle.greedy(lig, w.pocket, w.sampling)
    return {
        "config": "tiny (seed 1000)",
        "top_scores": [float(x) for x in s],
        "top_starts": [int(x) for x in st],
        "top_tors": [[int(v) for v in row] for row in t],
        "sum_all_start_scores": float(np.sum(e_all)),
        "maps_sum": float(np.sum(w.pocket.maps, dtype=np.float64)),
        "xyz_sum": float(np.sum(w.ligands.xyz, dtype=np.float64)),
    }


if __name__ == "__main__":
    out = os.path.join(HERE, "tiny_oracle.json")
    with open(out, "w") as f:
        json.dump(compute(), f, indent=1)
    print("wrote", out)

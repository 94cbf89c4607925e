"""Resumable screening of a large library (host side): the library is docked
chunk by chunk and every finished chunk is written atomically and recorded
in a journal, so a rerun after an interruption docks only the chunks that
are missing.  A ligand's result does not depend on the other ligands of its
chunk (each ligand's starts, merge and rescoring are its own), so the
chunked result equals a single run over the whole library.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np

from . import docking as D
from . import native as N


def _fingerprint(ligands, sampling, mode, chunk) -> str:
    h = hashlib.sha1()
    for a in (ligands.atom_offset, ligands.xyz, ligands.type, ligands.bond_offset, ligands.bonds,
              ligands.rotatable, np.asarray(sampling.quats)):
        h.update(np.ascontiguousarray(a).tobytes())
    h.update(json.dumps([int(sampling.n_anchor), int(sampling.torsion_steps), int(sampling.top_k),
                         float(sampling.clash_weight), float(sampling.clash_cutoff), mode, int(chunk)]).encode())
    return h.hexdigest()


def screen_library(pocket, ligands, sampling, journal_dir, chunk=50000, mode="bf16", tile=None,
                   on_chunk=None) -> np.ndarray:
    """Dock `ligands` in chunks of `chunk`, journaling into `journal_dir`;
    returns ligate_pose records [n, top_k].  `on_chunk(c)` (optional) is
    called after chunk c is journaled.  A journal written for other inputs
    raises ValueError."""
    os.makedirs(journal_dir, exist_ok=True)
    meta_path = os.path.join(journal_dir, "meta.json")
    fp = _fingerprint(ligands, sampling, mode, chunk)
    n = ligands.n
    n_chunks = (n + chunk - 1) // chunk
    if os.path.exists(meta_path):
        with open(meta_path) as f:
            meta = json.load(f)
        if meta.get("fingerprint") != fp:
            raise ValueError(f"{journal_dir} journals a different library or sampling")
    else:
        tmp = meta_path + ".tmp"
        with open(tmp, "w") as f:
            json.dump({"fingerprint": fp, "n_ligands": n, "chunk": chunk, "n_chunks": n_chunks}, f)
        os.replace(tmp, meta_path)
    journal = os.path.join(journal_dir, "journal.txt")
    done = set()
    if os.path.exists(journal):
        with open(journal) as f:
            done = {int(line) for line in f if line.strip()}

    def chunk_path(c):
        return os.path.join(journal_dir, f"chunk_{c:06d}.npy")

    todo = [c for c in range(n_chunks) if not (c in done and os.path.exists(chunk_path(c)))]
    if todo:
        ph = D.PocketHandle(pocket)
        try:
            for c in todo:
                c0, c1 = c * chunk, min(n, (c + 1) * chunk)
                bh = D.BatchHandle(ligands.subset(np.arange(c0, c1)))
                pl = D.Plan(ph, bh, sampling, mode=mode, tile=tile)
                try:
                    res = pl.result()
                finally:
                    pl.close()
                    bh.close()
                tmp = chunk_path(c) + ".tmp.npy"
                np.save(tmp, res)
                os.replace(tmp, chunk_path(c))
                with open(journal, "a") as f:
                    f.write(f"{c}\n")
                    f.flush()
                    os.fsync(f.fileno())
                if on_chunk is not None:
                    on_chunk(c)
        finally:
            ph.close()
    out = np.concatenate([np.load(chunk_path(c)) for c in range(n_chunks)]) if n_chunks else \
        np.zeros((0, sampling.top_k), N.POSE_DTYPE)
    return out

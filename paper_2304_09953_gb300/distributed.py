"""Multi-rank screening helpers (host side).

Ligands are independent (paper Sec. 1: virtual screening is embarrassingly
parallel), so a library is split into contiguous per-rank shards that each
rank docks on its own GPU with no collective on the data path.  The only
exchanges are the timing reduction (slowest rank) and, when a global
ranking is wanted, one all-gather of each shard's per-ligand best scores
(4 bytes per ligand).  Works with any torch.distributed backend (NCCL for
the GPUs, gloo for CPU tests).
"""
from __future__ import annotations

import numpy as np


def shard(n_total: int, rank: int, world: int, weights=None):
    """Contiguous shard (first index, count) of rank in [0, world).

    Without weights the ligand counts are balanced (they differ by at most
    one).  With per-ligand weights (e.g. the precomputed pose count of each
    ligand, workload.poses_per_ligand) the shards balance the work instead:
    ligand i goes to rank floor(world * (W_i + w_i / 2) / W), W_i the work
    before it and W the total, so the ranges are contiguous, ordered, and
    each rank's work is within one ligand's weight of W / world."""
    if world < 1 or not 0 <= rank < world or n_total < 0:
        raise ValueError("bad shard arguments")
    if weights is None:
        base, extra = divmod(n_total, world)
        first = rank * base + min(rank, extra)
        return first, base + (1 if rank < extra else 0)
    w = np.asarray(weights, np.float64)
    if w.shape != (n_total,) or np.any(w < 0):
        raise ValueError("weights must be n_total non-negative numbers")
    total = float(w.sum())
    if total <= 0.0:
        return shard(n_total, rank, world)
    mid = np.cumsum(w) - 0.5 * w
    owner = np.minimum((world * mid / total).astype(np.int64), world - 1)
    first = int(np.searchsorted(owner, rank, side="left"))
    last = int(np.searchsorted(owner, rank, side="right"))
    return first, last - first


def max_over_ranks(value: float, device=None) -> float:
    """Largest value over all ranks (the job's wall time is its slowest rank)."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    """Sum of a per-rank value over all ranks (e.g. the poses each rank scored)."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def gather_scores(local_best: np.ndarray, n_total: int, device=None, weights=None) -> np.ndarray:
    """All ranks' per-ligand best scores in global ligand order (every rank
    receives the full array).  Rank r must hold the shard given by
    shard(n_total, r, world, weights)."""
    import torch
    import torch.distributed as dist
    local_best = np.asarray(local_best, np.float32)
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return local_best.copy()
    world = dist.get_world_size()
    counts = [shard(n_total, r, world, weights)[1] for r in range(world)]
    width = max(counts) if counts else 0
    buf = torch.full((width,), float("inf"), dtype=torch.float32, device=device)
    buf[:len(local_best)] = torch.from_numpy(local_best).to(buf.device)
    parts = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf)
    return np.concatenate([parts[r][:counts[r]].cpu().numpy() for r in range(world)])


def top_fraction(scores: np.ndarray, frac: float) -> np.ndarray:
    """Indices of the ceil(n * frac) lowest scores, best first (ties: smaller
    index) -- the screening output of a campaign."""
    scores = np.asarray(scores)
    k = int(np.ceil(len(scores) * frac - 1e-9))
    return np.lexsort((np.arange(len(scores)), scores))[:k]

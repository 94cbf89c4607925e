"""Multi-rank path on CPU: two gloo ranks shard a library by per-ligand
work, reduce their timings to the slowest rank and merge per-ligand best
scores into the same global top 1% a single process computes."""
import os
import socket

import numpy as np
import pytest

from paper_2304_09953_gb300.distributed import shard, top_fraction


def test_shards_cover_the_library_once():
    for n in (0, 1, 7, 10000, 10001):
        for world in (1, 2, 3, 8):
            got = [shard(n, r, world) for r in range(world)]
            assert sum(c for _, c in got) == n
            assert [f for f, _ in got] == sorted(f for f, _ in got)
            for (f0, c0), (f1, _) in zip(got, got[1:]):
                assert f0 + c0 == f1
            assert max(c for _, c in got) - min(c for _, c in got) <= 1


def test_work_weighted_shards_balance_pose_counts():
    """Shards weighted by each ligand's pose count: contiguous and ordered,
    every ligand once, and each rank's work within one ligand's weight of
    the mean (the count-balanced split of the same library is not)."""
    from paper_2304_09953_gb300.workload import make_workload, poses_per_ligand
    w = make_workload("batched", n_ligands=3000)
    poses = poses_per_ligand(w.ligands, w.sampling).astype(np.float64)
    poses[:1000] *= 3.0  # a library whose first third is heavier
    for world in (1, 2, 3, 8):
        got = [shard(len(poses), r, world, poses) for r in range(world)]
        assert got[0][0] == 0 and sum(c for _, c in got) == len(poses)
        for (f0, c0), (f1, _) in zip(got, got[1:]):
            assert f0 + c0 == f1
        work = [poses[f:f + c].sum() for f, c in got]
        assert max(abs(x - poses.sum() / world) for x in work) <= poses.max()
    even = [poses[f:f + c].sum() for f, c in (shard(len(poses), r, 2) for r in range(2))]
    assert abs(even[0] - even[1]) > poses.max()
    assert shard(5, 1, 2, np.zeros(5)) == shard(5, 1, 2)


def test_top_fraction_ties_and_order():
    s = np.array([3.0, 1.0, 1.0, -2.0, 5.0, 1.0])
    assert list(top_fraction(s, 0.5)) == [3, 1, 2]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, n_total, q):
    import torch.distributed as dist
    from paper_2304_09953_gb300.distributed import gather_scores, max_over_ranks, shard, top_fraction
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rng = np.random.default_rng(7)
    scores = rng.normal(size=n_total).astype(np.float32)
    weights = rng.integers(1, 13, size=n_total).astype(np.float64)  # per-ligand pose counts
    first, count = shard(n_total, rank, world, weights)
    local = scores[first:first + count]
    t = max_over_ranks(1.0 + rank)
    merged = gather_scores(local, n_total, weights=weights)
    q.put((rank, t, top_fraction(merged, 0.01).tolist(), merged.tolist()))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("n_total", [1001, 64])
def test_two_gloo_ranks_merge_to_the_single_process_answer(n_total):
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, n_total, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    scores = np.random.default_rng(7).normal(size=n_total).astype(np.float32)
    want = top_fraction(scores, 0.01).tolist()
    for rank, t, top, merged in out:
        assert t == 2.0
        assert top == want
        np.testing.assert_array_equal(np.array(merged, np.float32), scores)

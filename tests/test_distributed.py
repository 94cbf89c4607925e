"""Multi-rank path on CPU: two gloo ranks shard a library, reduce their
timings to the slowest rank and merge per-ligand best scores into the same
global top 1% a single process computes."""
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
    first, count = shard(n_total, rank, world)
    scores = np.random.default_rng(7).normal(size=n_total).astype(np.float32)
    local = scores[first:first + count]
    t = max_over_ranks(1.0 + rank)
    merged = gather_scores(local, n_total)
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

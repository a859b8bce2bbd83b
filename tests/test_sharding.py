"""Multi-GPU path on the host (CPU, no GPU needed): traces are independent, so a batch shards
with no exchange step; checked here for dense and cost-balanced ragged splits, and over two
gloo ranks for the only collective, the max of the per-rank times."""
import os
import socket

import numpy as np
import pytest

from paper_2501_04194_gb300.sharding import max_over_ranks, shard_dense, shard_ragged


def test_dense_shards_cover_the_batch_once():
    for B in (0, 1, 7, 1024, 1025):
        for world in (1, 2, 3, 8):
            parts = [shard_dense(B, world, r) for r in range(world)]
            idx = np.concatenate([np.arange(B)[s] for s in parts])
            assert np.array_equal(idx, np.arange(B))
            sizes = [s.stop - s.start for s in parts]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard_dense(4, 2, 2)


def test_ragged_shards_are_a_balanced_partition():
    rng = np.random.default_rng(0)
    lengths = rng.integers(50, 20000, size=10000)
    fid = rng.integers(0, 16, size=10000)
    fcost = rng.uniform(1.0, 4.0, size=16)
    for world in (1, 2, 4, 8):
        parts = shard_ragged(lengths, world, formula_id=fid, formula_cost=fcost)
        allidx = np.sort(np.concatenate(parts))
        assert np.array_equal(allidx, np.arange(len(lengths)))
        cost = lengths * fcost[fid]
        loads = np.array([cost[p].sum() for p in parts])
        # longest-processing-time-first: within one largest item of the best split
        assert loads.max() - loads.min() <= cost.max()
    # equal lengths split evenly by count
    parts = shard_ragged(np.full(12, 100), 4)
    assert [len(p) for p in parts] == [3, 3, 3, 3]
    with pytest.raises(ValueError):
        shard_ragged([1, 2], 2, formula_cost=[1.0])


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, lengths):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = shard_ragged(lengths, world)[rank]
        got = [None] * world
        dist.all_gather_object(got, mine.tolist())
        flat = sorted(i for part in got for i in part)
        assert flat == list(range(len(lengths)))
        # the per-rank time the bench reports is the max over ranks
        assert max_over_ranks(0.5 + rank) == 0.5 + (world - 1)
        dense = shard_dense(1000, world, rank)
        sizes = [None] * world
        dist.all_gather_object(sizes, dense.stop - dense.start)
        assert sum(sizes) == 1000
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    import torch.multiprocessing as mp
    lengths = np.random.default_rng(1).integers(50, 5000, size=257)
    mp.spawn(_rank_main, args=(2, _free_port(), lengths), nprocs=2, join=True)


def test_max_over_ranks_without_a_group():
    assert max_over_ranks(3.25) == 3.25

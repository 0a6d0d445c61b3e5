"""Host logic of the multi-GPU path on CPU: two gloo ranks.

The path shards only by independent systems (replicas): each rank owns its
systems, nothing is exchanged on the data path, and the benchmark takes the
maximum time over ranks.  These tests run that logic with world size 2."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        shard = bench.replica_shard(256, rank, world)
        seed = bench.workload_seed(rank)
        # each rank "times" its own shard; the benchmark reports the slowest rank
        mine = [float(len(shard) + rank), float(seed)]
        mx = bench.max_over_ranks(mine, "cpu")
        out[rank] = (shard, seed, mx)
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_and_max():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    shards = [out[r][0] for r in range(world)]
    allv = sorted(v for sh in shards for v in sh)
    assert allv == list(range(256))  # every replica exactly once
    assert set(shards[0]).isdisjoint(shards[1])
    assert out[0][1] != out[1][1]  # independent seeds
    # both ranks agree on the maximum
    assert out[0][2] == out[1][2] == [max(len(shards[0]), len(shards[1]) + 1), max(out[0][1], out[1][1])]


def test_single_process_max_is_identity():
    import bench
    assert bench.max_over_ranks([3.0, 1.5], "cpu") == [3.0, 1.5]
    assert bench.replica_shard(5, 0, 1) == [0, 1, 2, 3, 4]

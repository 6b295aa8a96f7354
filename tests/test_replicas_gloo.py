"""The multi-GPU mode of bench.py runs independent replicas (no data-path collective): each
rank times its own solves, the step time is the maximum over ranks and the whole-job value is
the units of all ranks over that time. This checks that host logic with two gloo ranks on the
CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local = [1.5, 4.0][rank]                         # rank 1 is the slow replica
    slowest = bench.max_over_ranks(local)
    rate = bench.whole_job_rate(900, world, slowest)
    dist.barrier()
    out[rank] = (slowest, rate)
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_value():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    assert out[0] == out[1] == (4.0, 900 * 2 / 4.0)


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(2.5) == 2.5
    assert bench.whole_job_rate(300, 1, 2.0) == 150.0


def _shard_rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1504_07028_gb300 import shard, synth
    cfg = synth.CFG_BATCH
    # the shapes of the 64-image batch (H, W, K drawn as the batch scenes draw them)
    import numpy as np
    shapes = []
    for j in range(64):
        rng = np.random.default_rng(5000 + j)
        H, W = (int(v) for v in rng.integers(96, 513, size=2))
        K = int(rng.choice([4, 8, 16]))
        if j == 0:
            H, W = 97, 509
        elif j == 1:
            H, W = 512, 512
        shapes.append((H, W, K))
    costs = [shard.iteration_bytes(H, W, K, cfg.M) for H, W, K in shapes]
    mine = shard.partition(costs, world)[rank]
    got = [None] * world
    dist.all_gather_object(got, mine)
    out[rank] = (got, costs)
    dist.destroy_process_group()


def test_batch_sharding_over_two_gloo_ranks():
    """Every image of the batch lands on exactly one rank, both ranks agree on the placement,
    and the ranks' per-iteration bytes differ by at most one image's."""
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.spawn(_shard_rank, args=(world, port, out), nprocs=world, join=True)
    got0, costs = out[0]
    got1, _ = out[1]
    assert got0 == got1
    flat = sorted(i for part in got0 for i in part)
    assert flat == list(range(64))
    loads = [sum(costs[i] for i in part) for part in got0]
    assert max(loads) - min(loads) <= max(costs)


def test_partition_by_hand():
    from paper_1504_07028_gb300 import shard
    # 5 -> r0; 3 -> r1; 3 -> r1 (3 < 5); 2 -> r0 (5 < 6); 1 -> r1 (6 < 7): loads 7 and 7
    assert shard.partition([5, 3, 3, 2, 1], 2) == [[0, 3], [1, 2, 4]]
    assert shard.partition([1, 1, 1], 1) == [[0, 1, 2]]
    assert shard.partition([4], 3) == [[0], [], []]
    assert shard.iteration_bytes(145, 145, 16, 1) == 4 * 145 * 145 * 16 * 47

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

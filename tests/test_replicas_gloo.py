"""Host logic of the N-GPU bench (replicas: one independent sweep per rank)
run as two gloo ranks on the CPU: the job time is the slowest rank's, and the
throughput counts the sweeps of every rank."""
import os
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 100.0 + 50.0 * rank          # rank 1 is slower
    value, t_max = bench.aggregate(ms, 10, world, dist)
    out[rank] = (value, t_max)
    dist.destroy_process_group()


def test_replica_throughput_uses_slowest_rank():
    world = 2
    port = 29500 + (os.getpid() % 1000)
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, port, out), nprocs=world, start_method="spawn")
    for r in range(world):
        value, t_max = out[r]
        assert t_max == 150.0
        assert abs(value - 2 * 10 / 0.150) < 1e-9

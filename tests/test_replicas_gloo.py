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


def _shard_rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch
    import ttn_inputs as ti
    from paper_1905_01331_gb300 import instance_cost, shard_instances
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wls = ti.batched_chains()
    costs = [instance_cost(w.model.Lx, w.chi) for w in wls]
    mine = shard_instances(costs, world, rank)
    shards = [None] * world
    dist.all_gather_object(shards, mine)
    load = torch.tensor([sum(costs[i] for i in mine)], dtype=torch.float64)
    loads = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(loads, load)
    out[rank] = (shards, [float(x) for x in loads], sum(costs))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_batched_instances_shard_over_ranks(world):
    """C5's independent chains are split over ranks with no data-path
    collective: every rank computes the same assignment; together the ranks
    hold every instance exactly once; the load of the slowest rank is within
    one instance of the mean."""
    port = 29600 + world * 10 + (os.getpid() % 500)
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_shard_rank, args=(world, port, out), nprocs=world, start_method="spawn")
    shards, loads, total = out[0]
    for r in range(1, world):
        assert out[r][0] == shards
    flat = sorted(i for sh in shards for i in sh)
    assert flat == list(range(64))
    import ttn_inputs as ti
    from paper_1905_01331_gb300 import instance_cost
    biggest = max(instance_cost(w.model.Lx, w.chi) for w in ti.batched_chains())
    assert max(loads) - total / world <= biggest

"""Several ranks on CPU (gloo, world size 2): the instance sharding and the max-over-ranks timing
reduction that the benchmark uses for independent instances on several GPUs."""
import os
import socket

import pytest

import tsfcde_workloads as W
from paper_1603_00279_gb300.multirank import instance_cost, max_over_ranks, partition, shard


def _costs(count=64):
    return [instance_cost(q.n, q.M) for q in W.config_batch(count=count, M=16)]


def test_partition_is_complete_disjoint_and_balanced():
    costs = _costs(200)
    for world in (1, 2, 3, 8):
        parts = partition(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        # LPT bound: no rank exceeds the average by more than the largest single instance
        assert max(loads) <= sum(costs) / world + max(costs) + 1e-9
        assert all(shard(costs, world, r) == parts[r] for r in range(world))
    with pytest.raises(ValueError):
        shard(costs, 2, 2)


def test_max_over_ranks_without_a_group_is_the_value():
    assert max_over_ranks(3.5) == 3.5


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, costs, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = shard(costs, world, rank)
        everyone = [None] * world
        dist.all_gather_object(everyone, mine)
        t = max_over_ranks(1.0 + 1.5 * rank, dist)
        q.put((rank, mine, everyone, t))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_without_communication_and_take_the_slowest_time():
    import torch.multiprocessing as mp
    costs = _costs()
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, costs, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    # every rank computed the same partition on its own, and together they cover every instance
    assert out[0][2] == out[1][2] == [out[0][1], out[1][1]]
    assert sorted(out[0][1] + out[1][1]) == list(range(len(costs)))
    assert not set(out[0][1]) & set(out[1][1])
    # the step time is the slowest rank's
    assert out[0][3] == out[1][3] == 2.5

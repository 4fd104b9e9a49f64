"""Multi-rank host logic on CPU: two gloo ranks shard the 64-instance batch,
gather their shards and reduce a timing by max (no GPU involved)."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import fde_inputs as fi
from paper_1907_13428_gb300 import sharding


def _costs():
    return [sharding.instance_cost(p.nx, p.ny, p.nt) for p, _, _, _ in fi.config_batch_params()]


def test_shard_is_a_partition_and_balanced():
    costs = _costs()
    for world in (1, 2, 3, 4, 8):
        parts = sharding.shard(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        # greedy LPT: no rank exceeds the mean by more than the largest single cost
        assert max(loads) <= sum(loads) / world + max(costs) + 1e-9
        assert parts == sharding.shard(costs, world)  # deterministic
    with pytest.raises(ValueError):
        sharding.shard(costs, 0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        costs = _costs()
        mine = sharding.shard(costs, world)[rank]
        allp = sharding.gather_objects(mine)
        t = sharding.max_over_ranks(1.5 + rank)
        q.put((rank, allp, t))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_gather_and_reduce():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    for rank, allp, t in res:
        assert t == 1.5 + world - 1
        assert sorted(i for p in allp for i in p) == list(range(64))
        assert allp == sharding.shard(_costs(), world)

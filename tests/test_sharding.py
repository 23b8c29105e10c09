"""Scene sharding across ranks: the partition covers every scene once and is
balanced; two gloo ranks on CPU agree on it and reduce their timings."""
import os
import socket

import numpy as np
import pytest

from paper_2306_06946_gb300 import sharding


def test_partition_covers_every_scene_once_and_balances():
    rng = np.random.default_rng(0)
    costs = rng.lognormal(0.0, 1.0, size=64)
    for world in (1, 2, 3, 8):
        parts = sharding.partition(costs, world)
        assert sorted(i for p in parts for i in p) == list(range(64))
        loads = [costs[p].sum() if p else 0.0 for p in parts]
        assert max(loads) - min(loads) <= costs.max() + 1e-12
    assert sharding.partition([], 4) == [[], [], [], []]
    assert sharding.partition([5.0, 1.0], 4)[2:] == [[], []]
    with pytest.raises(ValueError):
        sharding.partition(costs, 0)
    with pytest.raises(ValueError):
        sharding.shard(costs, 2, 2)


def test_scene_cost_orders_by_size():
    assert sharding.scene_cost(60000, 1500) > sharding.scene_cost(9000, 300) > sharding.scene_cost(960, 40)


def _rank(rank, world, port, costs, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = sharding.shard(costs, world, rank)
        everyone = [None] * world
        dist.all_gather_object(everyone, mine)
        t, n = sharding.reduce_timing(0.5 + rank, len(mine))
        out.put((rank, everyone, t, n))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_shards_and_reduce_timing():
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    costs = [float(c) for c in np.random.default_rng(1).lognormal(0.0, 1.0, size=20)]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, costs, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, everyone, t, n in res:
        assert sorted(i for part in everyone for i in part) == list(range(20))
        assert everyone[rank] == sharding.shard(costs, 2, rank)
        assert t == 1.5 and n == 20

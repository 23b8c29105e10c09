"""Independent scenes split across ranks (one GPU per rank).

Scenes do not exchange data, so a batch is partitioned across ranks with no
collective on the data path; ranks meet only around the timed region (a
barrier) and to reduce the elapsed time (max over ranks) and the number of
steps done (sum) on the host side.
"""
from __future__ import annotations


def scene_cost(n_dof: int, m: int) -> float:
    """Relative cost of one time step of a scene: the dense bound of the
    forward-solve right-hand sides, n x 3m, plus the PGS sweep work (3m)^2."""
    return float(n_dof) * 3.0 * m + 9.0 * m * m


def partition(costs, world: int) -> list[list[int]]:
    """Longest-processing-time assignment of scenes to ``world`` ranks:
    scenes in decreasing cost (ties by index) go to the least loaded rank
    (ties to the lower rank).  Deterministic; every scene lands on one rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    load = [0.0] * world
    parts: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += float(costs[i])
    return [sorted(p) for p in parts]


def shard(costs, world: int, rank: int) -> list[int]:
    """The scenes rank ``rank`` steps."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    return partition(costs, world)[rank]


def reduce_timing(elapsed_s: float, steps: int, device=None) -> tuple[float, int]:
    """(max elapsed over ranks, total steps over ranks); the identity without
    an initialised process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(elapsed_s), int(steps)
    t = torch.tensor([float(elapsed_s)], dtype=torch.float64, device=device)
    c = torch.tensor([int(steps)], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), int(c.item())

"""Sharding of independent bound work across ranks (one process per GPU).

Branch-and-bound nodes and bound requests are independent units: rank r of
W bounds units r, r+W, r+2W, ...; no collective touches the data path, and
the per-unit results are gathered once at the end.  Users: bound_nodes_sharded
below (a batch of B&B nodes), bnb.BranchAndBound(group=...) (subtrees, with
the incumbent exchanged between rounds) and serve.serve_sharded (requests).
"""
from __future__ import annotations

from typing import List, Sequence, Tuple


def shard(units: Sequence, rank: int, world: int) -> List[Tuple[int, object]]:
    """(global index, unit) pairs owned by `rank` (round-robin)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world: %r/%r" % (rank, world))
    return [(i, u) for i, u in enumerate(units) if i % world == rank]


def gather_results(local: List[Tuple[int, int]], total: int, group=None) -> List[int]:
    """All ranks' (index, result) pairs -> results in global order (every rank)."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    parts = [None] * world
    dist.all_gather_object(parts, local, group=group)
    out = [None] * total
    for part in parts:
        for i, v in part:
            out[i] = v
    if any(v is None for v in out):
        raise RuntimeError("a unit was bounded by no rank")
    return out


def bound_nodes_sharded(F, D, nodes, iters: int, group=None, **kw) -> List[int]:
    """Bounds of B&B nodes (fac, loc) of one instance: this rank's share by
    one rlt2_batch_bound call on its GPU, every node's bound gathered on every
    rank in the original order.  kw: rlt2_batch_bound options."""
    import torch.distributed as dist

    from . import rlt2

    mine = shard(nodes, dist.get_rank(group), dist.get_world_size(group))
    local = []
    if mine:
        lbs, _ = rlt2.rlt2_batch_bound(F, D, [n for _, n in mine], iters, **kw)
        local = [(i, int(v)) for (i, _), v in zip(mine, lbs)]
    return gather_results(local, len(nodes), group)


"""Sharding of independent grids and requests over the GPUs of a node.

Batched and served work consists of independent simulations: a grid never
exchanges data with another.  So the ranks of a multi-GPU job (one process
per GPU) split the grids or the requests among themselves with no data-path
collective at all; each rank keeps its share resident on its own device and
advances it with its own ``lbm.Batch`` / ``serve.Server``.  The only
collectives are host-side: gathering the per-rank summaries on rank 0.

The split is deterministic and needs no communication: every rank computes
the same assignment from the same list.  Grids go to ranks by longest-first
greedy balancing of their work (nodes x steps); requests go, in arrival
order, to the rank with the least work assigned so far, so that each rank
sees a stream with the trace's arrival pattern.
"""
from __future__ import annotations

import heapq


def _work_grid(item) -> int:
    p, _ = item[:2]
    return int(p["nx"]) * int(p["ny"])


def assign_grids(grids, world: int, weight=_work_grid):
    """Rank of every grid (a list parallel to ``grids``): longest first, each
    to the currently least-loaded rank (ties to the lowest rank)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(grids)), key=lambda i: (-weight(grids[i]), i))
    heap = [(0, r) for r in range(world)]
    owner = [0] * len(grids)
    for i in order:
        load, r = heapq.heappop(heap)
        owner[i] = r
        heapq.heappush(heap, (load + weight(grids[i]), r))
    return owner


def shard_grids(grids, rank: int, world: int, weight=_work_grid):
    """The grids rank `rank` of `world` owns, with their indices in `grids`."""
    owner = assign_grids(grids, world, weight)
    return [(i, g) for i, g in enumerate(grids) if owner[i] == rank]


def assign_requests(trace, world: int):
    """Rank of every request of a trace (parallel list): in arrival order, to
    the rank with the least work (nodes x steps) so far."""
    if world < 1:
        raise ValueError("world must be >= 1")
    loads = [0] * world
    owner = {}
    for r in sorted(trace, key=lambda q: (q.arrival, q.rid)):
        k = min(range(world), key=lambda j: (loads[j], j))
        owner[r.rid] = k
        loads[k] += r.nodes * r.steps
    return [owner[r.rid] for r in trace]


def shard_trace(trace, rank: int, world: int):
    """The requests of `trace` that rank `rank` of `world` serves."""
    owner = assign_requests(trace, world)
    return [r for r, k in zip(trace, owner) if k == rank]


def gather_results(results, dist=None):
    """All ranks' result lists on rank 0 (the one-rank list without a
    process group); other ranks get None.  Host objects only (gloo or the
    NCCL group's object collectives), outside every timed data path."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return list(results)
    world = dist.get_world_size()
    out = [None] * world if dist.get_rank() == 0 else None
    dist.gather_object(list(results), out, dst=0)
    if dist.get_rank() != 0:
        return None
    return [r for part in out for r in part]

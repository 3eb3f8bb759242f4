"""Sharding of independent graphs over ranks (one process per GPU).

A batch of graphs, or a stream of served requests, consists of independent
problems: no edge crosses two graphs, so each rank colors its own share with
no exchange on the data path.  This module holds the host-side logic only:

- ``partition``: greedy longest-processing-time bin packing of the graphs on
  their adjacency entries (the work of every pass is proportional to them),
  identical on every rank, so no rank has to send the assignment;
- ``max_over_ranks``: the job time, the slowest rank's (a MAX all-reduce of
  one number, outside the timed work);
- ``gather``: the per-rank results collected on rank 0 (host objects).

A single graph is not sharded: splitting it needs a boundary-color exchange
every round and every class step (the paper's distributed design), so several
GPUs run independent replicas of it instead.
"""
from __future__ import annotations

import heapq

import torch
import torch.distributed as dist


def partition(weights, world_size: int):
    """Indices of the items each of `world_size` ranks takes: heaviest item
    first, each to the currently lightest rank (ties to the lower rank).
    Every item lands on exactly one rank; the result is deterministic."""
    if world_size < 1:
        raise ValueError("world_size must be >= 1")
    order = sorted(range(len(weights)), key=lambda i: (-int(weights[i]), i))
    heap = [(0, r) for r in range(world_size)]
    parts = [[] for _ in range(world_size)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + int(weights[i]), r))
    return [sorted(p) for p in parts]


def loads(weights, parts):
    return [sum(int(weights[i]) for i in p) for p in parts]


def _active():
    return dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1


def max_over_ranks(value: float, device=None) -> float:
    """The maximum of `value` over all ranks (the value itself on one rank)."""
    if not _active():
        return float(value)
    if device is None:
        device = torch.device("cuda", torch.cuda.current_device()) \
            if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather(obj, dst: int = 0):
    """Every rank's `obj` on rank `dst` (a list in rank order), None elsewhere."""
    if not _active():
        return [obj]
    out = [None] * dist.get_world_size() if dist.get_rank() == dst else None
    dist.gather_object(obj, out, dst=dst)
    return out

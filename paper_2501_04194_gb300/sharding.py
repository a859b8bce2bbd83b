"""Splitting a batch of traces over several GPUs (one process per GPU).

Robustness traces of different traces are independent, so a batch shards with no exchange
step at all: each rank evaluates its own traces and nothing is communicated on the data path
(weak scaling).  The only collective is the host-side max of the per-rank times a benchmark
reports.  A dense batch splits into contiguous trace ranges; a ragged batch (traces of
different lengths and formulas in one persistent launch) is balanced by its cost, the sum of
trace length times a per-formula cost, with the longest-processing-time-first rule.
"""
from __future__ import annotations

import heapq

import numpy as np


def shard_dense(B: int, world: int, rank: int) -> slice:
    """Traces [start, stop) of rank ``rank`` out of ``world`` for a dense batch of B traces
    (sizes differ by at most one)."""
    if world < 1 or not 0 <= rank < world or B < 0:
        raise ValueError("need world >= 1, 0 <= rank < world, B >= 0")
    q, r = divmod(B, world)
    start = rank * q + min(rank, r)
    return slice(start, start + q + (1 if rank < r else 0))


def shard_ragged(lengths, world: int, formula_id=None, formula_cost=None) -> list[np.ndarray]:
    """Trace indices of every rank for a ragged batch: traces sorted by cost (length x the cost
    of their formula, 1 by default), each given to the least-loaded rank so far.  Returns one
    sorted int64 index array per rank; together they hold every trace exactly once."""
    lengths = np.asarray(lengths, dtype=np.int64)
    if world < 1:
        raise ValueError("world must be >= 1")
    cost = lengths.astype(np.float64)
    if formula_cost is not None:
        if formula_id is None:
            raise ValueError("formula_cost needs formula_id")
        cost = cost * np.asarray(formula_cost, dtype=np.float64)[np.asarray(formula_id)]
    order = np.argsort(-cost, kind="stable")
    heap = [(0.0, r) for r in range(world)]
    parts: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(int(i))
        heapq.heappush(heap, (load + float(cost[i]), r))
    return [np.sort(np.asarray(p, dtype=np.int64)) for p in parts]


def max_over_ranks(value: float) -> float:
    """Largest ``value`` over the ranks of the default process group (the value itself when no
    group is initialised); the tensor lives on the GPU for NCCL groups, on the CPU otherwise."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())

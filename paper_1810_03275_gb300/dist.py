"""Multi-process helpers: slices are independent problems, so ranks share no data on
the solve path -- each rank takes a subset of the slices (balanced by their
per-iteration cost n^2 * views) and only timings are reduced across ranks."""
from __future__ import annotations

import os
from typing import List, Sequence, Tuple


def world() -> Tuple[int, int, int]:
    """(rank, world size, local rank) from the torchrun environment (1 process if unset)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return rank, ws, int(os.environ.get("LOCAL_RANK", rank))


def init(backend: str = None) -> Tuple[int, int, int]:
    import torch
    import torch.distributed as dist
    rank, ws, local = world()
    if ws > 1 and not dist.is_initialized():
        if backend is None:
            backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return rank, ws, local


def shard(costs: Sequence[float], rank: int, ws: int) -> List[int]:
    """Indices of the slices rank `rank` solves: longest-processing-time greedy
    assignment of the costs to `ws` ranks (deterministic, ties by index)."""
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    load = [0.0] * ws
    owner = [0] * len(costs)
    for i in order:
        r = min(range(ws), key=lambda k: (load[k], k))
        owner[i] = r
        load[r] += float(costs[i])
    return [i for i in range(len(costs)) if owner[i] == rank]


def _reduce(x: float, op) -> float:
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(x: float) -> float:
    import torch.distributed as dist
    return _reduce(x, dist.ReduceOp.MAX)


def sum_over_ranks(x: float) -> float:
    import torch.distributed as dist
    return _reduce(x, dist.ReduceOp.SUM)


def barrier() -> None:
    import torch.distributed as dist
    if dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()

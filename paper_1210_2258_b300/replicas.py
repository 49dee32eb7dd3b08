"""Several GPUs: independent replicas, no collective on the data path.

A single image does not shard (every pass of an iteration needs the whole image), so N GPUs run
N independent problems: replicas of the benchmark workload, or disjoint shares of a batch of
problems.  The only communication is the timing summary: the slowest rank's time and the total of
the iterations all ranks performed (torch.distributed, gloo on CPU tensors or NCCL on CUDA ones).
"""
from __future__ import annotations


def shard(sizes: list[int], rank: int, world: int) -> list[int]:
    """Problem indices of `rank` for a batch with the given pixel counts: problems are dealt
    largest first to the rank with the least work so far (ties to the lower rank), so every rank
    gets a similar number of pixels and every problem is on exactly one rank."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    load = [0] * world
    mine = []
    for i in sorted(range(len(sizes)), key=lambda k: (-sizes[k], k)):
        r = min(range(world), key=lambda q: (load[q], q))
        load[r] += sizes[i]
        if r == rank:
            mine.append(i)
    return sorted(mine)


def aggregate(total_ms: float, iterations: int, device=None) -> tuple[float, int]:
    """(max over ranks of total_ms, sum over ranks of iterations); the inputs unchanged on a
    single process.  `device` is where the reduction tensors live (a CUDA device for NCCL)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(total_ms), int(iterations)
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    n = torch.tensor([float(iterations)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t.item()), int(round(n.item()))

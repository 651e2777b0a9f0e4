"""One process per GPU: how work is split over ranks and how a job-level number is formed.

Sequences (and key-frame groups) are independent, so ranks share no data during an encode:
each rank takes its own units and the job's throughput is the points of all ranks divided by
the slowest rank's time.  The only collectives are these two reductions (and a barrier around
the timed region); they run on whatever process group the caller set up (NCCL on GPUs, gloo
on CPU).
"""
from __future__ import annotations


def shard(n_units: int, rank: int, world: int) -> list:
    """Units (e.g. sequence indices of a table) of one rank: round-robin, disjoint, covering all."""
    if not (0 <= rank < world):
        raise ValueError("rank out of range")
    return list(range(rank, n_units, world))


def job_value(points_local: float, seconds_local: float, dist=None, device="cpu"):
    """(throughput in Mpoints/s, slowest rank's seconds, all ranks' points) of one timed region.
    Without a process group the numbers are the local ones."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return points_local / seconds_local / 1e6, seconds_local, points_local
    import torch
    t = torch.tensor([float(seconds_local)], dtype=torch.float64, device=device)
    p = torch.tensor([float(points_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(p, op=dist.ReduceOp.SUM)
    seconds, points = float(t.item()), float(p.item())
    return points / seconds / 1e6, seconds, points

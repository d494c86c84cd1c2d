"""Weak scaling across ranks (one process per GPU).

Rays, stars and images are independent, so N ranks each trace their own
seeded copy of the workload with no collective on the data path; only the
timing and the unit counts are combined once at the end: the timed region is
the maximum over ranks, the units the sum.
"""
from __future__ import annotations


def rank_seeds(base_seed: int, nsub: int, rank: int) -> list[int]:
    """Seeds of the sub-batches of one rank (rank 0: the single-GPU workload)."""
    return [base_seed * 1000 + j + 100000 * rank for j in range(nsub)]


def reduce_totals(seconds: float, accepted: float, rays: float, device=None):
    """(max over ranks of seconds, sum of accepted steps, sum of rays); the
    inputs unchanged without an initialised process group of size > 1."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return seconds, accepted, rays
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([accepted, rays], dtype=torch.float64, device=device)
    dist.all_reduce(c)
    return float(t[0]), float(c[0]), float(c[1])

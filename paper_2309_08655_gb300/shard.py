"""One workload split across ranks (one process per GPU).

Rays, stars and images are independent; the paper's own tracers run in
parallel on computing clusters (Sec. 2.4).  Here one workload's rays are split
into contiguous ranges, one per rank (or, for a batch of uneven instances,
whole instances are assigned to ranks by their expected cost).  Each rank
samples its range with the weight normalisation of the whole workload
(``rt_sample_conversion_surface_part`` / ``rt_batch_set_norm``), traces it, and
bins it into int64 fixed-point sums (``rt_bin_part_*``).  The only data-path
collectives are the exact reduction of those sums: a MAX all-reduce of the
largest escaped weight (it fixes the common fixed-point scale) before
accumulation, and a SUM all-reduce of the int64 sums after it.  Integer
addition does not depend on the order, so the combined spectrum is bitwise
that of one GPU binning every ray.  The benchmark's timing is combined at the
end: the timed region is the maximum over ranks, the units the sum.
"""
from __future__ import annotations


def _world():
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return None
    return dist if dist.get_world_size() > 1 else None


def ray_range(n_total: int, world: int, rank: int) -> tuple[int, int]:
    """(first, count) of rank's contiguous share of n_total rays; the shares
    differ by at most one ray and cover 0 .. n_total - 1 in rank order."""
    if world < 1 or not 0 <= rank < world or n_total < 0:
        raise ValueError("need world >= 1, 0 <= rank < world, n_total >= 0")
    base, extra = divmod(n_total, world)
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def partition_by_cost(costs, world: int) -> list[int]:
    """Owner rank of each instance: longest-processing-time-first (each
    instance, in order of decreasing expected cost, to the rank with the least
    cost so far; ties to the lower index), deterministic on every rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    load = [0.0] * world
    owner = [0] * len(costs)
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        owner[i] = r
        load[r] += float(costs[i])
    return owner


def reduce_max_(t):
    """In place: element-wise MAX over ranks (int64 bit patterns of
    non-negative doubles order like their values).  Identity on one rank."""
    d = _world()
    if d is None:
        return t
    c = t.contiguous()
    d.all_reduce(c, op=d.ReduceOp.MAX)
    if c.data_ptr() != t.data_ptr():
        t.copy_(c)
    return t


def reduce_sum_(t):
    """In place: element-wise SUM over ranks (exact for int64).  Identity on
    one rank."""
    d = _world()
    if d is None:
        return t
    c = t.contiguous()
    d.all_reduce(c)
    if c.data_ptr() != t.data_ptr():
        t.copy_(c)
    return t


def bin_sharded(rt, stars, offsets, ld, n_totals, state, weight, status, nbins, nu_lo, nu_hi,
                acc, hist, out_of_range, stream=None):
    """Per-star spectra of a batch whose stars hold this rank's share of
    their rays, combined over ranks: for star s, rays offsets[s] ..
    offsets[s + 1] - 1 of the batch arrays (state row stride ld), n_totals[s]
    rays over all ranks.  acc: (nstars, RT_BIN_ACC_ENTRIES) int64 device
    scratch; hist: (nstars, nth, nph, nnu), out_of_range: (nstars,) float64."""
    nth, nph, nnu = nbins
    for s in range(len(stars)):
        o, n = offsets[s], offsets[s + 1] - offsets[s]
        rt.rt_bin_part_max(n, weight[o:], status[o:], nth, nph, nnu, acc[s], stream=stream)
    reduce_max_(acc[:, 0])
    for s, star in enumerate(stars):
        o, n = offsets[s], offsets[s + 1] - offsets[s]
        rt.rt_bin_part_accumulate(star, n, n_totals[s], state[:, o:], weight[o:], status[o:],
                                  nth, nph, nnu, nu_lo, nu_hi, acc[s], ld=ld, stream=stream)
    reduce_sum_(acc[:, 1:])
    for s in range(len(stars)):
        rt.rt_bin_part_finalize(nth, nph, nnu, n_totals[s], acc[s], hist[s], None, None,
                                out_of_range[s:s + 1], stream=stream)


def reduce_totals(seconds: float, accepted: float, rays: float, device=None):
    """(max over ranks of seconds, sum of accepted steps, sum of rays); the
    inputs unchanged without an initialised process group of size > 1."""
    import torch
    d = _world()
    if d is None:
        return seconds, accepted, rays
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    d.all_reduce(t, op=d.ReduceOp.MAX)
    c = torch.tensor([accepted, rays], dtype=torch.float64, device=device)
    d.all_reduce(c)
    return float(t[0]), float(c[0]), float(c[1])

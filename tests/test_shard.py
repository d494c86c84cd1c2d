"""Sharding host logic on CPU, and the exact reduction of fixed-point sums on
two gloo ranks.

Each rank takes its contiguous range of one workload's rays from
``shard.ray_range``, forms int64 fixed-point partial sums of its rays (the
fixed-point rule of the binning kernels, written out here in numpy: q =
rint(w 2^e) with 2^e the largest power of two keeping n_total x w_max x 2^e
below 2^62), and feeds them to the product's reductions; the reduced sums
must equal the single-rank sums bit for bit."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2309_08655_gb300 import shard  # noqa: E402

NRAYS, NBINS = 10007, 37


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _workload():
    rng = np.random.default_rng(5)
    w = rng.lognormal(-30.0, 3.0, NRAYS)          # weights spanning many decades [W]
    escaped = rng.random(NRAYS) < 0.7
    bins = rng.integers(0, NBINS, NRAYS)
    return w, escaped, bins


def _scale(wmax_bits: int, n_total: int) -> float:
    wmax = np.array([wmax_bits], dtype=np.int64).view(np.float64)[0]
    if not wmax > 0:
        return 1.0
    _, ex = np.frexp(wmax * n_total)              # wmax n = m 2^ex, m in [1/2, 1)
    return float(np.ldexp(1.0, 61 - (int(ex) - 1)))


def _partial(w, escaped, bins, first, count, wmax_bits, n_total):
    """[max bits | out-of-range | histogram] of rays first .. first + count - 1."""
    sl = slice(first, first + count)
    acc = np.zeros(2 + NBINS, dtype=np.int64)
    sc = _scale(wmax_bits, n_total)
    q = np.rint(w[sl][escaped[sl]] * sc).astype(np.int64)
    np.add.at(acc, 2 + bins[sl][escaped[sl]], q)
    acc[0] = wmax_bits
    return acc


def _max_bits(w, escaped, first, count):
    sl = slice(first, first + count)
    we = w[sl][escaped[sl]]
    return int(we.max().view(np.int64)) if we.size else 0


def _worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, escaped, bins = _workload()
        first, count = shard.ray_range(NRAYS, world, rank)
        m = torch.tensor([_max_bits(w, escaped, first, count)], dtype=torch.int64)
        shard.reduce_max_(m)                       # the common fixed-point scale
        acc = torch.from_numpy(_partial(w, escaped, bins, first, count, int(m[0]), NRAYS))
        shard.reduce_sum_(acc[1:])                 # a strided view: copied and back
        np.save(os.path.join(out_dir, f"acc{rank}.npy"), acc.numpy())
        t, a, r = shard.reduce_totals(1.0 + rank, 100.0 * (rank + 1), 10.0 + rank)
        with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
            f.write(f"{t} {a} {r}\n")
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_ray_ranges_cover_the_workload_once():
    for n in (0, 1, 5, 65536, 10007):
        for world in (1, 2, 3, 8):
            ranges = [shard.ray_range(n, world, r) for r in range(world)]
            assert ranges[0][0] == 0
            for (f0, c0), (f1, _) in zip(ranges, ranges[1:]):
                assert f0 + c0 == f1
            assert sum(c for _, c in ranges) == n
            assert max(c for _, c in ranges) - min(c for _, c in ranges) <= 1
    assert shard.ray_range(100, 1, 0) == (0, 100)
    with pytest.raises(ValueError):
        shard.ray_range(10, 2, 2)


def test_partition_by_cost_is_balanced_and_deterministic():
    rng = np.random.default_rng(3)
    costs = np.exp(rng.uniform(np.log(1e3), np.log(1e6), 256))   # config-3-like ray counts
    for world in (1, 2, 4, 8):
        owner = shard.partition_by_cost(costs, world)
        assert owner == shard.partition_by_cost(list(costs), world)
        load = np.bincount(owner, weights=costs, minlength=world)
        assert load.sum() == pytest.approx(costs.sum())
        # LPT: no rank exceeds the mean by more than the largest instance
        assert load.max() <= costs.sum() / world + costs.max()
    assert shard.partition_by_cost([5.0, 5.0, 1.0], 2) == [0, 1, 0]
    assert shard.partition_by_cost([1.0, 5.0, 5.0], 2) == [0, 0, 1]


def test_reductions_without_process_group_are_identity():
    t = torch.arange(5, dtype=torch.int64)
    assert torch.equal(shard.reduce_sum_(t.clone()), t)
    assert torch.equal(shard.reduce_max_(t.clone()), t)
    assert shard.reduce_totals(2.5, 7.0, 3.0) == (2.5, 7.0, 3.0)


def test_fixed_point_rule_keeps_sums_below_2_62():
    w, escaped, _ = _workload()
    b = _max_bits(w, escaped, 0, NRAYS)
    sc = _scale(b, NRAYS)
    wmax = np.array([b], dtype=np.int64).view(np.float64)[0]
    assert wmax * NRAYS * sc < 2.0 ** 62 and wmax * NRAYS * sc >= 2.0 ** 61


def test_sharded_sums_equal_single_rank_bitwise(tmp_path):
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    w, escaped, bins = _workload()
    single = _partial(w, escaped, bins, 0, NRAYS, _max_bits(w, escaped, 0, NRAYS), NRAYS)
    for r in range(2):
        acc = np.load(tmp_path / f"acc{r}.npy")
        assert np.array_equal(acc, single)        # bit for bit, every rank
        t, a, n = map(float, open(tmp_path / f"r{r}.txt").read().split())
        assert (t, a, n) == (2.0, 300.0, 21.0)     # max time, summed units
    assert single[2:].sum() > 0

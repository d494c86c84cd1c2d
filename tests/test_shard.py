"""Weak-scaling host logic on two gloo ranks (CPU): per-rank seeds are
disjoint and rank 0 reproduces the single-GPU workload; the end-of-run
reduction takes the maximum time and sums the units."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2309_08655_gb300 import shard  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t, acc, rays = shard.reduce_totals(1.0 + rank, 100.0 * (rank + 1), 10.0 + rank)
        with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
            f.write(f"{t} {acc} {rays}\n")
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_rank_seeds():
    s0 = shard.rank_seeds(1, 16, 0)
    s1 = shard.rank_seeds(1, 16, 1)
    assert s0 == [1000 + j for j in range(16)]
    assert not set(s0) & set(s1)


def test_reduce_totals_without_process_group_is_identity():
    assert shard.reduce_totals(2.5, 7.0, 3.0) == (2.5, 7.0, 3.0)


def test_reduce_totals_two_gloo_ranks(tmp_path):
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    for r in range(2):
        t, acc, rays = map(float, open(tmp_path / f"r{r}.txt").read().split())
        assert t == 2.0                 # max over ranks
        assert acc == 300.0             # 100 + 200
        assert rays == 21.0             # 10 + 11

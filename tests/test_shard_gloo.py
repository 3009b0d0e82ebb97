"""Sharded shell sum over two CPU ranks (gloo): each rank sums its group-aligned piece of the shell
range with the oracle, the fixed-order reduction adds the pieces, and every rank holds the full
tensor, equal to the single-process sum (shell-range additivity) and identical across ranks.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as tmp

from oracle import booster as ob
from oracle import vertex as ov
from paper_2107_13952_gb300 import shard

TJ, DL, SEED = (3, 2, 4, 3, 1, 4, 4, 4, 1, 4), 1, 4


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, outdir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b, e = shard.rank_range(DL, world, rank)
        bs = ob.random_boosters(TJ, DL, SEED)
        A = ov.vertex_amplitude(TJ, DL, bs, shells=range(b, e))
        (full,) = shard.reduce_fixed_order([torch.from_numpy(A)])
        np.save(os.path.join(outdir, "rank%d.npy" % rank), full.numpy())
    finally:
        dist.destroy_process_group()


def test_rank_ranges_partition_the_shells():
    for dl in (0, 1, 3, 10):
        for world in (1, 2, 3, 8):
            pieces = [shard.rank_range(dl, world, r) for r in range(world)]
            assert pieces[0][0] == 0 and pieces[-1][1] == (dl + 1) ** 6
            for (b0, e0), (b1, e1) in zip(pieces, pieces[1:]):
                assert e0 == b1 and b0 <= e0
            assert all(b % (dl + 1) ** 3 == 0 for b, _ in pieces)
    with pytest.raises(ValueError):
        shard.rank_range(1, 2, 2)


def test_two_rank_fixed_order_reduction(tmp_path):
    world = 2
    tmp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    r0 = np.load(tmp_path / "rank0.npy")
    r1 = np.load(tmp_path / "rank1.npy")
    assert np.array_equal(r0, r1)
    full = ov.vertex_amplitude(TJ, DL, ob.random_boosters(TJ, DL, SEED))
    assert np.linalg.norm(full) > 0
    assert np.linalg.norm(r0 - full) <= 1e-13 * np.linalg.norm(full)

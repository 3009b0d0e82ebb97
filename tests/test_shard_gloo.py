"""Sharded shell sums on CPU processes (no GPU): the cost-weighted split of the shell range, the
fixed-order reduction over two gloo ranks, and the recomputation of a lost rank's piece.

* pieces partition [0, (dl+1)^6) on group boundaries; the cost-weighted pieces carry near-equal
  shares of the canonical flop count (the split the paper's MPI distribution needs, Sec. 3
  "Parallelization");
* two gloo ranks: each sums its piece with the oracle, ``reduce_fixed_order`` adds them, every rank
  holds the single-process sum, bitwise identical across ranks;
* three processes share a FileStore; one leaves before publishing its piece (between steps, with
  nothing in flight); the survivors notice within the short limit, one of them recomputes the
  missing piece, and both return the full sum, bitwise identical.
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
from paper_2107_13952_gb300 import shard, shells

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
        b, e = shard.rank_range(DL, world, rank, shells.group_costs(TJ, DL))
        bs = ob.random_boosters(TJ, DL, SEED)
        A = ov.vertex_amplitude(TJ, DL, bs, shells=range(b, e))
        (full,) = shard.reduce_fixed_order([torch.from_numpy(A)])
        np.save(os.path.join(outdir, "rank%d.npy" % rank), full.numpy())
    finally:
        dist.destroy_process_group()


def test_rank_ranges_partition_the_shells():
    for dl in (0, 1, 3, 10):
        for world in (1, 2, 3, 8):
            for costs in (None, shells.group_costs((16,) * 10, dl) if dl == 10 else None):
                pieces = shard.shard_ranges(dl, world, costs)
                assert pieces[0][0] == 0 and pieces[-1][1] == (dl + 1) ** 6
                for (b0, e0), (b1, e1) in zip(pieces, pieces[1:]):
                    assert e0 == b1 and b0 <= e0
                assert all(b % (dl + 1) ** 3 == 0 for b, _ in pieces)
    with pytest.raises(ValueError):
        shard.rank_range(1, 2, 2)


def test_cost_weighted_pieces_balance_the_work():
    dl = 10
    costs = shells.group_costs((16,) * 10, dl)
    D3 = (dl + 1) ** 3
    for world in (2, 4, 8):
        even = [costs[b // D3:e // D3].sum() for b, e in shard.shard_ranges(dl, world)]
        weighted = [costs[b // D3:e // D3].sum() for b, e in shard.shard_ranges(dl, world, costs)]
        share = costs.sum() / world
        # within one group's cost of the equal share, and an imbalance (max/min - 1) at least ten
        # times smaller than that of the group-count split (10-30 % for the spin-8 vertex)
        assert max(abs(w - share) for w in weighted) <= costs.max()
        assert max(weighted) / min(weighted) - 1 <= 0.1 * (max(even) / min(even) - 1)


def test_two_rank_fixed_order_reduction(tmp_path):
    world = 2
    tmp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    r0 = np.load(tmp_path / "rank0.npy")
    r1 = np.load(tmp_path / "rank1.npy")
    assert np.array_equal(r0, r1)
    full = ov.vertex_amplitude(TJ, DL, ob.random_boosters(TJ, DL, SEED))
    assert np.linalg.norm(full) > 0
    assert np.linalg.norm(r0 - full) <= 1e-13 * np.linalg.norm(full)


def _resilient_worker(rank, world, store_path, outdir, lost):
    store = dist.FileStore(store_path, world)
    ranges = shard.shard_ranges(DL, world, shells.group_costs(TJ, DL))
    if rank == lost:
        return          # this process leaves before its step: nothing of it is in flight
    bs = ob.random_boosters(TJ, DL, SEED)

    def compute(b, e):
        return ov.vertex_amplitude(TJ, DL, bs, shells=range(b, e))
    total, redone = shard.resilient_sum(store, world, rank, ranges, compute, wait_s=1.0)
    np.save(os.path.join(outdir, "rank%d.npy" % rank), total)
    np.save(os.path.join(outdir, "redone%d.npy" % rank), np.array(redone, dtype=np.int64))


def test_lost_rank_is_recomputed(tmp_path):
    world, lost = 3, 1
    store_path = str(tmp_path / "store")
    tmp.spawn(_resilient_worker, args=(world, store_path, str(tmp_path), lost), nprocs=world, join=True)
    full = ov.vertex_amplitude(TJ, DL, ob.random_boosters(TJ, DL, SEED))
    got = [np.load(tmp_path / ("rank%d.npy" % r)) for r in range(world) if r != lost]
    assert np.array_equal(got[0], got[1])
    assert np.linalg.norm(got[0] - full) <= 1e-13 * np.linalg.norm(full)
    redone = sorted(int(v) for r in range(world) if r != lost for v in np.load(tmp_path / ("redone%d.npy" % r)))
    assert redone == [lost]       # exactly one survivor recomputed the missing piece

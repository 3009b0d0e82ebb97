"""The split shell sum through the library, as separate processes sharing one GPU (each builds
the tables its piece reads and sums its piece; the pieces do not wait on each other on the
device). One process leaves before its step; the survivors recompute its piece through the
library and every survivor returns the whole sum, bitwise identical across survivors and within
1e-13 of the single-process sum."""
import os

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as tmp

pytestmark = pytest.mark.gpu

TJ, GAMMA, DL, RULE = (5, 3, 4, 4, 6, 3, 4, 3, 4, 4), 1.2, 3, (40.0, 4, 10)


def _worker(rank, world, store_path, outdir, lost):
    import paper_2107_13952_gb300 as sf
    from paper_2107_13952_gb300 import shard, shells
    store = dist.FileStore(store_path, world)
    ranges = shard.shard_ranges(DL, world, shells.group_costs(TJ, DL))
    if rank == lost:
        return            # leaves before its step: nothing of it is in flight
    torch.cuda.set_device(0)
    sf.load()

    def compute(b, e):
        t = sf.sf_6j_table([sf.vertex(TJ, GAMMA, DL)], shell_range=(b, e))
        sf.sf_boosters(t, RULE)
        return sf.sf_vertex_amplitude(t, sf.SF_FP64, b, e)[0].cpu().numpy()
    total, redone = shard.resilient_sum(store, world, rank, ranges, compute, wait_s=5.0)
    np.save(os.path.join(outdir, "rank%d.npy" % rank), total)
    np.save(os.path.join(outdir, "redone%d.npy" % rank), np.array(redone, dtype=np.int64))


def test_split_sum_with_a_lost_process(lib, tmp_path):
    world, lost = 3, 2
    tmp.spawn(_worker, args=(world, str(tmp_path / "store"), str(tmp_path), lost), nprocs=world, join=True)
    t = lib.sf_6j_table([lib.vertex(TJ, GAMMA, DL)])
    lib.sf_boosters(t, RULE)
    full = lib.sf_vertex_amplitude(t)[0].cpu().numpy()
    got = [np.load(tmp_path / ("rank%d.npy" % r)) for r in range(world) if r != lost]
    assert np.array_equal(got[0], got[1])
    assert np.linalg.norm(got[0] - full) <= 1e-13 * np.linalg.norm(full)
    redone = sorted(int(v) for r in range(world) if r != lost for v in np.load(tmp_path / ("redone%d.npy" % r)))
    assert redone == [lost]

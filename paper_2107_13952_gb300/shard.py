"""Splitting one vertex's shell sum over processes, summing the partial tensors back, and
recomputing the piece of a process that left.

Shells are independent terms of the sum (Sec. 2 eq. vertex-ampl), so a process group divides the
linear shell range [0, (dl+1)^6) into contiguous pieces, each process runs
``sf_vertex_amplitude`` on its piece, and one reduction of the output tensor (D_i1..D_i5 doubles)
finishes the sum. The paper distributes the shell loops over MPI nodes (Sec. 3
"Parallelization"); here the pieces are aligned to groups of (dl+1)^3 shells (one
(l25, l35, l45) triple, the unit the shell kernel schedules) and balanced by cost: the prefix sums
of the per-group canonical flop count (``shells.group_costs``) are cut at equal fractions, so a
rank that gets the costly large-l25 groups gets fewer of them.

Two reductions:
* ``reduce_fixed_order``: all-gather over a process group and add in rank order on every rank
  (bitwise identical results everywhere, independent of the backend's internal order);
* ``resilient_sum``: through a key-value store (torch.distributed Store, e.g. a FileStore on a
  shared file system, which outlives any rank): every rank publishes its piece; a piece whose owner
  has not published within a short limit (the owner left between steps) is claimed by one survivor
  through an atomic counter and recomputed; every survivor then adds all pieces in rank order.
  No collective is involved, so a departed rank cannot block the others.
"""
import io
import time

import numpy as np


def _cut(costs, world):
    """Group boundaries g_0 = 0 <= g_1 <= ... <= g_world = len(costs) at equal fractions of the
    cumulative cost (the first group whose prefix reaches r/world of the total)."""
    c = np.asarray(costs, dtype=np.float64)
    n = len(c)
    pref = np.concatenate([[0.0], np.cumsum(c)])
    tot = pref[-1]
    bounds = [0]
    for r in range(1, world):
        if tot <= 0:
            g = n * r // world
        else:
            g = int(np.searchsorted(pref, tot * r / world, side="left"))
        bounds.append(min(max(g, bounds[-1]), n))
    bounds.append(n)
    return bounds


def shard_ranges(dl, world, costs=None):
    """[begin, end) of the linear shell indices of every rank of ``world``: group-aligned pieces,
    balanced by ``costs`` (one value per group, e.g. ``shells.group_costs``) or, without costs, by
    group count."""
    if world < 1:
        raise ValueError("world size %d" % world)
    D = int(dl) + 1
    per_group = D ** 3
    ngroups = D ** 3
    if costs is None:
        bounds = [ngroups * r // world for r in range(world + 1)]
    else:
        if len(costs) != ngroups:
            raise ValueError("need %d group costs, got %d" % (ngroups, len(costs)))
        bounds = _cut(costs, world)
    return [(bounds[r] * per_group, bounds[r + 1] * per_group) for r in range(world)]


def rank_range(dl, world, rank, costs=None):
    """[begin, end) of the linear shell indices that ``rank`` of ``world`` sums."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank %d outside a world of %d" % (rank, world))
    return shard_ranges(dl, world, costs)[rank]


def reduce_fixed_order(partials, group=None):
    """Sum each tensor of ``partials`` over the ranks of ``group``, in rank order, on every rank.

    ``partials``: list of tensors (same shapes and dtypes on every rank). Returns new tensors.
    """
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    out = []
    for p in partials:
        parts = [torch.empty_like(p) for _ in range(world)]
        dist.all_gather(parts, p.contiguous(), group=group)
        acc = parts[0].clone()
        for q in parts[1:]:
            acc += q
        out.append(acc)
    return out


def _put(store, key, arr):
    buf = io.BytesIO()
    np.save(buf, np.ascontiguousarray(arr), allow_pickle=False)
    store.set(key, buf.getvalue())


def _get(store, key):
    return np.load(io.BytesIO(store.get(key)), allow_pickle=False)


def resilient_sum(store, world, rank, ranges, compute, wait_s=2.0, poll_s=0.02, tag="step"):
    """Sum the pieces ``compute(begin, end)`` (numpy float64 arrays of one shape) over ``ranges``
    (one per rank), tolerating ranks that leave before publishing their piece.

    Rank ``rank`` computes and publishes its own piece under ``tag``, then waits up to ``wait_s``
    seconds for the others. A piece still missing after that is claimed by the first survivor to
    increment its claim counter (Store.add is atomic), which recomputes and publishes it; the other
    survivors keep waiting for it (bounded by ``wait_s`` after the claim, then they claim it too:
    pieces are deterministic, so a duplicate is identical). Returns (sum in rank order, list of
    ranks whose pieces this rank recomputed)."""
    mine = compute(*ranges[rank])
    _put(store, "%s/part/%d" % (tag, rank), mine)
    store.set("%s/done/%d" % (tag, rank), b"1")
    recomputed = []

    def have(r):
        return store.check(["%s/done/%d" % (tag, r)])

    def redo(r):
        _put(store, "%s/part/%d" % (tag, r), compute(*ranges[r]))
        store.set("%s/done/%d" % (tag, r), b"1")
        recomputed.append(r)

    deadline = time.time() + wait_s
    claimed_at = {}
    others = [r for r in range(world) if r != rank]
    while True:
        missing = [r for r in others if not have(r)]
        if not missing:
            break
        now = time.time()
        if now >= deadline:
            for r in missing:
                if r not in claimed_at:
                    claimed_at[r] = now
                    if store.add("%s/claim/%d" % (tag, r), 1) == 1:   # this rank won the claim
                        redo(r)
                elif now > claimed_at[r] + wait_s:                     # the claimant left as well
                    redo(r)
        time.sleep(poll_s)
    acc = None
    for r in range(world):
        p = mine if r == rank else _get(store, "%s/part/%d" % (tag, r))
        acc = p.copy() if acc is None else acc + p
    return acc, recomputed

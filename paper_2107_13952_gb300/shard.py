"""Splitting one vertex's shell sum over processes, and summing the partial tensors back.

Shells are independent terms of the sum (Sec. 2 eq. vertex-ampl), so a process group divides the
linear shell range [0, (dl+1)^6) into contiguous pieces, each process runs
``sf_vertex_amplitude`` on its piece, and one reduction of the output tensor (D_i1..D_i5 doubles)
finishes the sum. Pieces are aligned to groups of (dl+1)^3 shells (one (l25, l35, l45) triple),
the unit the shell kernel schedules, and balanced by group count.

The reduction gathers every rank's partial tensor and adds them in rank order on every rank, so
the result is bitwise identical on all ranks and independent of the collective's internal order
(an all_reduce would leave the order to the backend).
"""


def rank_range(dl, world, rank):
    """[begin, end) of the linear shell indices that ``rank`` of ``world`` sums."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank %d outside a world of %d" % (rank, world))
    D = int(dl) + 1
    per_group = D ** 3
    ngroups = D ** 3
    g0 = ngroups * rank // world
    g1 = ngroups * (rank + 1) // world
    return g0 * per_group, g1 * per_group


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

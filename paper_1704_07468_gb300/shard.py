"""Mask-sharded Gram computation across ranks.

Every (level m, position mask) pass of countAndUpdate is independent of the
others, and the cumulative mismatch profile C_m is the sum of the passes'
contributions (Section 2.2, "Parallelization"; Section S:5.3; Eq. 8).  A
dataset's c_gk masks are therefore split into contiguous slices, one per
rank; each rank computes its slice's C_0..C_M with
``gakco_gram_partial_device``, one sum all-reduce of the (M+1) x n x n
int32 buffers exchanges them, and every rank finishes with
``gakco_combine_device`` (Eq. 9, Eq. 7, normalisation).

Every contribution is a non-negative count and their sum is a C_m entry,
which the engine keeps below 2^31, so the int32 sum never overflows and is
exact in any order.  The all-reduce is the only collective; it runs through
``torch.distributed`` (NCCL on GPUs, gloo on CPU) on plain device buffers,
with no multicast loads of peer memory.
"""

from __future__ import annotations

__all__ = ["mask_slices", "rank_world", "sharded_profile", "sharded_gram"]


def mask_slices(nmasks, world, weights=None):
    """Split masks 0..nmasks-1 (level order) into ``world`` contiguous
    slices [begin, end) of near-equal total weight (default: one per mask).
    Slices may be empty when there are more ranks than masks."""
    if world < 1:
        raise ValueError("world must be >= 1")
    if nmasks < 0:
        raise ValueError("nmasks must be >= 0")
    w = [1.0] * nmasks if weights is None else [float(v) for v in weights]
    if len(w) != nmasks or any(v < 0 for v in w):
        raise ValueError("need one non-negative weight per mask")
    total = sum(w)
    bounds = [0]
    acc, i = 0.0, 0
    for r in range(1, world):
        target = total * r / world
        while i < nmasks and acc + w[i] / 2.0 <= target:
            acc += w[i]
            i += 1
        bounds.append(max(i, bounds[-1]))
    bounds.append(nmasks)
    return [(bounds[r], bounds[r + 1]) for r in range(world)]


def rank_world(group=None):
    """(rank, world size) of ``group``; (0, 1) without torch.distributed."""
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return 0, 1
    return dist.get_rank(group), dist.get_world_size(group)


def sharded_profile(partial, nmasks, C, group=None, weights=None):
    """Fill ``C`` (an int32 torch tensor of shape (M+1, n, n)) with the
    dataset's cumulative profiles: this rank calls ``partial(begin, end,
    C)`` for its slice of the masks, then one sum all-reduce over ``group``
    adds every rank's slice.  Returns this rank's (begin, end)."""
    import torch.distributed as dist

    rank, world = rank_world(group)
    begin, end = mask_slices(nmasks, world, weights)[rank]
    partial(begin, end, C)
    if world > 1:
        dist.all_reduce(C, op=dist.ReduceOp.SUM, group=group)
    return begin, end


def sharded_gram(ctx, codes_ptr, offsets, K, Khat=None, Nm=None, group=None, stream=None,
                 weights=None):
    """The Gram kernel of one dataset computed by all ranks of ``group``
    together.  ``codes_ptr`` is the device address of the dataset's codes on
    this rank's GPU, ``offsets`` the host int64 offsets; K (n x n int32),
    Khat (n x n float64) and Nm ((M+1) x n x n int32) are torch tensors on
    that GPU (Khat and Nm optional), written on every rank."""
    import torch

    n = len(offsets) - 1
    C = torch.empty((ctx.M + 1, n, n), dtype=torch.int32, device=K.device)

    def partial(begin, end, out):
        ctx.gram_partial_device(codes_ptr, offsets, begin, end, out.data_ptr(), stream)

    span = sharded_profile(partial, ctx.num_masks(), C, group, weights)
    ctx.combine_device(C.data_ptr(), n, K.data_ptr(),
                       Khat.data_ptr() if Khat is not None else None,
                       Nm.data_ptr() if Nm is not None else None, stream)
    return span

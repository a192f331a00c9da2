"""Data-parallel helpers: rays are independent, so views shard across ranks with no
exchange for rendering; a data-parallel fit sums the parameter gradients once per
step (the only collective the path has)."""


def shard_range(n, world, rank):
    """Contiguous [lo, hi) slice of n items for `rank` of `world` (sizes differ by <= 1)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad world/rank")
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def allreduce_sum_(tensors, group=None):
    """In-place sum of each tensor over the process group (fixed order of tensors)."""
    import torch.distributed as dist
    for t in tensors:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return tensors

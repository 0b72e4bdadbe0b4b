"""Sample sharding across ranks (host logic).

The LM step is additive over samples: every rank evaluates its contiguous
shard of the samples and contributes (sum |r|^2, J^T r, J^T J) partial sums;
one reduction of those partials per step gives the step of the whole sample
set.  The reduction gathers the partials and adds them in rank order, so the
result does not depend on the communication pattern.
"""
from __future__ import annotations


def shard_range(n: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous [begin, end) of rank `rank` out of `world` for n samples."""
    base, extra = divmod(n, world)
    b = rank * base + min(rank, extra)
    return b, b + base + (1 if rank < extra else 0)


def reduce_fixed_order(tensors, group=None):
    """Sum each tensor over ranks in rank order (all ranks receive the sum)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    out = []
    for t in tensors:
        parts = [torch.empty_like(t) for _ in range(world)]
        dist.all_gather(parts, t.contiguous(), group=group)
        s = parts[0].clone()
        for p in parts[1:]:
            s += p
        out.append(s)
    return out


def max_over_ranks(value: float, group=None) -> float:
    """The largest value of a scalar over ranks (slowest rank's time)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())

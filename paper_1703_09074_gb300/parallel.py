"""Rank bookkeeping for runs on several GPUs (one process per GPU).

The method partitions into independent problems (a batch of tensors, or
replicas of one decomposition), so ranks share no data: each rank takes its
own share of the problems, runs them on its own GPU, and only the timings are
combined (the slowest rank sets the step time).  torch.distributed carries
those few scalars; nothing of the decomposition crosses ranks.
"""

import torch


def rank_share(count, rank, world):
    """Indices of the problems rank ``rank`` of ``world`` runs: b = rank, rank + world, ..."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    return list(range(rank, count, world))


def _reduce(value, op, device):
    import torch.distributed as td
    if not (td.is_available() and td.is_initialized()) or td.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    td.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(value, device="cpu"):
    """The largest value over all ranks (the step time of the slowest rank)."""
    import torch.distributed as td
    return _reduce(value, td.ReduceOp.MAX, device)


def sum_over_ranks(value, device="cpu"):
    """The sum over all ranks (work done by the whole job)."""
    import torch.distributed as td
    return _reduce(value, td.ReduceOp.SUM, device)

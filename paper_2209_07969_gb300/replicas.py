"""Replica bookkeeping for several GPUs: independent simulations shard by request, with no
data-path collective; only the timing barrier and the max over ranks communicate."""


def shard(items, rank, world):
    """The requests rank `rank` of `world` runs: round-robin by index."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    return [it for i, it in enumerate(items) if i % world == rank]


def max_over_ranks(value, device=None):
    """Max of a float over the default process group (identity without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value, device=None):
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())

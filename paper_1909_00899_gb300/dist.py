"""Multi-process helpers for running the alignment path as one process per
GPU.  Every alignment is independent, so ranks never exchange data on the
path itself: each rank aligns its own replica (or shard) and only the timing
and the counts of work are combined, with the slowest rank deciding the
whole job's time."""
import os


def env():
    """(rank, world_size, local_rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(value, device=None):
    """The largest value over all ranks (the job's time is the slowest
    rank's); identity when torch.distributed is not initialised."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value, device=None):
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def shard(n, rank, world):
    """Contiguous [start, stop) share of n independent units for one rank."""
    per, rem = divmod(int(n), int(world))
    start = rank * per + min(rank, rem)
    return start, start + per + (1 if rank < rem else 0)

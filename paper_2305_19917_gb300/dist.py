"""Multi-process host logic (one process per GPU).

A triangular solve shards over right-hand sides with no exchange: for side
Left every column of X depends only on the same column of B (and on A, which
every rank holds), for side Right every row.  So N GPUs either solve N
independent problems (weak scaling) or split the right-hand sides of one
problem (strong scaling); neither needs a collective on the data path.  The
only collectives are host-side: a barrier around the timed region and the
maximum of the per-rank times.
"""
import os


def env_rank_world():
    """(rank, world_size, local_rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard_range(n, rank, world):
    """[start, stop) of the right-hand sides owned by `rank` when n of them
    are split as evenly as possible over `world` ranks (first n % world ranks
    get one more)."""
    if world <= 0 or not (0 <= rank < world) or n < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(n, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def max_over_ranks(value, device=None):
    """Maximum of a per-rank float over the default process group (returns
    `value` unchanged when no group is initialised)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()

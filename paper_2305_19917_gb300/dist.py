"""Multi-process solves (one process per GPU) and their host logic.

A triangular solve shards over right-hand sides with no exchange: for side
Left every column of X depends only on the same column of B (and on A, which
every rank holds), for side Right every row -- the paper's blocks spread over
several accelerators (Section V-C), cut along the independent direction.  So
N GPUs split the right-hand sides of one problem (solve_sharded): with a
fixed count per GPU that is weak scaling, with a fixed total strong scaling;
neither needs a collective on the data path.  The only collectives are
host-side: a barrier around the timed region and the maximum of the per-rank
times (and, where a caller wants X assembled on one rank, a gather after the
solve).
"""
import os


def env_rank_world():
    """(rank, world_size, local_rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard_range(n, rank, world, align=1):
    """[start, stop) of the right-hand sides owned by `rank` when n of them
    are split as evenly as possible over `world` ranks.  With align > 1 the
    split is made in whole groups of `align` right-hand sides (the last group
    possibly shorter), so every shard but the last starts and ends on a
    multiple of `align`; groups are dealt as evenly as possible (the first
    ranks get one more), and ranks beyond the number of groups get an empty
    range."""
    if world <= 0 or not (0 <= rank < world) or n < 0 or align < 1:
        raise ValueError("bad shard arguments")
    units = (n + align - 1) // align
    base, extra = divmod(units, world)
    u0 = rank * base + min(rank, extra)
    u1 = u0 + base + (1 if rank < extra else 0)
    return min(n, u0 * align), min(n, u1 * align)


# Right-hand sides per group of the mixed path's shards: its work is padded to
# whole 128-column tiles, so shards of whole tiles waste nothing.
SHARD_ALIGN = 128


def rhs_count(side, m, n):
    """Number of independent right-hand sides of an m x n B: its columns
    for side Left (op(A) X = alpha B), its rows for side Right."""
    return n if side == 0 else m


def shard_view(side, B, start, stop):
    """The part of the column-major B (torch tensor, m x n) that holds the
    right-hand sides [start, stop): columns for side Left, rows for side
    Right.  A view (no copy); it is itself a valid column-major operand with
    B's leading dimension."""
    return B[:, start:stop] if side == 0 else B[start:stop, :]


def solve_sharded(side, uplo, trans, diag, alpha, A, B, rank=None, world=None, total=None, path="mixed",
                  tol=1e-11, prec=0, max_iter=30, stream=None):
    """This rank's share of one triangular solve split over right-hand sides.

    Every rank holds all of A; the right-hand sides (columns of B for side
    Left, rows for side Right) are independent problems, so rank r solves
    the contiguous block shard_range(total, r, world, SHARD_ALIGN) in place
    with the library's solver, and no data moves between ranks.  With
    total=None, B is the whole m x n right-hand side and only the rank's
    block of it is read and written; otherwise B holds just the rank's block
    of a problem with `total` right-hand sides (its size must match).  path
    "mixed" runs gb_dtrsm_mixed (FP64 operands; tol / prec / max_iter as
    there), "plain" the plain gb_dtrsm / gb_strsm with the planner's plan.
    Returns (start, stop, status, iters, est_err) of this rank's block."""
    from . import api
    if rank is None or world is None:
        rank, world, _ = env_rank_world()
    m, n = B.shape
    if total is None:
        start, stop = shard_range(rhs_count(side, m, n), rank, world, SHARD_ALIGN)
        Bv = shard_view(side, B, start, stop)
    else:
        start, stop = shard_range(total, rank, world, SHARD_ALIGN)
        if rhs_count(side, m, n) != stop - start:
            raise ValueError(f"rank {rank}: B holds {rhs_count(side, m, n)} right-hand sides, "
                             f"its block has {stop - start}")
        Bv = B
    if Bv.numel() == 0:
        return start, stop, 0, 0, 0.0
    if path == "mixed":
        st, it, est = api.trsm_mixed(side, uplo, trans, diag, alpha, A, Bv, tol=tol, prec=prec, max_iter=max_iter,
                                     stream=stream)
        return start, stop, st, it, est
    if path != "plain":
        raise ValueError(f"unknown path {path!r}")
    api.trsm(side, uplo, trans, diag, alpha, A, Bv, stream=stream)
    return start, stop, 0, 0, 0.0


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

"""World-size-2 gloo tests of the multi-process host logic on CPU: shard
ranges tile the right-hand sides exactly (in whole 128-wide groups for the
sharded solve), the max-over-ranks reduction, and the sharded solve's own
block selection: each rank takes its block of B through the same view the
sharded solve hands to the library, marks it, and the marked blocks, gathered
over gloo, cover every right-hand side exactly once (columns for side Left,
rows for side Right).  The compute itself needs the GPU: the sharded solve
with the library's kernels is tested in test_dist_gpu.py."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2305_19917_gb300 import dist as gdist


def test_shard_range_tiles_exactly():
    for n in (0, 1, 7, 64, 1000, 16384):
        for world in (1, 2, 3, 4, 8):
            spans = [gdist.shard_range(n, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            for (a, b), (c, d) in zip(spans, spans[1:]):
                assert b == c
            sizes = [b - a for a, b in spans]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        gdist.shard_range(10, 2, 2)


def test_aligned_shards_are_whole_groups():
    al = gdist.SHARD_ALIGN
    for n in (0, 1, 127, 128, 129, 1000, 16384, 32768 + 5):
        for world in (1, 2, 3, 4, 8):
            spans = [gdist.shard_range(n, r, world, al) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            for (a, b), (c, d) in zip(spans, spans[1:]):
                assert b == c
            for a, b in spans:
                assert a == n or a % al == 0
                assert b == n or b % al == 0
            groups = [-(-(b - a) // al) for a, b in spans]
            assert max(groups) - min(groups) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, _ = gdist.env_rank_world()
        assert (r, w) == (rank, world)
        for side, (m, n) in ((0, (100, 300)), (1, (300, 100)), (0, (40, 3))):
            # column-major m x n, as the library takes it
            B = torch.zeros((n, m), dtype=torch.float64).t()
            total = gdist.rhs_count(side, m, n)
            a, b = gdist.shard_range(total, rank, world, gdist.SHARD_ALIGN)
            V = gdist.shard_view(side, B, a, b)
            assert V.stride(0) == 1 and (V.numel() == 0 or V.stride(1) == m)  # a column-major operand, ld m
            V.fill_(rank + 1)
            parts = [torch.zeros_like(B.t().contiguous()) for _ in range(world)]
            dist.all_gather(parts, B.t().contiguous())
            marks = sum(p.t() for p in parts)
            owner = sum((p.t() > 0).to(torch.int64) for p in parts)
            assert torch.all(owner == 1), (side, m, n)  # every entry written by exactly one rank
            for q in range(world):
                qa, qb = gdist.shard_range(total, q, world, gdist.SHARD_ALIGN)
                blk = gdist.shard_view(side, marks, qa, qb)
                assert torch.all(blk == q + 1)
        gdist.barrier()
        mx = gdist.max_over_ranks(float(rank + 10))
        assert mx == float(world - 1 + 10)
    finally:
        dist.destroy_process_group()


def test_gloo_world2_shard_blocks_cover_once():
    world = 2
    port = _free_port()
    mp.start_processes(_worker, args=(world, port), nprocs=world, join=True, start_method="spawn")

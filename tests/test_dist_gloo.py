"""World-size-2 gloo tests of the multi-process host logic on CPU: shard
ranges tile the right-hand sides exactly, the max-over-ranks reduction, and
that a column-sharded solve (each rank solving its own columns, here with the
CPU oracle as the compute) reassembles to the unsharded solution without any
exchange step."""
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


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, outdir):
    import torch.distributed as dist
    import oracle
    from paper_2305_19917_gb300 import inputs
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, _ = gdist.env_rank_world()
        assert (r, w) == (rank, world)
        m, n = 120, 37
        A, B = inputs.make_problem(0, 0, 0, 0, m, n, seed=3)
        a, b = gdist.shard_range(n, rank, world)
        X = oracle.dtrsm(0, 0, 0, 0, 1.5, A, B[:, a:b])
        np.save(os.path.join(outdir, f"x{rank}.npy"), X)
        gdist.barrier()
        mx = gdist.max_over_ranks(float(rank + 10))
        assert mx == float(world - 1 + 10)
    finally:
        dist.destroy_process_group()


def test_gloo_world2_sharded_solve(tmp_path):
    world = 2
    port = _free_port()
    mp.start_processes(_worker, args=(world, port, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    import oracle
    from paper_2305_19917_gb300 import inputs
    A, B = inputs.make_problem(0, 0, 0, 0, 120, 37, seed=3)
    Xfull = oracle.dtrsm(0, 0, 0, 0, 1.5, A, B)
    parts = [np.load(os.path.join(tmp_path, f"x{r}.npy")) for r in range(world)]
    assert np.array_equal(np.concatenate(parts, axis=1), Xfull)

"""The right-hand-side sharded solve on the GPU: two ranks (gloo process
group, both on cuda:0 -- their kernels are independent, there is no
collective on the data path) each solve their block of one problem with the
library's mixed and plain paths; the blocks, gathered over gloo to rank 0,
match the oracle and the unsharded solve of the same problem."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

pytestmark = pytest.mark.gpu

CASES = [  # side, uplo, trans, diag, m, n, path
    (0, 0, 0, 0, 300, 700, "mixed"),
    (1, 1, 1, 0, 650, 200, "mixed"),
    (0, 1, 0, 1, 257, 300, "plain"),
    (1, 0, 1, 1, 385, 129, "plain"),
]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2305_19917_gb300 import build
    build.build()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, outdir):
    import torch
    import torch.distributed as dist
    from paper_2305_19917_gb300 import api, inputs
    from paper_2305_19917_gb300 import dist as gdist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        for ci, (side, uplo, trans, diag, m, n, path) in enumerate(CASES):
            A, B = inputs.make_problem(side, uplo, trans, diag, m, n, seed=100 + ci)
            Ad = api.to_device_colmajor(A, torch.float64)
            Bd = api.to_device_colmajor(B, torch.float64)
            a, b, st, it, est = gdist.solve_sharded(side, uplo, trans, diag, 1.5, Ad, Bd, path=path)
            torch.cuda.synchronize()
            assert st == 0, (ci, st, it, est)
            # the rest of B is untouched
            rest = np.asarray(Bd.cpu().numpy())
            mask = np.ones_like(rest, dtype=bool)
            if side == 0:
                mask[:, a:b] = False
            else:
                mask[a:b, :] = False
            assert np.array_equal(rest[mask], B[mask]), ci
            # gather every rank's block to rank 0 (host tensors over gloo)
            X = torch.from_numpy(rest)
            parts = [torch.zeros_like(X) for _ in range(world)] if rank == 0 else None
            dist.gather(X, parts, dst=0)
            if rank == 0:
                full = np.array(B)
                for q, p in enumerate(parts):
                    qa, qb = gdist.shard_range(gdist.rhs_count(side, m, n), q, world, gdist.SHARD_ALIGN)
                    if side == 0:
                        full[:, qa:qb] = p.numpy()[:, qa:qb]
                    else:
                        full[qa:qb, :] = p.numpy()[qa:qb, :]
                np.save(os.path.join(outdir, f"x{ci}.npy"), full)
    finally:
        dist.destroy_process_group()


def test_sharded_solve_two_ranks_matches_oracle(tmp_path):
    import torch

    import oracle
    from paper_2305_19917_gb300 import api, inputs
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    for ci, (side, uplo, trans, diag, m, n, path) in enumerate(CASES):
        A, B = inputs.make_problem(side, uplo, trans, diag, m, n, seed=100 + ci)
        X = np.load(os.path.join(tmp_path, f"x{ci}.npy"))
        Xo = oracle.dtrsm(side, uplo, trans, diag, 1.5, A, B)
        tol = 1e-10 if path == "mixed" else 1e-12
        assert np.linalg.norm(X - Xo) <= tol * np.linalg.norm(Xo), ci
        # the unsharded solve of the same problem by the same path
        Ad = api.to_device_colmajor(A, torch.float64)
        Bd = api.to_device_colmajor(B, torch.float64)
        if path == "mixed":
            st, _, _ = api.trsm_mixed(side, uplo, trans, diag, 1.5, Ad, Bd)
            assert st == 0
        else:
            api.trsm(side, uplo, trans, diag, 1.5, Ad, Bd)
        torch.cuda.synchronize()
        Xu = Bd.cpu().numpy()
        assert np.linalg.norm(X - Xu) <= tol * np.linalg.norm(Xo), ci

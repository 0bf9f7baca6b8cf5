"""GPU parity of the batched persistent solve (device work queue, CUDA graph)
against the CPU oracle, instance by instance."""
import numpy as np
import pytest

import oracle
from paper_2305_19917_gb300 import inputs
from tests.helpers import fwd_err

pytestmark = pytest.mark.gpu
TOL = {0: 1e-12, 1: 1e-4}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2305_19917_gb300 import build
    build.build()


def _device_batch(items, dtype):
    import torch
    from paper_2305_19917_gb300 import api
    tdt = torch.float64 if dtype == 0 else torch.float32
    keep = []
    descs = []
    for it in items:
        Ad = api.to_device_colmajor(it["A"], tdt)
        Bd = api.to_device_colmajor(it["B"], tdt) if it["B"].size else torch.zeros(0, device="cuda", dtype=tdt)
        keep.append((Ad, Bd))
        m, n = it["B"].shape
        k = m if it["side"] == 0 else n
        descs.append(dict(side=it["side"], uplo=it["uplo"], trans=it["trans"], diag=it["diag"], m=m, n=n,
                          alpha=it["alpha"], A_ptr=Ad.data_ptr(), lda=max(1, k), B_ptr=Bd.data_ptr(),
                          ldb=max(1, m)))
    return keep, descs


def _random_items(count, seed, kmax=300, nmax=70, big=()):
    rng = np.random.default_rng(seed)
    items = []
    for i in range(count):
        side, uplo, trans, diag = (int(x) for x in rng.integers(0, 2, 4))
        m = int(rng.integers(1, kmax)) if i not in big else 600
        n = int(rng.integers(1, nmax))
        A, B = inputs.make_problem(side, uplo, trans, diag, m, n, seed=1000 * seed + i)
        items.append(dict(side=side, uplo=uplo, trans=trans, diag=diag, alpha=float(rng.choice([1.0, -0.5, 2.0])),
                          A=A, B=B))
    return items


@pytest.mark.parametrize("dtype", [0, 1])
def test_batched_mixed_forms_and_sizes(dtype):
    import torch
    from paper_2305_19917_gb300 import api
    items = _random_items(60, seed=1 + dtype, big=(3, 40))
    items.append(dict(side=0, uplo=0, trans=0, diag=0, alpha=1.0, A=np.eye(5), B=np.zeros((5, 0))))
    keep, descs = _device_batch(items, dtype)
    st = api.gb_trsm_batched(dtype, descs, torch.cuda.current_stream().cuda_stream)
    assert st == 0, api.gb_status_string(st)
    for it, (Ad, Bd) in zip(items, keep):
        if it["B"].size == 0:
            continue
        X = Bd.double().cpu().numpy()
        Xo = oracle.dtrsm(it["side"], it["uplo"], it["trans"], it["diag"], it["alpha"], it["A"], it["B"])
        assert fwd_err(X, Xo) <= TOL[dtype], (it["side"], it["uplo"], it["trans"], it["diag"], it["B"].shape)


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("tile", [1, 2])
def test_batched_tiles_mixed_forms(dtype, tile):
    """Both tile shapes of the batched kernel (units of 8 PER tile right-hand
    sides) on the mixed forms, ragged sizes and two large instances."""
    import torch
    from paper_2305_19917_gb300 import api
    items = _random_items(40, seed=11 + dtype + 2 * tile, nmax=150, big=(5,))
    keep, descs = _device_batch(items, dtype)
    plan = api.BatchedPlan(dtype, descs, tile=tile)
    assert plan.tile == tile
    plan.run(torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    plan.close()
    for it, (Ad, Bd) in zip(items, keep):
        X = Bd.double().cpu().numpy()
        Xo = oracle.dtrsm(it["side"], it["uplo"], it["trans"], it["diag"], it["alpha"], it["A"], it["B"])
        assert fwd_err(X, Xo) <= TOL[dtype], (tile, it["side"], it["uplo"], it["trans"], it["diag"], it["B"].shape)


@pytest.mark.parametrize("dtype", [0, 1])
def test_batched_autotune_restores_b_and_picks_a_tile(dtype):
    import torch
    from paper_2305_19917_gb300 import api
    items = inputs.make_batch(300, seed=13)
    keep, descs = _device_batch(items, dtype)
    before = [Bd.clone() for _, Bd in keep]
    tile, ms = api.gb_batched_autotune(dtype, descs, reps=2, stream=torch.cuda.current_stream().cuda_stream)
    assert tile in (1, 2) and all(t > 0 for t in ms)
    assert ms[tile - 1] == min(ms)
    for (_, Bd), B0 in zip(keep, before):
        assert torch.equal(Bd, B0)


@pytest.mark.parametrize("dtype", [0, 1])
def test_batched_plan_replay_and_config_recipe(dtype):
    """The 4096-instance uneven recipe (m log-uniform in [16, 512], n in
    [1, 256], side/uplo uniform); sampled instances vs the oracle after two
    replays of the same plan (inputs reset in between)."""
    import torch
    from paper_2305_19917_gb300 import api
    items = inputs.make_batch(4096, seed=7)
    keep, descs = _device_batch(items, dtype)
    originals = [Bd.clone() for _, Bd in keep]
    tile, _ = api.gb_batched_autotune(dtype, descs, reps=2, stream=torch.cuda.current_stream().cuda_stream)
    plan = api.BatchedPlan(dtype, descs, tile=tile)
    info = plan.info()
    assert info["large_instances"] == 0 and info["units"] >= 4096
    for _ in range(2):
        for (_, Bd), B0 in zip(keep, originals):
            Bd.copy_(B0)
        plan.run(torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
    plan.close()
    for idx in range(0, 4096, 97):
        it = items[idx]
        X = keep[idx][1].double().cpu().numpy()
        Xo = oracle.dtrsm(it["side"], it["uplo"], it["trans"], it["diag"], it["alpha"], it["A"], it["B"])
        assert fwd_err(X, Xo) <= TOL[dtype], idx

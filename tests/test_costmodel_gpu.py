"""The learned cost model: trained on the GPU by the library's own kernels
from the committed autotuner timings (420 shapes x 48 plans, m and n
log-uniform in [64, 32768]), judged on held-out shapes (80/20 split on
shapes) by its regret t(chosen) / t(best) - 1 against exhaustive search; and
what it gains over the method without it -- the Section V-style analytic
model (fitted rates) and a fixed nb = 128 plan."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2305_19917_gb300 import build
    build.build()


def test_regret_on_held_out_shapes():
    from paper_2305_19917_gb300 import costmodel
    rows = costmodel.load_db(costmodel.DEFAULT_DB)
    assert len(rows) >= 20000
    tr, te = costmodel.split_shapes(rows, 0.8, seed=0)
    _, stats = costmodel.evaluate(tr, te, epochs=200)
    assert stats["mlp"]["mean"] <= 0.10, stats
    assert stats["mlp"]["mean"] < stats["analytic"]["mean"], stats
    assert stats["mlp"]["mean"] < stats["fixed_nb128"]["mean"], stats


def test_committed_model_drives_the_planner():
    import torch
    import oracle
    from paper_2305_19917_gb300 import api, costmodel, inputs
    assert api.gb_plan_set_model(costmodel.DEFAULT_MODEL) == 0
    try:
        st, plan, ms = api.gb_plan_choose(0, 0, 0, 0, 2048, 512)
        assert st == 0 and ms > 0
        assert plan in api.gb_plan_candidates(0)
        # the planner's choice is used by gb_dtrsm and gives the right answer
        A, B = inputs.make_problem(1, 1, 0, 0, 300, 700, seed=3)
        Ad = api.to_device_colmajor(A, torch.float64)
        Bd = api.to_device_colmajor(B, torch.float64)
        api.trsm(1, 1, 0, 0, 1.5, Ad, Bd)
        torch.cuda.synchronize()
        Xo = oracle.dtrsm(1, 1, 0, 0, 1.5, A, B)
        assert np.linalg.norm(Bd.cpu().numpy() - Xo) <= 1e-12 * np.linalg.norm(Xo)
    finally:
        api.gb_plan_set_model(None)
    st, plan, _ = api.gb_plan_choose(0, 0, 0, 0, 2048, 512)
    assert st == api.STATUS_NO_MODEL


def test_autotune_picks_the_fastest_measured_plan():
    import torch
    from paper_2305_19917_gb300 import api, autotune
    s = dict(dtype=0, side=0, uplo=0, trans=0, m=1024, n=256)
    A, B = autotune.make_inputs(s, 1)
    B0 = B.clone()
    best, best_ms = api.gb_autotune(0, 0, 0, 0, 0, 1024, 256, 1.0, A.data_ptr(), 1024, B.data_ptr(), 1024,
                                    torch.cuda.current_stream().cuda_stream)
    assert best in api.gb_plan_candidates(0) and best_ms > 0
    assert torch.equal(B, B0)  # B restored

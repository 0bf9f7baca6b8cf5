"""The learned cost model: trained on the GPU by the library's own kernels
from the committed autotuner timings (420 shapes x 48 plans, m and n
log-uniform in [64, 32768]; plus 150 FP64 shapes timed in plain FP64 and in
five mixed-precision configurations), evaluated on held-out shapes (80/20
split on shapes) by its regret t(chosen) / t(best) - 1 against exhaustive
search; and what it gains over the method without it -- the paper's
analytic models (Section V) with measured task times, a fitted-rates
variant and a fixed nb = 128 plan -- and, for the precision decision, over
always-plain-FP64 and always-BF16."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2305_19917_gb300 import build
    build.build()


def test_regret_on_held_out_shapes():
    """Held-out regret of the network against exhaustive search, and against
    the paper's analytic models (Section V Comp(i) of the recursive,
    iterative and blocked models with task times measured on the GPU: the
    argmin over the plans they describe, and the recursive model with the
    stop rule 2 TS(i+1) < TS(i)), a fitted-rates variant and a fixed plan."""
    from paper_2305_19917_gb300 import costmodel
    rows = costmodel.load_db(costmodel.DEFAULT_DB)
    assert len(rows) >= 20000
    comps = costmodel.load_components(costmodel.DEFAULT_COMP_DB)
    assert len(comps) >= 400
    tr, te = costmodel.split_shapes(rows, 0.8, seed=0)
    _, stats = costmodel.evaluate(tr, te, epochs=800, components=comps)
    assert stats["covered_shapes"] == stats["shapes"], stats
    assert stats["mlp"]["mean"] <= 0.06, stats
    assert stats["mlp"]["mean"] < stats["paper_comp_argmin"]["mean"], stats
    assert stats["mlp"]["mean"] < stats["paper_stop_rule"]["mean"], stats
    assert stats["mlp"]["mean"] < stats["analytic"]["mean"], stats
    assert stats["mlp"]["mean"] < stats["fixed_nb128"]["mean"], stats


def test_precision_choice_regret():
    """The planner chooses the precision for a request of FP64-level
    accuracy (plain FP64, or mixed BF16 / FP8 with a leaf order): held-out
    regret against exhaustive search over those candidates, where a mixed
    run that missed the accuracy would be charged the plain fallback; it
    must stay within 10 % and beat always-plain and always-BF16-1024."""
    from paper_2305_19917_gb300 import costmodel
    rows = costmodel.load_db(costmodel.DEFAULT_DB)
    prec = costmodel.load_db(costmodel.DEFAULT_PREC_DB)
    assert len(prec) >= 6 * 100
    _, st = costmodel.evaluate_precision(rows, prec)
    assert st["mlp"]["mean"] <= 0.03, st
    assert st["mlp"]["mean"] < st["always_plain_fp64"]["mean"], st
    assert st["mlp"]["mean"] <= st["always_bf16_1024"]["mean"] + 0.005, st


def test_committed_model_chooses_precision():
    """The C planner's precision decision with the committed network agrees
    with the network's own predictions, and the chosen configuration solves
    to the mixed path's accuracy."""
    import torch
    import oracle
    from paper_2305_19917_gb300 import api, costmodel, inputs
    assert api.gb_plan_set_model(costmodel.DEFAULT_MODEL) == 0
    try:
        model = costmodel.MLP.load(costmodel.DEFAULT_MODEL)
        for side, uplo, trans, m, n in ((0, 0, 0, 16384, 16384), (1, 1, 0, 3000, 2048), (0, 1, 1, 2048, 512)):
            st, prec, leaf, plan, ms = api.gb_plan_choose_precision(side, uplo, trans, m, n)
            assert st == 0 and ms > 0
            k = m if side == 0 else n
            cands = [dict(dtype=costmodel.PREC_DTYPE[p], side=side, uplo=uplo, trans=trans, m=m, n=n, **pl)
                     for p, lf, pl in api.gb_plan_mixed_candidates(k)]
            st0, plain, _ = api.gb_plan_choose(0, side, uplo, trans, m, n)
            cands.append(dict(dtype=0, side=side, uplo=uplo, trans=trans, m=m, n=n, **plain))
            pred = model.predict_log_ms(costmodel.features(cands))
            best = cands[int(np.argmin(pred))]
            if prec < 0:
                assert best["dtype"] == 0
            else:
                assert best["dtype"] == costmodel.PREC_DTYPE[prec] and best["nb"] == leaf
        # run the choice for one shape and check it against the oracle
        side, uplo, trans, m, n = 0, 1, 1, 2048, 512
        st, prec, leaf, plan, ms = api.gb_plan_choose_precision(side, uplo, trans, m, n)
        A, B = inputs.make_problem(side, uplo, trans, 0, m, n, seed=5)
        Ad = api.to_device_colmajor(A, torch.float64)
        Bd = api.to_device_colmajor(B, torch.float64)
        if prec < 0:
            api.trsm(side, uplo, trans, 0, 1.5, Ad, Bd)
        else:
            r = api.gb_dtrsm_mixed_leaf(side, uplo, trans, 0, m, n, 1.5, Ad.data_ptr(), m, Bd.data_ptr(), m, 1e-11,
                                        prec, 30, leaf, torch.cuda.current_stream().cuda_stream)
            assert r[0] == 0, r
        torch.cuda.synchronize()
        Xo = oracle.dtrsm(side, uplo, trans, 0, 1.5, A, B)
        assert np.linalg.norm(Bd.cpu().numpy() - Xo) <= 1e-10 * np.linalg.norm(Xo)
    finally:
        api.gb_plan_set_model(None)
    st, prec, leaf, plan, ms = api.gb_plan_choose_precision(0, 0, 0, 4096, 4096)
    assert st == api.STATUS_NO_MODEL and prec == -1


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

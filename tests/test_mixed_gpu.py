"""GPU parity of the mixed-precision solve (BF16 tensor-core updates + split
residual refinement) against the FP64 CPU oracle: forward error <= 1e-10."""
import itertools

import numpy as np
import pytest

import oracle
from paper_2305_19917_gb300 import inputs
from tests.helpers import fwd_err

pytestmark = pytest.mark.gpu

COMBOS = list(itertools.product((0, 1), (0, 1), (0, 1), (0, 1)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2305_19917_gb300 import build
    build.build()


def _mixed(side, uplo, trans, diag, alpha, A, B, tol=1e-11, max_iter=30):
    import torch
    from paper_2305_19917_gb300 import api
    Ad = api.to_device_colmajor(A, torch.float64)
    Bd = api.to_device_colmajor(B, torch.float64)
    st, it, est = api.trsm_mixed(side, uplo, trans, diag, alpha, Ad, Bd, tol=tol, max_iter=max_iter)
    torch.cuda.synchronize()
    return Bd.cpu().numpy(), st, it, est


@pytest.mark.parametrize("side,uplo,trans,diag", COMBOS)
def test_mixed_all_forms(side, uplo, trans, diag):
    m, n = 300, 170
    A, B = inputs.make_problem(side, uplo, trans, diag, m, n, seed=11)
    Xo = oracle.dtrsm(side, uplo, trans, diag, 1.5, A, B)
    X, st, it, est = _mixed(side, uplo, trans, diag, 1.5, A, B)
    assert st == 0 and 1 <= it <= 10, (st, it, est)
    assert fwd_err(X, Xo) <= 1e-10


@pytest.mark.parametrize("side,uplo,trans,diag,m,n,ldpad", [
    (0, 0, 0, 0, 300, 170, 3), (0, 1, 0, 0, 257, 130, 1), (0, 0, 1, 1, 384, 64, 5), (1, 1, 1, 0, 140, 333, 3)])
def test_mixed_padded_leading_dimensions(side, uplo, trans, diag, m, n, ldpad):
    """B inside a buffer with ldb = m + ldpad (odd paddings, so the columns
    change their 16-byte alignment one to the next) and A with lda = k + 2:
    the solution matches the oracle and nothing outside the m x n matrix
    (canaries in the padding rows) is written."""
    import torch
    from paper_2305_19917_gb300 import api
    A, B = inputs.make_problem(side, uplo, trans, diag, m, n, seed=31 + m)
    Xo = oracle.dtrsm(side, uplo, trans, diag, 1.5, A, B)
    k = A.shape[0]
    abuf = torch.full((k, k + 2), 7.0, dtype=torch.float64, device="cuda").t()
    Ad = abuf[:k, :k]
    Ad.copy_(torch.as_tensor(A))
    canary = 1234.5
    bbuf = torch.full((n, m + ldpad), canary, dtype=torch.float64, device="cuda").t()
    Bd = bbuf[:m, :n]
    Bd.copy_(torch.as_tensor(B))
    st, it, est = api.trsm_mixed(side, uplo, trans, diag, 1.5, Ad, Bd, tol=1e-11)
    torch.cuda.synchronize()
    assert st == 0, (st, it, est)
    assert fwd_err(Bd.cpu().numpy(), Xo) <= 1e-10
    assert bool(torch.all(bbuf[m:, :n] == canary).item())


@pytest.mark.parametrize("m,n", [(1, 1), (2, 300), (129, 7), (512, 512), (700, 129)])
def test_mixed_ragged_sizes(m, n):
    A, B = inputs.make_problem(0, 0, 0, 0, m, n, seed=m + n)
    Xo = oracle.dtrsm(0, 0, 0, 0, 1.0, A, B)
    X, st, it, est = _mixed(0, 0, 0, 0, 1.0, A, B)
    assert st == 0
    assert fwd_err(X, Xo) <= 1e-10


def test_mixed_unreferenced_nan_not_read():
    A, B = inputs.make_problem(0, 1, 1, 1, 256, 64, seed=4, poison=True)
    Ac, _ = inputs.make_problem(0, 1, 1, 1, 256, 64, seed=4)
    Xo = oracle.dtrsm(0, 1, 1, 1, 1.5, Ac, B)
    X, st, it, est = _mixed(0, 1, 1, 1, 1.5, A, B)
    assert st == 0 and np.all(np.isfinite(X))
    assert fwd_err(X, Xo) <= 1e-10


def test_mixed_reports_non_convergence():
    A, B = inputs.make_problem(0, 0, 0, 0, 256, 64, seed=2)
    X, st, it, est = _mixed(0, 0, 0, 0, 1.0, A, B, tol=1e-30, max_iter=1)
    from paper_2305_19917_gb300 import api
    assert st == api.STATUS_NOT_CONVERGED and it == 1 and est > 0


def test_mixed_alpha_zero():
    A = np.full((40, 40), np.nan)
    B = np.ones((40, 10))
    X, st, it, est = _mixed(0, 0, 0, 0, 0.0, A, B)
    assert st == 0 and np.array_equal(X, np.zeros_like(B))


@pytest.mark.parametrize("m,n", [(16384, 16384), (32768, 4096)])
def test_mixed_config_scale_sampled(m, n):
    """Mixed-precision configuration sizes: sampled right-hand sides vs the
    oracle, and the accuracy of the BF16 low-precision solve itself.  The
    refinement hides an inaccurate low solve (it converges anyway, in more
    steps), so the first correction's size relative to X (the contraction of
    the iteration) is bounded directly: on this diagonally dominant recipe the
    BF16 solve (BF16 operands, split-precision diagonal solves) reaches
    rho_1 < 1e-4 (about 6.7e-5 at 16384^2), and two steps reach 1e-11."""
    import torch
    from paper_2305_19917_gb300 import api
    A, B = inputs.make_problem(0, 0, 0, 0, m, n, seed=0)
    Ad = api.to_device_colmajor(A, torch.float64)
    Bd = api.to_device_colmajor(B, torch.float64)
    st, it, est = api.trsm_mixed(0, 0, 0, 0, 1.5, Ad, Bd, tol=1e-11)
    hist = api.gb_mixed_history()
    assert st == 0, (st, it, est)
    assert it == 2 and hist[0][0] < 1e-4, (it, hist)
    cols = [0, 7, n // 2, n - 1]
    X = Bd[:, cols].cpu().numpy()
    Xo = oracle.dtrsm(0, 0, 0, 0, 1.5, A, B[:, cols])
    assert fwd_err(X, Xo) <= 1e-10


@pytest.mark.parametrize("side,uplo,trans,diag,prec", [(1, 1, 1, 0, 0), (0, 1, 1, 1, 0), (1, 0, 0, 0, 1)])
def test_mixed_other_forms_config_scale_sampled(side, uplo, trans, diag, prec):
    """Mixed solves in other forms at 16384^2 (a Right-side form transposes
    B into the canonical view, an Upper form reverses the indices): sampled
    rows (side Right: each row of X depends only on its row of B) or columns,
    the last ones included, vs the oracle within 1e-10."""
    import torch
    from paper_2305_19917_gb300 import api
    m = n = 16384
    A, B = inputs.make_problem_device(side, uplo, trans, diag, m, n, seed=70 + side + 2 * uplo)
    idx = [0, 1, m // 2, m - 2, m - 1]
    Bs = (B[idx, :] if side == 1 else B[:, idx]).cpu().numpy()
    st, it, est = api.trsm_mixed(side, uplo, trans, diag, 1.5, A, B, tol=1e-11, prec=prec, max_iter=60)
    torch.cuda.synchronize()
    assert st == 0 and 1 <= it <= 12, (st, it, est, api.gb_mixed_history())
    Xs = (B[idx, :] if side == 1 else B[:, idx]).cpu().numpy()
    Xo = oracle.dtrsm(side, uplo, trans, diag, 1.5, A.cpu().numpy(), Bs)
    assert fwd_err(Xs, Xo) <= 1e-10


@pytest.mark.parametrize("m,n", [(16384, 16384), (32768, 4096)])
def test_mixed_fp8_config_scale_sampled(m, n):
    """FP8 E4M3 updates (per-128x128-block power-of-two scales) at the
    mixed-precision configuration sizes: sampled right-hand sides vs the
    oracle within 1e-10; the refinement step count is bounded and reported."""
    import torch
    from paper_2305_19917_gb300 import api
    A, B = inputs.make_problem_device(0, 0, 0, 0, m, n, seed=7)
    cols = [0, 5, n // 2, n - 1]
    Bs = B[:, cols].cpu().numpy()
    st, it, est = api.trsm_mixed(0, 0, 0, 0, 1.5, A, B, tol=1e-11, prec=api.PREC_FP8, max_iter=60)
    torch.cuda.synchronize()
    hist = api.gb_mixed_history()
    assert st == 0 and 1 <= it <= 12, (st, it, est, hist)
    Xo = oracle.dtrsm(0, 0, 0, 0, 1.5, A.cpu().numpy(), Bs)
    assert fwd_err(B[:, cols].cpu().numpy(), Xo) <= 1e-10, (it, hist)


@pytest.mark.parametrize("side,uplo,trans,diag", [(0, 0, 0, 0), (1, 1, 1, 0), (0, 1, 0, 1), (1, 0, 1, 1)])
def test_mixed_fp8_block_scaled_updates(side, uplo, trans, diag):
    """FP8 E4M3 GEMM updates with per-block power-of-two scales: the
    refinement still reaches the FP64-level tolerance (more steps than BF16)."""
    import torch
    from paper_2305_19917_gb300 import api
    m, n = 600, 300
    A, B = inputs.make_problem(side, uplo, trans, diag, m, n, seed=21)
    Xo = oracle.dtrsm(side, uplo, trans, diag, 1.5, A, B)
    Ad = api.to_device_colmajor(A, torch.float64)
    Bd = api.to_device_colmajor(B, torch.float64)
    st, it, est = api.trsm_mixed(side, uplo, trans, diag, 1.5, Ad, Bd, tol=1e-11, prec=api.PREC_FP8, max_iter=60)
    torch.cuda.synchronize()
    assert st == 0 and it <= 40, (st, it, est, api.gb_mixed_history())
    assert fwd_err(Bd.cpu().numpy(), Xo) <= 1e-10


@pytest.mark.parametrize("max_iter", [3, 5])
def test_long_refinement_folds_kept_corrections(max_iter):
    """tol = 0 runs max_iter refinement steps: beyond the corrections kept as
    digit slices the library folds them into X; the solution stays right."""
    import torch
    from paper_2305_19917_gb300 import api
    side, uplo, trans, diag, m, n, alpha = 0, 1, 1, 0, 300, 77, -1.25
    A, B = inputs.make_problem(side, uplo, trans, diag, m, n, seed=21)
    Ad = api.to_device_colmajor(A, torch.float64)
    Bd = api.to_device_colmajor(B, torch.float64)
    st, it, est = api.trsm_mixed(side, uplo, trans, diag, alpha, Ad, Bd, tol=0.0, max_iter=max_iter)
    torch.cuda.synchronize()
    assert it == max_iter and st in (0, api.STATUS_NOT_CONVERGED)
    Xo = oracle.dtrsm(side, uplo, trans, diag, alpha, A, B)
    X = Bd.cpu().numpy()
    assert np.linalg.norm(X - Xo) <= 1e-10 * np.linalg.norm(Xo)


def test_out_of_fp32_range_is_reported_not_silent():
    """The low-precision solve works in FP32/BF16 on power-of-two scaled
    right-hand sides: a solution that grows beyond the FP32 range relative to
    its right-hand side (here X(i) ~ 3^i from a unit triangle with -2 below
    the diagonal), or non-finite data, cannot be refined, and the call says so
    with GB_STATUS_RANGE and leaves B as it was, instead of returning a wrong X
    as if it had converged."""
    import torch
    from paper_2305_19917_gb300 import api
    m, n = 256, 16
    A, B = inputs.make_problem(0, 0, 0, 0, m, n, seed=31)
    G = np.tril(np.full((m, m), -2.0), -1) + np.eye(m)   # X(i) = 3^i B(0) for B = e_0
    cases = [(A, np.where(np.arange(n) == 5, np.nan, B)), (G, B)]
    for Am, bad in cases:
        Ad = api.to_device_colmajor(Am, torch.float64)
        Bd = api.to_device_colmajor(bad, torch.float64)
        st, it, est = api.gb_dtrsm_mixed(0, 0, 0, 0, m, n, 1.0, Ad.data_ptr(), m, Bd.data_ptr(), m, 1e-11,
                                         api.PREC_BF16, 4, torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert st == api.STATUS_RANGE
        np.testing.assert_array_equal(Bd.cpu().numpy(), bad)
    assert "range" in api.gb_status_string(api.STATUS_RANGE)


@pytest.mark.parametrize("scale", [1e-300, 1e-310, 1e-40, 1e30, 1e300])
@pytest.mark.parametrize("side", [0, 1])
def test_scale_of_b_does_not_matter(scale, side):
    """Right-hand sides far outside the FP32 range (down to FP64 subnormals,
    up to 1e300) and alpha far from 1 are solved to full accuracy: every
    column is scaled by a power of two for the low-precision solve and scaled
    back exactly.  Columns of different scales are independent."""
    import torch
    from paper_2305_19917_gb300 import api
    m, n = (200, 12) if side == 0 else (12, 200)
    A, B = inputs.make_problem(side, 0, 0, 0, m, n, seed=32)
    # per right-hand side: the given scale, 1, and a mix (columns for left, rows for right)
    w = np.array([scale, 1.0, scale * 1e6 if scale < 1 else scale * 1e-6] * 4)
    Bs = B * w[None, :] if side == 0 else B * w[:, None]
    alpha = 2.0 ** -300 if scale > 1 else 1.0
    Xo = oracle.dtrsm(side, 0, 0, 0, alpha, A, Bs)
    Ad = api.to_device_colmajor(A, torch.float64)
    Bd = api.to_device_colmajor(Bs, torch.float64)
    st, it, est = api.trsm_mixed(side, 0, 0, 0, alpha, Ad, Bd)
    torch.cuda.synchronize()
    X = Bd.cpu().numpy()
    assert st == 0, (st, it, est)
    Xc, Oc = (X, Xo) if side == 0 else (X.T, Xo.T)
    for j in range(Xc.shape[1]):
        # norms of columns rescaled by their largest entry: a plain 2-norm of
        # entries near 1e209 overflows to inf and the comparison would hold
        # for any result
        s = np.abs(Oc[:, j]).max()
        assert np.isfinite(s) and s > 0 and np.all(np.isfinite(Xc[:, j])), (j, w[j])
        assert np.linalg.norm((Xc[:, j] - Oc[:, j]) / s) <= 1e-10 * np.linalg.norm(Oc[:, j] / s), (j, w[j])


def test_concurrent_solves_from_two_host_threads():
    """Two host threads solving different problems on their own streams at
    the same time (the binding releases the interpreter lock during a call):
    the cached low-precision graphs are shared per device, and both results
    still match the oracle."""
    import threading
    import torch
    from paper_2305_19917_gb300 import api
    probs = [(0, 0, 0, 0, 300, 170, 1.5, 41), (1, 1, 1, 0, 96, 257, -0.5, 42)]
    errs, fails = {}, []

    def run(idx):
        try:
            side, uplo, trans, diag, m, n, alpha, seed = probs[idx]
            A, B = inputs.make_problem(side, uplo, trans, diag, m, n, seed=seed)
            Xo = oracle.dtrsm(side, uplo, trans, diag, alpha, A, B)
            s = torch.cuda.Stream()
            worst = 0.0
            for _ in range(4):
                with torch.cuda.stream(s):
                    Ad = api.to_device_colmajor(A, torch.float64)
                    Bd = api.to_device_colmajor(B, torch.float64)
                s.synchronize()
                st, it, est = api.trsm_mixed(side, uplo, trans, diag, alpha, Ad, Bd, stream=s)
                s.synchronize()
                assert st == 0, st
                worst = max(worst, fwd_err(Bd.cpu().numpy(), Xo))
            errs[idx] = worst
        except Exception as e:  # reported below, in the main thread
            fails.append(repr(e))

    ts = [threading.Thread(target=run, args=(i,)) for i in range(2)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert not fails, fails
    assert errs[0] <= 1e-10 and errs[1] <= 1e-10, errs

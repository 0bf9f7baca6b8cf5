"""GPU parity of the Cholesky factorisation (gb_dpotrf / gb_spotrf: the
recursive model of Section V-A on this library's triangular solve, the use
Section VIII names) against the CPU oracle (oracle/potrf_oracle.c).

Acceptance: FP64 factor within 1e-12 (normwise relative) of the oracle's and
backward error ||A - L L^T||_F / ||A||_F <= 10 n 2^-53; FP32 within 1e-4 and
10 n 2^-24.  Both triangles' forms, ragged orders around the 64-column
leaves, the other triangle untouched, padded leading dimensions, the info
convention for matrices that are not positive definite, and n = 8192 / 16384
checked on sampled columns of L L^T."""
import numpy as np
import pytest

import oracle
from paper_2305_19917_gb300 import inputs

pytestmark = pytest.mark.gpu

U64, U32 = 2.0 ** -53, 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2305_19917_gb300 import build
    build.build()


def _tri(F, uplo):
    return np.tril(F) if uplo == 0 else np.triu(F)


def _gpu_potrf(uplo, A, dtype="f64", ldpad=0, canary=777.0):
    import torch
    from paper_2305_19917_gb300 import api
    tdt = torch.float64 if dtype == "f64" else torch.float32
    n = A.shape[0]
    buf = torch.full((max(n, 1), n + ldpad), canary, dtype=tdt, device="cuda").t()
    Ad = buf[:n, :n]
    Ad.copy_(torch.as_tensor(A).to(tdt))
    info = api.potrf(uplo, Ad)
    torch.cuda.synchronize()
    pad_ok = bool(torch.all(buf[n:, :n] == canary).item()) if ldpad else True
    return Ad.double().cpu().numpy(), info, pad_ok


@pytest.mark.parametrize("uplo", [0, 1])
@pytest.mark.parametrize("n", [1, 2, 31, 63, 64, 65, 127, 128, 129, 300, 1000])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_potrf_matches_oracle(uplo, n, dtype):
    A = inputs.make_spd(n, seed=n + 7 * uplo)
    Fo, info_o = oracle.dpotrf(uplo, A)
    assert info_o == 0
    F, info, _ = _gpu_potrf(uplo, A, dtype)
    assert info == 0
    T, To = _tri(F, uplo), _tri(Fo, uplo)
    tol, u = (1e-12, U64) if dtype == "f64" else (1e-4, U32)
    assert np.linalg.norm(T - To) <= tol * np.linalg.norm(To)
    L = T if uplo == 0 else T.T
    assert np.linalg.norm(A - L @ L.T) <= 10 * n * u * np.linalg.norm(A)


@pytest.mark.parametrize("uplo", [0, 1])
def test_other_triangle_untouched_and_padding(uplo):
    n = 200
    A = inputs.make_spd(n, seed=3)
    P = A.copy(order="F")
    other = np.triu_indices(n, 1) if uplo == 0 else np.tril_indices(n, -1)
    P[other] = np.nan
    F, info, pad_ok = _gpu_potrf(uplo, P, "f64", ldpad=5)
    assert info == 0 and pad_ok
    assert np.all(np.isnan(F[other]))
    Fo, _ = oracle.dpotrf(uplo, A)
    assert np.linalg.norm(_tri(F, uplo) - _tri(Fo, uplo)) <= 1e-12 * np.linalg.norm(_tri(Fo, uplo))


@pytest.mark.parametrize("uplo", [0, 1])
@pytest.mark.parametrize("bad", [0, 5, 64, 100, 257])
def test_info_first_non_positive_pivot(uplo, bad):
    n = 300
    A = inputs.make_spd(n, seed=9)
    A[bad, bad] = -1.0
    _, info_o = oracle.dpotrf(uplo, A)
    _, info, _ = _gpu_potrf(uplo, A)
    assert info == info_o == bad + 1


def test_zero_order_and_arguments():
    import torch
    from paper_2305_19917_gb300 import api
    assert api.gb_dpotrf(0, 0, 0, 1) == (0, 0)
    A = torch.zeros((4, 4), dtype=torch.float64, device="cuda")
    assert api.gb_dpotrf(2, 4, A.data_ptr(), 4)[0] == -1
    assert api.gb_dpotrf(0, -1, A.data_ptr(), 4)[0] == -2
    assert api.gb_dpotrf(0, 4, 0, 4)[0] == -3
    assert api.gb_dpotrf(0, 4, A.data_ptr(), 3)[0] == -4


@pytest.mark.parametrize("uplo,n", [(0, 16384), (1, 8192)])
def test_potrf_config_scale_sampled(uplo, n):
    """n = 16384 (lower) and 8192 (upper), FP64: sampled columns of L L^T
    against A (each column j of L L^T is L times row j of L)."""
    import torch
    from paper_2305_19917_gb300 import api
    A = inputs.make_spd_device(n, seed=11 + uplo)
    cols = [0, 1, n // 3, n // 2 + 5, n - 2, n - 1]
    Acols = A[:, cols].cpu().numpy()
    info = api.potrf(uplo, A)
    torch.cuda.synchronize()
    assert info == 0
    F = A.cpu().numpy()
    L = np.tril(F) if uplo == 0 else np.triu(F).T
    R = L @ L[cols, :].T
    anorm = np.linalg.norm(Acols)
    assert np.linalg.norm(R - Acols) <= 10 * n * U64 * anorm

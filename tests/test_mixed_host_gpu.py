"""gb_dtrsm_mixed_host (operands in host memory) against the FP64 oracle and
against the device entry point, on the GPU."""
import numpy as np
import pytest

import oracle
from paper_2305_19917_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2305_19917_gb300 import build
    build.build()


def _host(a, pinned):
    import torch
    t = torch.from_numpy(np.array(a.T, order="C", copy=True)).t()  # column-major copy (never aliases a)
    return t.pin_memory() if pinned else t


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("side,uplo,trans,diag,m,n,alpha", [
    (0, 0, 0, 0, 300, 170, 1.5), (0, 1, 1, 0, 257, 64, -0.5), (1, 0, 0, 1, 96, 300, 2.0),
    (1, 1, 1, 0, 130, 130, 1.0), (0, 0, 1, 1, 1, 5, 1.0)])
def test_host_entry_matches_oracle_and_device_entry(pinned, side, uplo, trans, diag, m, n, alpha):
    import torch
    from paper_2305_19917_gb300 import api
    A, B = inputs.make_problem(side, uplo, trans, diag, m, n, seed=5, poison=True)
    Xo = oracle.dtrsm(side, uplo, trans, diag, alpha, A, B)
    Ah, Bh = _host(A, pinned), _host(B, pinned)
    if pinned:
        assert Bh.stride(0) == 1
    st, it, est = api.trsm_mixed_host(side, uplo, trans, diag, alpha, Ah, Bh)
    X = Bh.numpy()
    assert st == 0 and it >= 1
    assert np.isfinite(X).all()  # the NaN-poisoned unreferenced triangle was never read
    assert np.linalg.norm(X - Xo) <= TOL * np.linalg.norm(Xo)
    Ad = api.to_device_colmajor(A, torch.float64)
    Bd = api.to_device_colmajor(B, torch.float64)
    api.trsm_mixed(side, uplo, trans, diag, alpha, Ad, Bd)
    torch.cuda.synchronize()
    assert np.linalg.norm(X - Bd.cpu().numpy()) <= TOL * np.linalg.norm(Xo)


def test_host_entry_rejects_device_tensors():
    import torch
    from paper_2305_19917_gb300 import api
    A = torch.zeros((4, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        api.trsm_mixed_host(0, 0, 0, 0, 1.0, A, A)

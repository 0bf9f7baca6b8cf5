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


@pytest.mark.parametrize("blocks", [2, 3])
@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("side,uplo,trans,diag,m,n,alpha", [
    (0, 0, 0, 0, 300, 330, 1.5), (0, 1, 1, 1, 200, 260, -0.5), (1, 0, 1, 0, 390, 180, 2.0),
    (1, 1, 0, 0, 257, 140, 1.0)])
def test_pipelined_column_blocks_match_oracle(monkeypatch, blocks, pinned, side, uplo, trans, diag, m, n, alpha):
    """The host solve in 2 or 3 column blocks (ragged last block; columns of B
    for side = left, rows for right) gives the oracle's solution in every
    block, and the per-solve report covers all of them."""
    from paper_2305_19917_gb300 import api
    monkeypatch.setenv("GB_MIXED_HOST_BLOCKS", str(blocks))
    A, B = inputs.make_problem(side, uplo, trans, diag, m, n, seed=11, poison=True)
    Xo = oracle.dtrsm(side, uplo, trans, diag, alpha, A, B)
    Ah, Bh = _host(A, pinned), _host(B, pinned)
    st, it, est = api.trsm_mixed_host(side, uplo, trans, diag, alpha, Ah, Bh)
    X = Bh.numpy()
    assert st == 0 and it >= 1 and 0 < est <= 1e-11
    assert np.isfinite(X).all()
    # every right-hand side (column of X for left, row for right) on its own
    Xc, Oc = (X, Xo) if side == 0 else (X.T, Xo.T)
    for j in range(Xc.shape[1]):
        assert np.linalg.norm(Xc[:, j] - Oc[:, j]) <= TOL * np.linalg.norm(Oc[:, j]), j
    hist = api.gb_mixed_history()  # merged over the blocks: the longest refinement
    assert len(hist) == it and all(r > 0 for r, _ in hist)


@pytest.mark.parametrize("side", [0, 1])
def test_pipelined_failure_in_a_later_block_leaves_b_unchanged(monkeypatch, side):
    """A non-finite right-hand side in the second block returns
    GB_STATUS_RANGE after the first block's solution already went back to
    the host: the library restores it, and B is left exactly as it was."""
    from paper_2305_19917_gb300 import api
    monkeypatch.setenv("GB_MIXED_HOST_BLOCKS", "2")
    m, n = (200, 300) if side == 0 else (300, 200)
    A, B = inputs.make_problem(side, 0, 0, 0, m, n, seed=12)
    if side == 0:
        B[7, 280] = np.inf   # block 2 = columns 256..299
    else:
        B[280, 7] = np.inf   # block 2 = rows 256..299
    Bh = _host(B, True)
    B0 = Bh.numpy().copy()
    st, it, est = api.trsm_mixed_host(side, 0, 0, 0, 1.0, _host(A, True), Bh)
    assert st == api.STATUS_RANGE
    assert np.array_equal(Bh.numpy(), B0)

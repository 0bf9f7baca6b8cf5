"""The no-allocation entry point gb_dtrsm_mixed_noalloc, through the C-ABI.

It exists for callers that must not allocate device memory (their memory is
owned by another allocator, or the allocator may not be called where they
run); it works from a fixed scratch array inside the library.  Checked here:
two calls in a row on different problems (so the second sees the first's
leftovers in the shared scratch) each match gb_dtrsm_mixed on the same
inputs within the mixed path's 1e-10 tolerance (and the FP64 oracle), and a
problem larger than the scratch is refused without touching B.
This file is collected last on purpose.
"""
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


def _run(fn_name, side, uplo, trans, diag, alpha, A, B):
    import torch
    from paper_2305_19917_gb300 import api
    Ad = api.to_device_colmajor(A, torch.float64)
    Bd = api.to_device_colmajor(B, torch.float64)
    m, n = B.shape
    fn = getattr(api, fn_name)
    st, it, est = fn(side, uplo, trans, diag, m, n, alpha, Ad.data_ptr(), Ad.stride(1) if Ad.shape[1] > 1 else m,
                     Bd.data_ptr(), Bd.stride(1) if n > 1 else m, 1e-11, api.PREC_BF16, 30,
                     torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return st, Bd.cpu().numpy()


@pytest.mark.parametrize("first,second", [
    ((0, 0, 0, 0, 300, 170, 1.5, 11), (1, 1, 1, 1, 200, 256, -0.5, 12)),
])
def test_noalloc_matches_allocating_entry_twice(first, second):
    for side, uplo, trans, diag, m, n, alpha, seed in (first, second):
        A, B = inputs.make_problem(side, uplo, trans, diag, m, n, seed)
        st_ref, X_ref = _run("gb_dtrsm_mixed", side, uplo, trans, diag, alpha, A, B)
        st, X = _run("gb_dtrsm_mixed_noalloc", side, uplo, trans, diag, alpha, A, B)
        assert st_ref == 0 and st == 0, (st_ref, st)
        assert np.linalg.norm(X - X_ref) <= TOL * np.linalg.norm(X_ref)
        Xo = oracle.dtrsm(side, uplo, trans, diag, alpha, A, B)
        assert np.linalg.norm(X - Xo) <= TOL * np.linalg.norm(Xo)


def test_noalloc_refuses_problems_beyond_its_scratch():
    import torch
    from paper_2305_19917_gb300 import api
    m = n = 1024  # padded work space ~45 MB > 16 MiB
    A, B = inputs.make_problem(0, 0, 0, 0, m, n, seed=1)
    Ad = api.to_device_colmajor(A, torch.float64)
    Bd = api.to_device_colmajor(B, torch.float64)
    st, it, est = api.gb_dtrsm_mixed_noalloc(0, 0, 0, 0, m, n, 1.0, Ad.data_ptr(), m, Bd.data_ptr(), m, 1e-11,
                                             api.PREC_BF16, 30, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert st == api.STATUS_SCRATCH_TOO_SMALL
    assert np.array_equal(Bd.cpu().numpy(), B)

"""GPU tests of the tcgen05 BF16 GEMM update C = alpha*C - A*B.

The reference is computed on the CPU in FP64 from the same BF16 values (no
GPU result feeds it).  Besides accuracy on ragged shapes, one test checks the
property the split-precision residual relies on: products of small integers
(|digit| <= 32) summed over K <= 16384 stay exact in the FP32 accumulator, so
the GPU result must equal the exact integer sum.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2305_19917_gb300 import build
    build.build()


def _run(A_bf, B_bf, C0, alpha):
    """A_bf: torch bf16 (M, K) row-major on CPU; B_bf: torch bf16 (K, N);
    C0: numpy float32 (M, N).  Returns the GPU C as float64 numpy."""
    import torch
    from paper_2305_19917_gb300 import api
    M, K = A_bf.shape
    N = B_bf.shape[1]
    Ad = A_bf.contiguous().cuda()                 # row-major, lda = K
    Bd = B_bf.t().contiguous().cuda()             # (N, K) row-major = column-major K x N, ldb = K
    Cd = torch.as_tensor(np.asarray(C0, dtype=np.float32)).t().contiguous().cuda()  # (N, M) -> col-major
    st = api.gb_bf16_gemm_update(M, N, K, Ad.data_ptr(), K, Bd.data_ptr(), K, Cd.data_ptr(), M, alpha, 0)
    assert st == 0, api.gb_status_string(st)
    torch.cuda.synchronize()
    assert api.gb_device_status(1) == 0
    return Cd.t().double().cpu().numpy()


@pytest.mark.parametrize("M,N,K", [(128, 256, 64), (300, 700, 192), (1, 1, 64), (129, 257, 1024),
                                   (512, 512, 4096), (1000, 16300, 192), (2048, 16384, 128)])
def test_bf16_gemm_matches_fp64_reference(M, N, K):
    """Ragged and tile-aligned shapes; the last two take the persistent
    kernel, with 128-wide tiles (8 x 128 of them fill 6.7 rounds of the SMs
    against 3.4 rounds of 8 x 64 256-wide ones; ragged edges in both M and N)
    and with 256-wide tiles."""
    import torch
    g = torch.Generator().manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    B = torch.randn(K, N, generator=g).to(torch.bfloat16)
    C0 = torch.randn(M, N, generator=g).numpy().astype(np.float32)
    alpha = 1.5
    got = _run(A, B, C0, alpha)
    ref = alpha * C0.astype(np.float64) - A.double().numpy() @ B.double().numpy()
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err < 1e-5, err


def test_integer_sums_are_exact_up_to_2_pow_24():
    import torch
    M, N, K = 128, 256, 16384
    rng = np.random.default_rng(0)
    Ai = rng.integers(-32, 33, size=(M, K))
    Bi = rng.integers(-32, 33, size=(K, N))
    # one row/column pair at the extreme: every product +1024, sum 2^24
    Ai[0, :] = 32
    Bi[:, 0] = 32
    A = torch.as_tensor(Ai, dtype=torch.float32).to(torch.bfloat16)
    B = torch.as_tensor(Bi, dtype=torch.float32).to(torch.bfloat16)
    got = _run(A, B, np.zeros((M, N), np.float32), 1.0)
    ref = -(Ai.astype(np.int64) @ Bi.astype(np.int64))
    assert ref[0, 0] == -(2 ** 24)
    assert np.array_equal(got, ref.astype(np.float64))


def test_rejects_bad_arguments():
    from paper_2305_19917_gb300 import api
    assert api.gb_bf16_gemm_update(-1, 1, 64, 16, 64, 16, 64, 16, 1, 1.0, 0) == -1
    assert api.gb_bf16_gemm_update(4, 4, 48, 16, 64, 16, 64, 16, 4, 1.0, 0) == -3
    assert api.gb_bf16_gemm_update(4, 4, 64, 16, 60, 16, 64, 16, 4, 1.0, 0) == -5

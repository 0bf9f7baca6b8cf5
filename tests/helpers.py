"""Shared helpers of the GPU parity tests (test-side code only)."""
import numpy as np

import oracle

U64 = 2.0 ** -53
U32 = 2.0 ** -24


def fwd_err(X, Xref):
    den = np.linalg.norm(Xref)
    return float(np.linalg.norm(X - Xref) / (den if den > 0 else 1.0))


def bwd_err(side, uplo, trans, diag, alpha, A, B, X):
    """Normwise backward error eta = ||aB - op(A)X|| / (||op(A)|| ||X|| + |a| ||B||)
    in the infinity norm, the residual taken with compensated sums."""
    R = oracle.dresidual(side, uplo, trans, diag, alpha, A, B, X)
    k = B.shape[0] if side == 0 else B.shape[1]
    T = oracle.op_dense(uplo, trans, diag, A, k)
    den = np.linalg.norm(T, np.inf) * np.linalg.norm(X, np.inf) + abs(alpha) * np.linalg.norm(B, np.inf)
    return float(np.linalg.norm(R, np.inf) / (den if den > 0 else 1.0))


def gpu_solve(side, uplo, trans, diag, alpha, A, B, dtype="f64", plan=None, ldpad=0, canary=1234.5):
    """Run the library's solve on copies of A, B; returns (X, padding_ok)."""
    import torch
    from paper_2305_19917_gb300 import api
    tdt = torch.float64 if dtype == "f64" else torch.float32
    m, n = B.shape
    k = A.shape[0]
    Ad = api.to_device_colmajor(A, tdt)
    buf = torch.full((max(n, 1), m + ldpad), canary, dtype=tdt, device="cuda").t()
    Bd = buf[:m, :n] if n > 0 else buf[:m, :0]
    if m > 0 and n > 0:
        Bd.copy_(torch.as_tensor(B).to(tdt))
    api.trsm(side, uplo, trans, diag, alpha, Ad, Bd, plan=plan)
    torch.cuda.synchronize()
    X = Bd.double().cpu().numpy() if m > 0 and n > 0 else np.zeros((m, n))
    pad_ok = True
    if ldpad > 0 and n > 0:
        pad_ok = bool(torch.all(buf[m:, :n] == canary).item())
    return X, pad_ok

"""CPU oracle for the triangular solve -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never imports, links or runs anything here, and this
package imports nothing from the product.

Contents
  * ``dtrsm``      -- plain FP64 substitution (C, ``trsm_oracle.c``): the
                      definition of the paper's triangular system solver
                      (Section IV, L x = b with many right-hand sides),
                      generalised to the BLAS ?trsm side/uplo/trans/diag forms.
  * ``dresidual``  -- R = alpha*B - op(A)*X with compensated (Dot2) sums.
  * ``exact``      -- exact rational Gauss-Jordan elimination (``exact.py``).
  * ``mlp``        -- FP64 forward/backward/Adam of the cost-model MLP.
  * ``models``     -- the paper's computation models (Section V): refinement
                      level, stop rule, task counts and Comp(i) formulas.
  * ``dpotrf``     -- plain Cholesky-Crout factorisation (C, ``potrf_oracle.c``),
                      the factorisation the paper names as the next user of its
                      solver (Section VIII).
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        l = ctypes.CDLL(path)
        i64, dbl, ip = ctypes.c_int64, ctypes.c_double, ctypes.c_int
        pd = ctypes.POINTER(ctypes.c_double)
        l.oracle_dtrsm.argtypes = [ip, ip, ip, ip, i64, i64, dbl, pd, i64, pd, i64, ip]
        l.oracle_dtrsm.restype = ip
        l.oracle_dresidual.argtypes = [ip, ip, ip, ip, i64, i64, dbl, pd, i64, pd, i64,
                                       pd, i64, pd, i64, ip]
        l.oracle_dresidual.restype = ip
        l.oracle_max_threads.argtypes = []
        l.oracle_max_threads.restype = ip
        pf = ctypes.POINTER(ctypes.c_float)
        l.oracle_mlp_param_count.argtypes = [ip]
        l.oracle_mlp_param_count.restype = i64
        l.oracle_mlp_loss_grad.argtypes = [pf, ip, pf, pf, i64, pd, pd]
        l.oracle_mlp_loss_grad.restype = dbl
        l.oracle_adam.argtypes = [pd, pd, pd, pd, i64, dbl, dbl, dbl, dbl, ip]
        l.oracle_adam.restype = None
        l.oracle_dpotrf.argtypes = [ip, i64, pd, i64]
        l.oracle_dpotrf.restype = i64
        _lib = l
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _fortran64(x):
    return np.asfortranarray(np.asarray(x, dtype=np.float64))


def max_threads() -> int:
    return lib().oracle_max_threads()


def dtrsm(side, uplo, trans, diag, alpha, A, B, nthreads=0):
    """Return X solving op(A) X = alpha B (side 0) or X op(A) = alpha B (side 1).

    A, B: 2-D arrays (any order; copied to column-major FP64).  side/uplo/
    trans/diag are 0/1 as in BLAS (Left/Lower/NoTrans/NonUnit = 0).
    nthreads <= 0 uses the OpenMP default.
    """
    A = _fortran64(A)
    X = _fortran64(B).copy(order="F")
    m, n = X.shape
    k = m if side == 0 else n
    assert A.shape[0] >= k and A.shape[1] >= k
    lda = max(1, A.shape[0])
    ldb = max(1, m)
    rc = lib().oracle_dtrsm(side, uplo, trans, diag, m, n, float(alpha), _ptr(A), lda,
                            _ptr(X), ldb, int(nthreads))
    if rc != 0:
        raise ValueError(f"oracle_dtrsm: invalid argument {-rc}")
    return X


def dtrsm_inplace(side, uplo, trans, diag, alpha, A, X, nthreads=0):
    """In-place variant on a column-major FP64 array X (used for timing)."""
    assert X.flags.f_contiguous and X.dtype == np.float64
    assert A.flags.f_contiguous and A.dtype == np.float64
    m, n = X.shape
    rc = lib().oracle_dtrsm(side, uplo, trans, diag, m, n, float(alpha), _ptr(A),
                            max(1, A.shape[0]), _ptr(X), max(1, m), int(nthreads))
    if rc != 0:
        raise ValueError(f"oracle_dtrsm: invalid argument {-rc}")


def dresidual(side, uplo, trans, diag, alpha, A, B, X, nthreads=0):
    """R = alpha*B - op(A)*X (Left) or alpha*B - X*op(A) (Right), each entry
    accurate to about 2^-106 relative to sum |a||x| (compensated dot)."""
    A = _fortran64(A)
    B = _fortran64(B)
    X = _fortran64(X)
    m, n = B.shape
    R = np.zeros((m, n), dtype=np.float64, order="F")
    lib().oracle_dresidual(side, uplo, trans, diag, m, n, float(alpha), _ptr(A),
                           max(1, A.shape[0]), _ptr(B), max(1, m), _ptr(X), max(1, m),
                           _ptr(R), max(1, m), int(nthreads))
    return R


def op_dense(uplo, trans, diag, A, k):
    """Dense k x k op(A) with zeros outside the referenced triangle and ones on
    a unit diagonal (reads only the referenced part of A)."""
    A = np.asarray(A, dtype=np.float64)[:k, :k]
    mask = np.tril(np.ones((k, k), dtype=bool), -1) if uplo == 0 else \
        np.triu(np.ones((k, k), dtype=bool), 1)
    T = np.where(mask, A, 0.0)
    T[np.diag_indices(k)] = 1.0 if diag == 1 else np.diagonal(A)
    return T.T.copy() if trans == 1 else T


def dpotrf(uplo, A):
    """(F, info): the Cholesky factor of the symmetric positive definite A
    (uplo 0: lower L with A = L L^T; 1: upper U with A = U^T U) written over
    the named triangle of a column-major copy of A (the other triangle is
    copied unchanged); info = 0, or j + 1 when column j has a non-positive
    pivot (LAPACK convention)."""
    F = _fortran64(A).copy(order="F")
    n = F.shape[0]
    assert F.shape[1] == n
    info = lib().oracle_dpotrf(int(uplo), n, _ptr(F), max(1, n))
    if info < 0:
        raise ValueError(f"oracle_dpotrf: invalid argument {-info}")
    return F, int(info)


# ---- cost-model network (FP64) ---------------------------------------------------

def mlp_param_count(D):
    return lib().oracle_mlp_param_count(D)


def mlp_loss_grad(params, X, T, want_grad=True):
    """(loss, predictions, gradient) of the 3 x 64 GELU network, FP64."""
    P = np.ascontiguousarray(params, dtype=np.float32)
    X = np.ascontiguousarray(X, dtype=np.float32)
    T = np.ascontiguousarray(T, dtype=np.float32)
    n, D = X.shape
    y = np.zeros(n)
    g = np.zeros(P.size) if want_grad else None
    pf = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))  # noqa: E731
    loss = lib().oracle_mlp_loss_grad(pf(P), D, pf(X), pf(T), n, _ptr(y), _ptr(g) if want_grad else None)
    return loss, y, g


def adam_step(p, g, m, v, lr, b1, b2, eps, step):
    """One FP64 Adam step, in place on float64 arrays p, m, v."""
    for a in (p, g, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    lib().oracle_adam(_ptr(p), _ptr(g), _ptr(m), _ptr(v), p.size, lr, b1, b2, eps, step)

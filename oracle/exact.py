"""Exact rational triangular solve -- TEST INFRASTRUCTURE ONLY.

Brute force, sharing nothing with substitution: the dense op(A) is built
(zeros outside the referenced triangle, ones on a unit diagonal), then the
augmented system [op(A) | alpha*B] is reduced by Gauss-Jordan elimination in
``fractions.Fraction`` (any nonzero pivot, row swaps allowed).  The right-side
form X op(A) = alpha B is solved as its transpose op(A)^T X^T = alpha B^T.

Every binary64 value is an exact rational, so for inputs that are doubles the
result is the exact X = alpha op(A)^{-1} B (or alpha B op(A)^{-1}); the FP64
oracle's rounding error is measured against it.  Meant for m, n <= 8.
"""
from fractions import Fraction


def _frac(v):
    return v if isinstance(v, Fraction) else Fraction(float(v))


def dense_op(uplo, trans, diag, A, k):
    """k x k list-of-lists of Fractions: op(A) restricted to its triangle."""
    T = [[Fraction(0)] * k for _ in range(k)]
    for r in range(k):
        for c in range(k):
            if r == c:
                val = Fraction(1) if diag == 1 else _frac(A[r][c])
            elif (uplo == 0 and r > c) or (uplo == 1 and r < c):
                val = _frac(A[r][c])
            else:
                continue
            if trans == 1:
                T[c][r] = val
            else:
                T[r][c] = val
    return T


def gauss_jordan(M, Rhs):
    """Solve M Y = Rhs exactly (M square, nonsingular).  Returns Y."""
    k = len(M)
    ncol = len(Rhs[0]) if k else 0
    aug = [list(M[i]) + list(Rhs[i]) for i in range(k)]
    for col in range(k):
        piv = next(r for r in range(col, k) if aug[r][col] != 0)
        aug[col], aug[piv] = aug[piv], aug[col]
        p = aug[col][col]
        aug[col] = [v / p for v in aug[col]]
        for r in range(k):
            if r != col and aug[r][col] != 0:
                f = aug[r][col]
                aug[r] = [a - f * b for a, b in zip(aug[r], aug[col])]
    return [row[k:k + ncol] for row in aug]


def exact_trsm(side, uplo, trans, diag, alpha, A, B):
    """Exact X for op(A) X = alpha B (side 0) or X op(A) = alpha B (side 1).

    A: k x k (nested lists or 2-D array), B: m x n.  Returns m x n Fractions.
    """
    m = len(B)
    n = len(B[0]) if m else 0
    al = _frac(alpha)
    if side == 0:
        T = dense_op(uplo, trans, diag, A, m)
        rhs = [[al * _frac(B[i][j]) for j in range(n)] for i in range(m)]
        return gauss_jordan(T, rhs)
    T = dense_op(uplo, trans, diag, A, n)
    Tt = [[T[c][r] for c in range(n)] for r in range(n)]          # op(A)^T
    rhs = [[al * _frac(B[i][j]) for i in range(m)] for j in range(n)]  # alpha B^T
    Yt = gauss_jordan(Tt, rhs)                                       # X^T
    return [[Yt[j][i] for j in range(n)] for i in range(m)]

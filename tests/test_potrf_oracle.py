"""Pins of the Cholesky oracle (oracle/potrf_oracle.c), the factorisation the
paper names as the next user of its triangular solver (Section VIII).

Each check is fixed by mathematics, not by the oracle itself:
  * A = I gives L = I, a diagonal A gives L = sqrt(diag) (exact);
  * A(i, j) = min(i, j) (1-based) has the all-ones lower triangle as its
    factor, the symmetric Pascal matrix C(i + j, i) the lower Pascal matrix
    C(i, j): integer closed forms, reproduced exactly;
  * random SPD matrices of the Cholesky recipe: L L^T reproduces A to a few
    units of n u (residual computed in exact rational arithmetic), and L
    matches LAPACK's factor (numpy.linalg.cholesky);
  * the upper factor is the transpose of the lower one, bit for bit;
  * only the named triangle is read (NaN in the other one);
  * info = j + 1 at the first non-positive pivot (LAPACK convention);
  * planted mistakes in the oracle's C source each break a pin.
"""
import os
import shutil
import subprocess
import tempfile
from fractions import Fraction
from math import comb

import numpy as np
import pytest

import oracle
from paper_2305_19917_gb300 import inputs

U = 2.0 ** -53


def test_identity_and_diagonal_exact():
    for uplo in (0, 1):
        F, info = oracle.dpotrf(uplo, np.eye(9))
        assert info == 0 and np.array_equal(F, np.eye(9))
        d = np.array([4.0, 9.0, 2.0, 0.25, 1e-300, 7.0])
        F, info = oracle.dpotrf(uplo, np.diag(d))
        assert info == 0 and np.array_equal(np.diag(F), np.sqrt(d))


@pytest.mark.parametrize("uplo", [0, 1])
def test_min_matrix_factor_is_all_ones(uplo):
    n = 12
    A = np.array([[min(i, j) for j in range(1, n + 1)] for i in range(1, n + 1)], dtype=float)
    F, info = oracle.dpotrf(uplo, A)
    assert info == 0
    T = np.tril(F) if uplo == 0 else np.triu(F).T
    assert np.array_equal(T, np.tril(np.ones((n, n))))


@pytest.mark.parametrize("uplo", [0, 1])
def test_pascal_matrix_factor_is_lower_pascal(uplo):
    n = 14
    A = np.array([[comb(i + j, i) for j in range(n)] for i in range(n)], dtype=float)
    L = np.array([[comb(i, j) for j in range(n)] for i in range(n)], dtype=float)
    F, info = oracle.dpotrf(uplo, A)
    assert info == 0
    T = np.tril(F) if uplo == 0 else np.triu(F).T
    assert np.array_equal(T, L)


def _exact_residual_rel(A, T):
    """|| A - T T^T ||_F / ||A||_F in exact rational arithmetic."""
    n = A.shape[0]
    Tq = [[Fraction(float(T[i, j])) for j in range(n)] for i in range(n)]
    num = Fraction(0)
    for i in range(n):
        for j in range(n):
            s = sum((Tq[i][k] * Tq[j][k] for k in range(n)), Fraction(0))
            r = Fraction(float(A[i, j])) - s
            num += r * r
    den = sum(Fraction(float(v)) ** 2 for v in A.ravel())
    return (float(num) / float(den)) ** 0.5


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (7, 2), (16, 3)])
def test_residual_exact_and_lapack(n, seed):
    A = inputs.make_spd(n, seed)
    F, info = oracle.dpotrf(0, A)
    assert info == 0
    L = np.tril(F)
    assert _exact_residual_rel(A, L) <= 4 * n * U
    Lref = np.linalg.cholesky(A)
    assert np.linalg.norm(L - Lref) <= 8 * n * U * np.linalg.norm(Lref)


def test_upper_is_transpose_of_lower_bitwise():
    A = inputs.make_spd(40, seed=5)
    Fl, il = oracle.dpotrf(0, A)
    Fu, iu = oracle.dpotrf(1, A)
    assert il == iu == 0
    assert np.array_equal(np.tril(Fl), np.triu(Fu).T)


def test_other_triangle_not_read():
    A = inputs.make_spd(30, seed=6)
    for uplo in (0, 1):
        P = A.copy(order="F")
        if uplo == 0:
            P[np.triu_indices(30, 1)] = np.nan
        else:
            P[np.tril_indices(30, -1)] = np.nan
        F, info = oracle.dpotrf(uplo, P)
        Fr, _ = oracle.dpotrf(uplo, A)
        T, Tr = (np.tril(F), np.tril(Fr)) if uplo == 0 else (np.triu(F), np.triu(Fr))
        assert info == 0 and np.array_equal(T, Tr)


def test_info_reports_first_bad_pivot():
    assert oracle.dpotrf(0, np.array([[1.0, 2.0], [2.0, 1.0]]))[1] == 2
    assert oracle.dpotrf(1, np.array([[1.0, 2.0], [2.0, 1.0]]))[1] == 2
    assert oracle.dpotrf(0, np.zeros((3, 3)))[1] == 1
    A = np.eye(5)
    A[2, 2] = -1.0
    assert oracle.dpotrf(0, A)[1] == 3
    A = inputs.make_spd(6, seed=1)
    A[4, 4] = np.nan
    assert oracle.dpotrf(1, A)[1] == 5


# ---------------------------------------------------------------- mutations

MUTATIONS = [
    ("diagonal sum runs one term too far",
     "for (int64_t k = 0; k < j; k++) d -= A_(j, k) * A_(j, k);",
     "for (int64_t k = 0; k <= j; k++) d -= A_(j, k) * A_(j, k);"),
    ("wrong sign in the column sum",
     "for (int64_t k = 0; k < j; k++) s -= A_(i, k) * A_(j, k);",
     "for (int64_t k = 0; k < j; k++) s += A_(i, k) * A_(j, k);"),
    ("transposed index in the upper column sum",
     "for (int64_t k = 0; k < j; k++) s -= A_(k, i) * A_(k, j);",
     "for (int64_t k = 0; k < j; k++) s -= A_(i, k) * A_(k, j);"),
    ("no square root of the lower pivot",
     "const double ljj = sqrt(d);",
     "const double ljj = d;"),
    ("column not divided by the upper pivot",
     "A_(j, i) = s / ujj;",
     "A_(j, i) = s;"),
    ("first term of each sum dropped",
     "for (int64_t k = 0; k < j; k++) s -= A_(i, k) * A_(j, k);",
     "for (int64_t k = 1; k < j; k++) s -= A_(i, k) * A_(j, k);"),
]


def _pins_pass_with(so_path):
    import ctypes
    l = ctypes.CDLL(so_path)
    l.oracle_dpotrf.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.POINTER(ctypes.c_double), ctypes.c_int64]
    l.oracle_dpotrf.restype = ctypes.c_int64

    def potrf(uplo, A):
        F = np.asfortranarray(np.array(A, dtype=np.float64))
        info = l.oracle_dpotrf(uplo, F.shape[0], F.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), F.shape[0])
        return F, info

    n = 10
    Am = np.array([[min(i, j) for j in range(1, n + 1)] for i in range(1, n + 1)], dtype=float)
    Ap = np.array([[comb(i + j, i) for j in range(n)] for i in range(n)], dtype=float)
    Lp = np.array([[comb(i, j) for j in range(n)] for i in range(n)], dtype=float)
    for uplo in (0, 1):
        for A, Lx in ((Am, np.tril(np.ones((n, n)))), (Ap, Lp)):
            F, info = potrf(uplo, A)
            T = np.tril(F) if uplo == 0 else np.triu(F).T
            if info != 0 or not np.array_equal(T, Lx):
                return False
        A = inputs.make_spd(9, seed=4)
        F, info = potrf(uplo, A)
        T = np.tril(F) if uplo == 0 else np.triu(F).T
        if info != 0 or np.linalg.norm(T @ T.T - A) > 64 * 9 * U * np.linalg.norm(A):
            return False
    return True


def test_pins_catch_planted_mistakes():
    src_path = os.path.join(os.path.dirname(oracle.__file__), "potrf_oracle.c")
    with open(src_path) as f:
        src = f.read()
    tmp = tempfile.mkdtemp()
    try:
        def build(text, d):
            os.makedirs(d, exist_ok=True)
            c, so = os.path.join(d, "m.c"), os.path.join(d, "m.so")
            with open(c, "w") as f:
                f.write(text)
            subprocess.run(["gcc", "-O1", "-fPIC", "-shared", "-ffp-contract=off", "-o", so, c, "-lm"], check=True)
            return so
        assert _pins_pass_with(build(src, os.path.join(tmp, "orig")))
        for i, (desc, old, new) in enumerate(MUTATIONS):
            assert src.count(old) == 1, desc
            assert not _pins_pass_with(build(src.replace(old, new), os.path.join(tmp, str(i)))), desc
    finally:
        shutil.rmtree(tmp)

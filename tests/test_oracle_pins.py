"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Every check here is CPU-only.  The oracle is the plain definition of the
paper's triangular system solver (Section IV: L x = b with many right-hand
sides), extended to the BLAS ?trsm forms; these tests tie it to
  * special cases with a known closed form (identity, diagonal, bidiagonal),
  * exact rational Gauss-Jordan elimination (brute force, m, n <= 8),
  * the residual invariant of a backward-stable substitution,
  * the transpose / anti-transpose identities that link the eight cases,
  * LAPACK's triangular solve (scipy) as an independent library routine,
  * the not-referenced rules of the BLAS interface,
and a mutation test shows that plausible mistakes planted in the oracle's C
source are caught by these pins.
"""
import itertools
import os
import shutil
import subprocess
import tempfile
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import exact
from paper_2305_19917_gb300 import inputs

U = 2.0 ** -53
COMBOS = list(itertools.product((0, 1), (0, 1), (0, 1), (0, 1)))  # side, uplo, trans, diag


def _k(side, m, n):
    return m if side == 0 else n


def _dense_opA(uplo, trans, diag, A, k):
    return oracle.op_dense(uplo, trans, diag, A, k)


def _apply(side, opA, X):
    return opA @ X if side == 0 else X @ opA


def _relerr(X, Y):
    den = np.linalg.norm(Y)
    return np.linalg.norm(X - Y) / (den if den > 0 else 1.0)


# ---------------------------------------------------------------- special cases

@pytest.mark.parametrize("side,uplo,trans,diag", COMBOS)
def test_identity_gives_alpha_b_bitwise(side, uplo, trans, diag):
    m, n = 23, 17
    k = _k(side, m, n)
    rng = np.random.default_rng(5)
    A = np.asfortranarray(np.eye(k))
    if diag == 1:
        A[np.diag_indices(k)] = 7.25  # not read with a unit diagonal
    B = rng.standard_normal((m, n))
    alpha = 1.5
    X = oracle.dtrsm(side, uplo, trans, diag, alpha, A, B)
    assert np.array_equal(X, alpha * B)


@pytest.mark.parametrize("side,uplo,trans,diag", COMBOS)
def test_diagonal_gives_alpha_b_over_d_bitwise(side, uplo, trans, diag):
    m, n = 19, 21
    k = _k(side, m, n)
    rng = np.random.default_rng(11)
    d = rng.uniform(1.0, 2.0, k)
    A = np.asfortranarray(np.diag(d))
    B = rng.standard_normal((m, n))
    alpha = -0.75
    X = oracle.dtrsm(side, uplo, trans, diag, alpha, A, B)
    if diag == 1:
        expect = alpha * B
    elif side == 0:
        expect = (alpha * B) / d[:, None]
    else:
        expect = (alpha * B) / d[None, :]
    assert np.array_equal(X, expect)


def _bidiag_lower_inverse(d, l):
    """Exact inverse of the lower bidiagonal matrix with diagonal d and
    subdiagonal l (L[i+1, i] = l[i]):
        (L^-1)_ij = (-1)^(i-j) prod_{k=j}^{i-1} l_k / prod_{k=j}^{i} d_k, i >= j."""
    k = len(d)
    inv = [[Fraction(0)] * k for _ in range(k)]
    for j in range(k):
        num, den = Fraction(1), Fraction(d[j])
        inv[j][j] = 1 / den
        for i in range(j + 1, k):
            num *= Fraction(l[i - 1])
            den *= Fraction(d[i])
            inv[i][j] = (-1) ** (i - j) * num / den
    return inv


@pytest.mark.parametrize("side,uplo,trans", list(itertools.product((0, 1), (0, 1), (0, 1))))
def test_bidiagonal_closed_form(side, uplo, trans):
    m, n = 12, 9
    k = _k(side, m, n)
    rng = np.random.default_rng(3 + 4 * side + 2 * uplo + trans)
    d = rng.uniform(1.0, 2.0, k)
    l = rng.uniform(-1.0, 1.0, k - 1)
    Lfull = np.diag(d) + np.diag(l, -1)           # lower bidiagonal
    A = Lfull if uplo == 0 else Lfull.T.copy()    # upper: stored transpose
    B = rng.standard_normal((m, n))
    alpha = 1.5
    Linv = _bidiag_lower_inverse([Fraction(float(x)) for x in d], [Fraction(float(x)) for x in l])
    # op(A) is L or L^T; op(A)^-1 is Linv or Linv^T accordingly.
    op_is_lower = (uplo == 0) != (trans == 1)
    inv = Linv if op_is_lower else [list(r) for r in zip(*Linv)]
    Bf = [[Fraction(float(B[i, j])) for j in range(n)] for i in range(m)]
    al = Fraction(alpha)
    if side == 0:
        Xe = [[al * sum(inv[i][q] * Bf[q][j] for q in range(k)) for j in range(n)] for i in range(m)]
    else:
        Xe = [[al * sum(Bf[i][q] * inv[q][j] for q in range(k)) for j in range(n)] for i in range(m)]
    Xe = np.array([[float(v) for v in row] for row in Xe])
    X = oracle.dtrsm(side, uplo, trans, 0, alpha, A, B)
    assert _relerr(X, Xe) <= 4 * k * U


# ------------------------------------------------------------- exact rationals

@pytest.mark.parametrize("side,uplo,trans,diag", COMBOS)
def test_exact_rational_small(side, uplo, trans, diag):
    for seed, (m, n) in enumerate([(1, 1), (2, 3), (3, 2), (5, 7), (8, 8), (7, 4)]):
        A, B = inputs.make_problem(side, uplo, trans, diag, m, n, seed=100 + seed)
        k = _k(side, m, n)
        alpha = 1.5
        Xe = exact.exact_trsm(side, uplo, trans, diag, alpha, A.tolist(), B.tolist())
        Xe = np.array([[float(v) for v in row] for row in Xe])
        X = oracle.dtrsm(side, uplo, trans, diag, alpha, A, B)
        T = _dense_opA(uplo, trans, diag, A, k)
        kappa = np.linalg.norm(T, np.inf) * np.linalg.norm(np.linalg.inv(T), np.inf)
        assert _relerr(X, Xe) <= 4 * k * U * kappa, (m, n)


def test_exact_solver_itself_on_known_system():
    # [[2, 0], [3, 4]] x = [2, 11]  ->  x = [1, 2]  (hand-checked)
    X = exact.exact_trsm(0, 0, 0, 0, 1, [[2, 0], [3, 4]], [[2], [11]])
    assert X == [[Fraction(1)], [Fraction(2)]]
    # X [[2, 1], [0, 4]] = [[4, 10]] -> X = [2, 2]
    X = exact.exact_trsm(1, 1, 0, 0, 1, [[2, 1], [0, 4]], [[4, 10]])
    assert X == [[Fraction(2), Fraction(2)]]


# ---------------------------------------------------------- residual invariant

@pytest.mark.parametrize("side,uplo,trans,diag", COMBOS)
def test_residual_invariant(side, uplo, trans, diag):
    m, n = 150, 37
    A, B = inputs.make_problem(side, uplo, trans, diag, m, n, seed=7)
    alpha = 1.5
    X = oracle.dtrsm(side, uplo, trans, diag, alpha, A, B)
    R = oracle.dresidual(side, uplo, trans, diag, alpha, A, B, X)
    k = _k(side, m, n)
    T = _dense_opA(uplo, trans, diag, A, k)
    An = np.linalg.norm(T, np.inf)
    eta = np.linalg.norm(R, np.inf) / (An * np.linalg.norm(X, np.inf) + abs(alpha) * np.linalg.norm(B, np.inf))
    assert eta <= k * U


def test_dresidual_matches_exact_rationals():
    side, uplo, trans, diag = 0, 0, 0, 0
    m, n = 6, 3
    A, B = inputs.make_problem(side, uplo, trans, diag, m, n, seed=1)
    rng = np.random.default_rng(2)
    X = rng.standard_normal((m, n))
    alpha = 1.5
    R = oracle.dresidual(side, uplo, trans, diag, alpha, A, B, X)
    T = exact.dense_op(uplo, trans, diag, A.tolist(), m)
    for i in range(m):
        for j in range(n):
            ex = Fraction(alpha) * Fraction(float(B[i, j])) - sum(
                T[i][q] * Fraction(float(X[q, j])) for q in range(m))
            scale = sum(abs(T[i][q] * Fraction(float(X[q, j]))) for q in range(m))
            assert abs(Fraction(R[i, j]) - ex) <= Fraction(2 * U) * abs(ex) + Fraction(4 * U * U) * scale


# ------------------------------------------------------------ transpose links

@pytest.mark.parametrize("diag", (0, 1))
@pytest.mark.parametrize("uplo", (0, 1))
def test_upper_notrans_equals_lower_trans_of_transpose(uplo, diag):
    m, n = 64, 29
    A, B = inputs.make_problem(0, uplo, 0, diag, m, n, seed=17)
    X1 = oracle.dtrsm(0, uplo, 0, diag, 1.5, A, B)
    X2 = oracle.dtrsm(0, 1 - uplo, 1, diag, 1.5, A.T.copy(), B)
    assert _relerr(X1, X2) <= 2 * m * U


@pytest.mark.parametrize("uplo,trans,diag", list(itertools.product((0, 1), (0, 1), (0, 1))))
def test_right_side_is_transposed_left_side(uplo, trans, diag):
    m, n = 31, 45
    A, B = inputs.make_problem(1, uplo, trans, diag, m, n, seed=23)
    XR = oracle.dtrsm(1, uplo, trans, diag, -2.0, A, B)
    XL = oracle.dtrsm(0, uplo, 1 - trans, diag, -2.0, A, B.T.copy())
    assert _relerr(XR.T, XL) <= 2 * n * U


@pytest.mark.parametrize("trans,diag", list(itertools.product((0, 1), (0, 1))))
def test_anti_transpose_links_lower_and_upper(trans, diag):
    # J A J with J the exchange matrix turns lower into upper; reversing the
    # rows of B reverses the rows of X.
    m, n = 40, 11
    A, B = inputs.make_problem(0, 0, trans, diag, m, n, seed=31)
    X1 = oracle.dtrsm(0, 0, trans, diag, 1.0, A, B)
    AJ = np.asfortranarray(A[::-1, ::-1])
    X2 = oracle.dtrsm(0, 1, trans, diag, 1.0, AJ, np.asfortranarray(B[::-1, :]))
    assert _relerr(X1, X2[::-1, :]) <= 2 * m * U


# ------------------------------------------------------------- library routine

@pytest.mark.parametrize("side,uplo,trans,diag", COMBOS)
def test_against_lapack_triangular_solve(side, uplo, trans, diag):
    sl = pytest.importorskip("scipy.linalg")
    m, n = 57, 33
    A, B = inputs.make_problem(side, uplo, trans, diag, m, n, seed=41)
    X = oracle.dtrsm(side, uplo, trans, diag, 1.5, A, B)
    if side == 0:
        Y = sl.solve_triangular(A, 1.5 * B, lower=(uplo == 0), trans=trans, unit_diagonal=bool(diag))
    else:
        # X op(A) = aB  <=>  op(A)^T X^T = aB^T
        Y = sl.solve_triangular(A, 1.5 * B.T, lower=(uplo == 0), trans=1 - trans,
                                unit_diagonal=bool(diag)).T
    assert _relerr(X, Y) <= 4 * _k(side, m, n) * U


# --------------------------------------------------------- interface semantics

@pytest.mark.parametrize("side,uplo,trans,diag", COMBOS)
def test_unreferenced_entries_are_not_read(side, uplo, trans, diag):
    m, n = 33, 20
    A0, B = inputs.make_problem(side, uplo, trans, diag, m, n, seed=9)
    A1, _ = inputs.make_problem(side, uplo, trans, diag, m, n, seed=9, poison=True)
    X0 = oracle.dtrsm(side, uplo, trans, diag, 1.5, A0, B)
    X1 = oracle.dtrsm(side, uplo, trans, diag, 1.5, A1, B)
    assert np.all(np.isfinite(X1))
    assert np.array_equal(X0, X1)


def test_alpha_zero_does_not_read_a_or_b():
    A = np.full((6, 6), np.nan, order="F")
    B = np.full((6, 4), np.nan, order="F")
    for side, uplo, trans, diag in COMBOS:
        k = 6
        X = oracle.dtrsm(side, uplo, trans, diag, 0.0, A[:k, :k], B)
        assert np.array_equal(X, np.zeros((6, 4)))


def test_empty_and_argument_errors():
    X = oracle.dtrsm(0, 0, 0, 0, 1.0, np.zeros((0, 0)), np.zeros((0, 5)))
    assert X.shape == (0, 5)
    X = oracle.dtrsm(0, 0, 0, 0, 1.0, np.eye(3), np.zeros((3, 0)))
    assert X.shape == (3, 0)
    with pytest.raises(ValueError, match="argument 1"):
        oracle.dtrsm(2, 0, 0, 0, 1.0, np.eye(2), np.ones((2, 2)))
    with pytest.raises(ValueError, match="argument 4"):
        oracle.dtrsm(0, 0, 0, 5, 1.0, np.eye(2), np.ones((2, 2)))


def test_thread_count_does_not_change_bits():
    A, B = inputs.make_problem(0, 0, 0, 0, 300, 64, seed=2)
    X1 = oracle.dtrsm(0, 0, 0, 0, 1.0, A, B, nthreads=1)
    Xn = oracle.dtrsm(0, 0, 0, 0, 1.0, A, B, nthreads=max(2, oracle.max_threads()))
    assert np.array_equal(X1, Xn)


# --------------------------------------------------------------- golden file

def test_golden_exact_solution():
    import json
    path = os.path.join(os.path.dirname(__file__), "golden", "exact_small.json")
    with open(path) as f:
        g = json.load(f)
    for case in g["cases"]:
        A = np.array(case["A"], dtype=np.float64)
        B = np.array(case["B"], dtype=np.float64)
        Xe = np.array([[float(Fraction(v)) for v in row] for row in case["X_exact"]])
        X = oracle.dtrsm(case["side"], case["uplo"], case["trans"], case["diag"], case["alpha"], A, B)
        assert _relerr(X, Xe) <= 64 * U


# ---------------------------------------------------------------- mutations

MUTATIONS = [
    # (description, original text, mutated text)
    ("alpha dropped in Left/Lower/N",
     "for (int64_t i = 0; i < m; i++) B_(i, j) = alpha * B_(i, j);\n        for (int64_t k = 0; k < m; k++) {",
     "for (int64_t i = 0; i < m; i++) B_(i, j) = B_(i, j);\n        for (int64_t k = 0; k < m; k++) {"),
    ("wrong sign in Left/Lower/T",
     "for (int64_t i = k + 1; i < m; i++) s -= A_(i, k) * B_(i, j);",
     "for (int64_t i = k + 1; i < m; i++) s += A_(i, k) * B_(i, j);"),
    ("transposed operand in Left/Upper/T",
     "for (int64_t i = 0; i < k; i++) s -= A_(i, k) * B_(i, j);",
     "for (int64_t i = 0; i < k; i++) s -= A_(k, i) * B_(i, j);"),
    ("off-by-one term dropped in Right/Lower/N",
     "for (int64_t k = c + 1; k < n; k++) s -= B_(r, k) * A_(k, c);",
     "for (int64_t k = c + 2; k < n; k++) s -= B_(r, k) * A_(k, c);"),
    ("diagonal ignored in Right/Upper/N",
     "double xc = unit ? B_(r, c) : B_(r, c) / A_(c, c);",
     "double xc = B_(r, c);"),
    ("unit flag inverted in Right/Upper/T",
     "for (int64_t k = c + 1; k < n; k++) s -= B_(r, k) * A_(c, k);\n            B_(r, c) = unit ? s : s / A_(c, c);\n        }\n    }\n}\n\n/* side:",
     "for (int64_t k = c + 1; k < n; k++) s -= B_(r, k) * A_(c, k);\n            B_(r, c) = unit ? s / A_(c, c) : s;\n        }\n    }\n}\n\n/* side:"),
]


def _mutant_lib(tmpdir, src_text):
    import ctypes
    c = os.path.join(tmpdir, "m.c")
    so = os.path.join(tmpdir, "m.so")
    with open(c, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", "-O1", "-fPIC", "-shared", "-ffp-contract=off", "-o", so, c, "-lm"], check=True)
    l = ctypes.CDLL(so)
    return l


def _pins_pass_with(lib_handle):
    """Run a compact version of the pins above against another build."""
    import ctypes
    saved = oracle._lib
    i64, dbl, ip = ctypes.c_int64, ctypes.c_double, ctypes.c_int
    pd = ctypes.POINTER(ctypes.c_double)
    lib_handle.oracle_dtrsm.argtypes = [ip, ip, ip, ip, i64, i64, dbl, pd, i64, pd, i64, ip]
    lib_handle.oracle_dtrsm.restype = ip
    lib_handle.oracle_dresidual.argtypes = [ip, ip, ip, ip, i64, i64, dbl, pd, i64, pd, i64, pd, i64, pd, i64, ip]
    lib_handle.oracle_dresidual.restype = ip
    lib_handle.oracle_max_threads.restype = ip
    oracle._lib = lib_handle
    try:
        for side, uplo, trans, diag in COMBOS:
            m, n = 7, 6
            A, B = inputs.make_problem(side, uplo, trans, diag, m, n, seed=77)
            Xe = exact.exact_trsm(side, uplo, trans, diag, 1.5, A.tolist(), B.tolist())
            Xe = np.array([[float(v) for v in row] for row in Xe])
            X = oracle.dtrsm(side, uplo, trans, diag, 1.5, A, B)
            if not (_relerr(X, Xe) <= 64 * _k(side, m, n) * U):
                return False
        return True
    finally:
        oracle._lib = saved


def test_pins_catch_planted_mistakes():
    src_path = os.path.join(os.path.dirname(oracle.__file__), "trsm_oracle.c")
    with open(src_path) as f:
        src = f.read()
    tmp = tempfile.mkdtemp()
    try:
        # the unmutated source passes
        assert _pins_pass_with(_mutant_lib(tmp, src))
        for i, (desc, old, new) in enumerate(MUTATIONS):
            assert src.count(old) == 1, desc
            d = os.path.join(tmp, str(i))
            os.makedirs(d)
            assert not _pins_pass_with(_mutant_lib(d, src.replace(old, new))), desc
    finally:
        shutil.rmtree(tmp)

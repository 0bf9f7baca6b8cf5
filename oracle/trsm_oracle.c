/*
 * CPU oracle for the triangular solve.  TEST INFRASTRUCTURE ONLY: nothing on
 * the product path may call, link or execute this file; only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg use it.
 *
 * What it computes: the plain definition of the triangular system solver of
 * the paper (Section IV: L x = b with a dense lower-triangular L, extended to
 * many right-hand sides), generalised to the BLAS ?trsm forms
 *     side = Left :  op(A) X = alpha B      (A is m x m, B is m x n)
 *     side = Right:  X op(A) = alpha B      (A is n x n, B is m x n)
 * with op(A) = A or A^T, A lower or upper triangular, unit or non-unit
 * diagonal.  X overwrites B.  All matrices are column-major with leading
 * dimensions lda / ldb.
 *
 * Each of the eight (side, uplo, trans) cases is written out on its own as a
 * straight substitution (no transpose tricks, no blocking, no reordering), so
 * that the identities linking the cases are genuine tests.  Only the
 * referenced triangle of A is read; with a unit diagonal the diagonal is not
 * read.  alpha == 0 sets X = 0 without reading A or B (BLAS convention).
 *
 * Arithmetic: IEEE binary64, compiled with -ffp-contract=off and without
 * -ffast-math, fixed operation order => bit-reproducible on x86-64 and arm64.
 * Parallelism (OpenMP) is only across independent right-hand sides (columns
 * for Left, rows for Right); each one is computed in the same order whatever
 * the thread count.
 *
 * The accurate residual oracle_dresidual() computes R = alpha B - op(A) X
 * (Left) or alpha B - X op(A) (Right) with error-free transformations
 * (TwoProduct by fma, TwoSum; the compensated dot product of Ogita, Rump and
 * Oishi, 2005), accurate to about u^2 relative to |A||X|.  It serves as the
 * reference for the split-precision residual of the mixed-precision path.
 */
#include <stdint.h>
#include <math.h>
#include <stddef.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define A_(i, j) A[(size_t)(i) + (size_t)(j) * (size_t)lda]
#define B_(i, j) B[(size_t)(i) + (size_t)(j) * (size_t)ldb]

static void set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Left, Lower, NoTrans: forward substitution, column (axpy) form.
 * t = alpha*b; for k = 0..m-1: x_k = t_k / a_kk; t_i -= a_ik x_k (i > k). */
static void left_lower_n(int unit, int64_t m, int64_t n, double alpha,
                         const double *A, int64_t lda, double *B, int64_t ldb)
{
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; j++) {
        for (int64_t i = 0; i < m; i++) B_(i, j) = alpha * B_(i, j);
        for (int64_t k = 0; k < m; k++) {
            double xk = unit ? B_(k, j) : B_(k, j) / A_(k, k);
            B_(k, j) = xk;
            for (int64_t i = k + 1; i < m; i++) B_(i, j) -= A_(i, k) * xk;
        }
    }
}

/* Left, Lower, Trans: A^T is upper, backward substitution, dot form.
 * x_k = (t_k - sum_{i>k} a_ik x_i) / a_kk for k = m-1..0. */
static void left_lower_t(int unit, int64_t m, int64_t n, double alpha,
                         const double *A, int64_t lda, double *B, int64_t ldb)
{
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; j++) {
        for (int64_t k = m - 1; k >= 0; k--) {
            double s = alpha * B_(k, j);
            for (int64_t i = k + 1; i < m; i++) s -= A_(i, k) * B_(i, j);
            B_(k, j) = unit ? s : s / A_(k, k);
        }
    }
}

/* Left, Upper, NoTrans: backward substitution, column (axpy) form.
 * for k = m-1..0: x_k = t_k / a_kk; t_i -= a_ik x_k (i < k). */
static void left_upper_n(int unit, int64_t m, int64_t n, double alpha,
                         const double *A, int64_t lda, double *B, int64_t ldb)
{
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; j++) {
        for (int64_t i = 0; i < m; i++) B_(i, j) = alpha * B_(i, j);
        for (int64_t k = m - 1; k >= 0; k--) {
            double xk = unit ? B_(k, j) : B_(k, j) / A_(k, k);
            B_(k, j) = xk;
            for (int64_t i = 0; i < k; i++) B_(i, j) -= A_(i, k) * xk;
        }
    }
}

/* Left, Upper, Trans: A^T is lower, forward substitution, dot form.
 * x_k = (t_k - sum_{i<k} a_ik x_i) / a_kk for k = 0..m-1. */
static void left_upper_t(int unit, int64_t m, int64_t n, double alpha,
                         const double *A, int64_t lda, double *B, int64_t ldb)
{
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; j++) {
        for (int64_t k = 0; k < m; k++) {
            double s = alpha * B_(k, j);
            for (int64_t i = 0; i < k; i++) s -= A_(i, k) * B_(i, j);
            B_(k, j) = unit ? s : s / A_(k, k);
        }
    }
}

/* Right side: row r of X satisfies x_r op(A) = alpha b_r, i.e. for every
 * column c: sum_k x_rk op(A)_kc = alpha b_rc. */

/* Right, Lower, NoTrans: op(A)_kc = a_kc, nonzero for k >= c -> backward in c.
 * x_c = (alpha b_c - sum_{k>c} x_k a_kc) / a_cc. */
static void right_lower_n(int unit, int64_t m, int64_t n, double alpha,
                          const double *A, int64_t lda, double *B, int64_t ldb)
{
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < m; r++) {
        for (int64_t c = n - 1; c >= 0; c--) {
            double s = alpha * B_(r, c);
            for (int64_t k = c + 1; k < n; k++) s -= B_(r, k) * A_(k, c);
            B_(r, c) = unit ? s : s / A_(c, c);
        }
    }
}

/* Right, Lower, Trans: op(A)_kc = a_ck, nonzero for k <= c -> forward in c.
 * x_c = (alpha b_c - sum_{k<c} x_k a_ck) / a_cc. */
static void right_lower_t(int unit, int64_t m, int64_t n, double alpha,
                          const double *A, int64_t lda, double *B, int64_t ldb)
{
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < m; r++) {
        for (int64_t c = 0; c < n; c++) {
            double s = alpha * B_(r, c);
            for (int64_t k = 0; k < c; k++) s -= B_(r, k) * A_(c, k);
            B_(r, c) = unit ? s : s / A_(c, c);
        }
    }
}

/* Right, Upper, NoTrans: op(A)_kc = a_kc, nonzero for k <= c -> forward in c.
 * Column (axpy) form over the row: once x_c is known, subtract x_c a_cj from
 * every later t_j (j > c). */
static void right_upper_n(int unit, int64_t m, int64_t n, double alpha,
                          const double *A, int64_t lda, double *B, int64_t ldb)
{
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < m; r++) {
        for (int64_t c = 0; c < n; c++) B_(r, c) = alpha * B_(r, c);
        for (int64_t c = 0; c < n; c++) {
            double xc = unit ? B_(r, c) : B_(r, c) / A_(c, c);
            B_(r, c) = xc;
            for (int64_t j = c + 1; j < n; j++) B_(r, j) -= xc * A_(c, j);
        }
    }
}

/* Right, Upper, Trans: op(A)_kc = a_ck, nonzero for k >= c -> backward in c.
 * x_c = (alpha b_c - sum_{k>c} x_k a_ck) / a_cc. */
static void right_upper_t(int unit, int64_t m, int64_t n, double alpha,
                          const double *A, int64_t lda, double *B, int64_t ldb)
{
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < m; r++) {
        for (int64_t c = n - 1; c >= 0; c--) {
            double s = alpha * B_(r, c);
            for (int64_t k = c + 1; k < n; k++) s -= B_(r, k) * A_(c, k);
            B_(r, c) = unit ? s : s / A_(c, c);
        }
    }
}

/* side: 0 Left, 1 Right; uplo: 0 Lower, 1 Upper; trans: 0 N, 1 T;
 * diag: 0 NonUnit, 1 Unit.  Returns 0, or -i when argument i is invalid
 * (1-based, in the order of the signature). */
int oracle_dtrsm(int side, int uplo, int trans, int diag, int64_t m, int64_t n,
                 double alpha, const double *A, int64_t lda, double *B,
                 int64_t ldb, int nthreads)
{
    if (side != 0 && side != 1) return -1;
    if (uplo != 0 && uplo != 1) return -2;
    if (trans != 0 && trans != 1) return -3;
    if (diag != 0 && diag != 1) return -4;
    if (m < 0) return -5;
    if (n < 0) return -6;
    int64_t k = side == 0 ? m : n;
    if (lda < (k > 1 ? k : 1)) return -9;
    if (ldb < (m > 1 ? m : 1)) return -11;
    if (m == 0 || n == 0) return 0;
    set_threads(nthreads);
    if (alpha == 0.0) {
        for (int64_t j = 0; j < n; j++)
            for (int64_t i = 0; i < m; i++) B_(i, j) = 0.0;
        return 0;
    }
    int unit = diag == 1;
    if (side == 0) {
        if (uplo == 0) {
            if (trans == 0) left_lower_n(unit, m, n, alpha, A, lda, B, ldb);
            else            left_lower_t(unit, m, n, alpha, A, lda, B, ldb);
        } else {
            if (trans == 0) left_upper_n(unit, m, n, alpha, A, lda, B, ldb);
            else            left_upper_t(unit, m, n, alpha, A, lda, B, ldb);
        }
    } else {
        if (uplo == 0) {
            if (trans == 0) right_lower_n(unit, m, n, alpha, A, lda, B, ldb);
            else            right_lower_t(unit, m, n, alpha, A, lda, B, ldb);
        } else {
            if (trans == 0) right_upper_n(unit, m, n, alpha, A, lda, B, ldb);
            else            right_upper_t(unit, m, n, alpha, A, lda, B, ldb);
        }
    }
    return 0;
}

/* ---- accurate residual ------------------------------------------------ */

/* Error-free transformations: a + b = s + e exactly; a * b = p + e exactly. */
static inline void two_sum(double a, double b, double *s, double *e)
{
    double x = a + b;
    double z = x - a;
    *e = (a - (x - z)) + (b - z);
    *s = x;
}

static inline void two_prod(double a, double b, double *p, double *e)
{
    double x = a * b;
    *e = fma(a, b, -x);
    *p = x;
}

/* Element of op(A) (k x k) at (i, j), honouring uplo/trans/diag and reading
 * only the referenced triangle (0 outside it, 1 on a unit diagonal). */
static inline double op_a(int uplo, int trans, int diag, const double *A,
                          int64_t lda, int64_t i, int64_t j)
{
    int64_t r = trans ? j : i, c = trans ? i : j;  /* element of A itself */
    if (r == c) return diag ? 1.0 : A_(r, c);
    if (uplo == 0 ? (r > c) : (r < c)) return A_(r, c);
    return 0.0;
}

/* R = alpha*B - op(A)*X (side Left) or alpha*B - X*op(A) (side Right),
 * each entry a compensated dot product (Dot2).  X and R are m x n. */
int oracle_dresidual(int side, int uplo, int trans, int diag, int64_t m,
                     int64_t n, double alpha, const double *A, int64_t lda,
                     const double *B, int64_t ldb, const double *X,
                     int64_t ldx, double *R, int64_t ldr, int nthreads)
{
    if (m <= 0 || n <= 0) return 0;
    set_threads(nthreads);
    int64_t kdim = side == 0 ? m : n;
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; j++) {
        for (int64_t i = 0; i < m; i++) {
            double s, c, p, e, t;
            two_prod(alpha, B[(size_t)i + (size_t)j * ldb], &s, &c);
            for (int64_t k = 0; k < kdim; k++) {
                double a, x;
                if (side == 0) {
                    a = op_a(uplo, trans, diag, A, lda, i, k);
                    x = X[(size_t)k + (size_t)j * ldx];
                } else {
                    a = op_a(uplo, trans, diag, A, lda, k, j);
                    x = X[(size_t)i + (size_t)k * ldx];
                }
                if (a == 0.0) continue;
                two_prod(-a, x, &p, &e);
                two_sum(s, p, &s, &t);
                c += t + e;
            }
            R[(size_t)i + (size_t)j * ldr] = s + c;
        }
    }
    return 0;
}

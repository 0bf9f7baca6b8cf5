/*
 * CPU oracle for the Cholesky factorisation.  TEST INFRASTRUCTURE ONLY:
 * nothing on the product path may call, link or execute this file; only the
 * test suite uses it.
 *
 * What it computes: the factorisation the paper names as the next user of
 * its triangular solver (Section VIII, future work: Cholesky and QR on the
 * same TS machinery).  For a symmetric positive definite A (n x n,
 * column-major, leading dimension lda):
 *     uplo = 0 (lower):  A = L L^T, L lower triangular with a positive
 *                        diagonal, written over the lower triangle of A;
 *     uplo = 1 (upper):  A = U^T U, U upper triangular, written over the
 *                        upper triangle.
 * Only the named triangle is read and written.  Definition used, column by
 * column (the Cholesky-Crout order), for the lower case:
 *     l_jj = sqrt(a_jj - sum_{k<j} l_jk^2)
 *     l_ij = (a_ij - sum_{k<j} l_ik l_jk) / l_jj      for i > j,
 * each sum taken in increasing k.  The upper case is written out on its own
 * with u_ji in place of l_ij (the same arithmetic in the same order), so
 * that the transpose identity between the two is a genuine test.
 *
 * Return value (LAPACK ?potrf convention): 0 on success; j + 1 when the
 * quantity under the square root of column j is not positive (or is NaN):
 * the leading minor of order j + 1 is not positive definite and the
 * factorisation stops there (columns >= j are left partly written).
 *
 * Arithmetic: IEEE binary64, -ffp-contract=off, fixed operation order =>
 * bit-reproducible on x86-64 and arm64.  sqrt is the C library's correctly
 * rounded square root.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>

#define A_(i, j) A[(size_t)(i) + (size_t)(j) * (size_t)lda]

static int64_t potrf_lower(int64_t n, double *A, int64_t lda)
{
    for (int64_t j = 0; j < n; j++) {
        double d = A_(j, j);
        for (int64_t k = 0; k < j; k++) d -= A_(j, k) * A_(j, k);
        if (!(d > 0.0)) return j + 1;
        const double ljj = sqrt(d);
        A_(j, j) = ljj;
        for (int64_t i = j + 1; i < n; i++) {
            double s = A_(i, j);
            for (int64_t k = 0; k < j; k++) s -= A_(i, k) * A_(j, k);
            A_(i, j) = s / ljj;
        }
    }
    return 0;
}

static int64_t potrf_upper(int64_t n, double *A, int64_t lda)
{
    for (int64_t j = 0; j < n; j++) {
        double d = A_(j, j);
        for (int64_t k = 0; k < j; k++) d -= A_(k, j) * A_(k, j);
        if (!(d > 0.0)) return j + 1;
        const double ujj = sqrt(d);
        A_(j, j) = ujj;
        for (int64_t i = j + 1; i < n; i++) {
            double s = A_(j, i);
            for (int64_t k = 0; k < j; k++) s -= A_(k, i) * A_(k, j);
            A_(j, i) = s / ujj;
        }
    }
    return 0;
}

/* uplo 0 = lower, 1 = upper.  Returns -1 / -2 / -4 for an invalid uplo / n
 * / lda (LAPACK argument numbering: uplo, n, A, lda), else the info above. */
int64_t oracle_dpotrf(int uplo, int64_t n, double *A, int64_t lda)
{
    if (uplo != 0 && uplo != 1) return -1;
    if (n < 0) return -2;
    if (lda < (n > 1 ? n : 1)) return -4;
    return uplo == 0 ? potrf_lower(n, A, lda) : potrf_upper(n, A, lda);
}

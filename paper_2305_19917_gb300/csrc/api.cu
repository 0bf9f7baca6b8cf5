// C-ABI entry points of the plain FP64/FP32 solve: argument checking,
// canonicalisation of the 16 BLAS forms, plan choice and the kernel-launching
// executor for the decomposition drivers.
#include <cstdio>
#include "common.cuh"
#include "driver.cuh"
#include "plan.cuh"

namespace gb {

static thread_local int tl_last_cuda_error = 0;
void set_cuda_error(cudaError_t e) { tl_last_cuda_error = (int)e; }

namespace {

// Executor that launches the kernels of each task on the canonical view.
template <typename T>
struct LaunchExec {
    const Canon<T> &c;
    int64_t nb;  // plan block size (inner blocking of large TS tasks)
    int status = 0;
    LaunchExec(const Canon<T> &c_, int64_t nb_) : c(c_), nb(nb_) {}
    bool ok() const { return status == 0; }
    void ts(int64_t b0, int64_t nr, T a)
    {
        if (status) return;
        if (nr <= 64) {
            status = launch_diag_solve(c, b0, (int)nr, a);
            return;
        }
        // A TS task larger than the diagonal kernel is itself solved blocked.
        int64_t inner = nb < nr ? nb : 64;
        if (inner > 64 && inner >= nr) inner = 64;
        drive_blocked(*this, b0, b0 + nr, inner, a, c.forward);
    }
    void gemm(int64_t ci0, int64_t M, int64_t ak0, int64_t K, T a)
    {
        if (status) return;
        status = launch_gemm_update(c, ci0, M, ak0, K, a);
    }
};

template <typename T>
int trsm_impl(int side, int uplo, int trans, int diag, int64_t m, int64_t n, T alpha,
              const T *A, int64_t lda, T *B, int64_t ldb, const gb_plan *plan, void *stream)
{
    if (side != GB_LEFT && side != GB_RIGHT) return -1;
    if (uplo != GB_LOWER && uplo != GB_UPPER) return -2;
    if (trans != GB_NOTRANS && trans != GB_TRANS) return -3;
    if (diag != GB_NONUNIT && diag != GB_UNIT) return -4;
    if (m < 0) return -5;
    if (n < 0) return -6;
    const int64_t k = side == GB_LEFT ? m : n;
    const bool empty = (m == 0 || n == 0);
    if (A == nullptr && !empty && alpha != T(0)) return -8;
    if (lda < (k > 1 ? k : 1)) return -9;
    if (B == nullptr && !empty) return -10;
    if (ldb < (m > 1 ? m : 1)) return -11;
    gb_plan p;
    if (plan != nullptr) {
        if (!plan_valid(*plan)) return -12;
        p = *plan;
    }
    if (empty) return 0;

    Canon<T> c;
    c.A = A;
    c.lda = lda;
    c.mt = side == GB_LEFT ? (trans == GB_TRANS) : (trans == GB_NOTRANS);
    c.forward = (uplo == GB_LOWER) != c.mt;
    c.unit = diag == GB_UNIT;
    c.B = B;
    c.ldb = ldb;
    c.left = side == GB_LEFT;
    c.k = k;
    c.ncols = side == GB_LEFT ? n : m;
    c.alpha = alpha;
    c.stream = static_cast<cudaStream_t>(stream);

    if (alpha == T(0)) return launch_zero(c);
    if (plan == nullptr || plan->driver == GB_DRIVER_AUTO)
        p = choose_plan(sizeof(T) == 8 ? GB_DTYPE_F64 : GB_DTYPE_F32, side, uplo, trans, m, n);
    LaunchExec<T> e(c, p.nb);
    drive_plan(e, p.driver, k, p.nb, p.depth, alpha, c.forward);
    return e.status;
}

// Executor that only counts the plan-level tasks.
struct CountExec {
    int64_t n_ts = 0, n_gemm = 0, n_blocks = 0;
    double madds = 0;
    int64_t nb = 1;
    bool ok() const { return true; }
    void ts(int64_t, int64_t, double) { n_ts++; }
    void gemm(int64_t, int64_t M, int64_t, int64_t K, double)
    {
        n_gemm++;
        madds += double(M) * double(K);
        n_blocks += ((M + nb - 1) / nb) * ((K + nb - 1) / nb);
    }
};

}  // namespace
}  // namespace gb

extern "C" {

int gb_dtrsm(int side, int uplo, int trans, int diag, int64_t m, int64_t n, double alpha,
             const double *A, int64_t lda, double *B, int64_t ldb, void *stream)
{
    return gb::trsm_impl<double>(side, uplo, trans, diag, m, n, alpha, A, lda, B, ldb, nullptr, stream);
}

int gb_strsm(int side, int uplo, int trans, int diag, int64_t m, int64_t n, float alpha,
             const float *A, int64_t lda, float *B, int64_t ldb, void *stream)
{
    return gb::trsm_impl<float>(side, uplo, trans, diag, m, n, alpha, A, lda, B, ldb, nullptr, stream);
}

int gb_dtrsm_plan(int side, int uplo, int trans, int diag, int64_t m, int64_t n, double alpha,
                  const double *A, int64_t lda, double *B, int64_t ldb, const gb_plan *plan,
                  void *stream)
{
    return gb::trsm_impl<double>(side, uplo, trans, diag, m, n, alpha, A, lda, B, ldb, plan, stream);
}

int gb_strsm_plan(int side, int uplo, int trans, int diag, int64_t m, int64_t n, float alpha,
                  const float *A, int64_t lda, float *B, int64_t ldb, const gb_plan *plan,
                  void *stream)
{
    return gb::trsm_impl<float>(side, uplo, trans, diag, m, n, alpha, A, lda, B, ldb, plan, stream);
}

int gb_plan_counts(const gb_plan *plan, int64_t k, int64_t *n_diag, int64_t *n_gemm,
                   int64_t *n_offdiag_blocks, double *gemm_madds_per_col)
{
    if (plan == nullptr || !gb::plan_valid(*plan) || plan->driver == GB_DRIVER_AUTO) return -1;
    if (k < 0) return -2;
    gb::CountExec e;
    e.nb = plan->nb;
    gb::drive_plan(e, plan->driver, k, (int64_t)plan->nb, plan->depth, 1.0, true);
    if (n_diag) *n_diag = e.n_ts;
    if (n_gemm) *n_gemm = e.n_gemm;
    if (n_offdiag_blocks) *n_offdiag_blocks = e.n_blocks;
    if (gemm_madds_per_col) *gemm_madds_per_col = e.madds;
    return 0;
}

const char *gb_status_string(int status)
{
    if (status < 0) return "invalid argument (status -i names argument i)";
    switch (status) {
    case GB_STATUS_OK: return "success";
    case GB_STATUS_NOT_CONVERGED: return "iterative refinement did not reach the tolerance";
    case GB_STATUS_CUDA_ERROR: return "CUDA error (see gb_last_cuda_error)";
    case GB_STATUS_TIMEOUT: return "device-side wait exceeded its iteration limit";
    case GB_STATUS_NO_MODEL: return "no cost model loaded";
    case GB_STATUS_SCRATCH_TOO_SMALL: return "problem too large for the fixed no-allocation scratch";
    case GB_STATUS_RANGE: return "operands outside the FP32 range of the low-precision solve";
    default: return "unknown status";
    }
}

int gb_last_cuda_error(void) { return gb::tl_last_cuda_error; }

int gb_version(void) { return 100; }

}  // extern "C"

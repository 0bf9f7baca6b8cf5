// C-ABI entry points of the plain FP64/FP32 solve: argument checking,
// canonicalisation of the 16 BLAS forms, plan choice and the kernel-launching
// executor for the decomposition drivers.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <mutex>
#include "common.cuh"
#include "driver.cuh"
#include "plan.cuh"

namespace gb {

static thread_local int tl_last_cuda_error = 0;
void set_cuda_error(cudaError_t e) { tl_last_cuda_error = (int)e; }

std::atomic<int> g_lookahead{1};

namespace {

std::mutex g_side_mu;
cudaStream_t g_side_stream[64] = {nullptr};

// A library stream per device for the trailing part of split updates.
int side_stream(cudaStream_t *out)
{
    int dev = 0;
    GB_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return GB_STATUS_CUDA_ERROR;
    std::lock_guard<std::mutex> lk(g_side_mu);
    if (!g_side_stream[dev]) GB_CUDA(cudaStreamCreateWithFlags(&g_side_stream[dev], cudaStreamNonBlocking));
    *out = g_side_stream[dev];
    return 0;
}

// Executor that launches the kernels of each task on the canonical view.
//
// Lookahead (the overlap of the diagonal solve with the off-diagonal
// updates that the paper's blocked model aims at, Section V-C, and names as
// future work, Section VIII): a gemm task whose rows extend beyond the next
// diagonal block is split in two.  The head -- the next block's `nb` rows,
// the first ones the schedule needs -- runs on the caller's stream, so the
// next TS task can start at once; the tail -- every other row -- runs on a
// second stream at the same time.  Dependencies: the tail is ordered after
// everything issued on the caller's stream so far (an event: it reads the X
// rows just solved and writes rows those launches may have written), and
// any later launch on the caller's stream that touches rows written by an
// outstanding tail first waits for the latest tail (the tails run in order
// on their stream).  The solve joins the second stream before it returns.
template <typename T>
struct LaunchExec {
    const Canon<T> &c;
    int64_t nb;  // plan block size (inner blocking of large TS tasks)
    int status = 0;
    bool lookahead = false;
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_tail = nullptr;
    int64_t pend_lo = 0, pend_hi = 0;  // rows written by tails not yet waited for
    LaunchExec(const Canon<T> &c_, int64_t nb_) : c(c_), nb(nb_) {}
    ~LaunchExec()
    {
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_tail) cudaEventDestroy(ev_tail);
    }
    bool ok() const { return status == 0; }
    int enable_lookahead()
    {
        GB_TRY(side_stream(&side));
        GB_CUDA(cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming));
        GB_CUDA(cudaEventCreateWithFlags(&ev_tail, cudaEventDisableTiming));
        lookahead = true;
        return 0;
    }
    // Before a launch on the caller's stream that touches rows [r0, r1).
    void settle(int64_t r0, int64_t r1)
    {
        if (status || pend_hi <= pend_lo || r1 <= pend_lo || r0 >= pend_hi) return;
        status = check(cudaStreamWaitEvent(c.stream, ev_tail, 0));
        pend_lo = pend_hi = 0;
    }
    // End of the solve: the caller's stream waits for the last tail.
    int join()
    {
        if (lookahead && !status && pend_hi > pend_lo) status = check(cudaStreamWaitEvent(c.stream, ev_tail, 0));
        pend_lo = pend_hi = 0;
        return status;
    }
    void ts(int64_t b0, int64_t nr, T a)
    {
        if (status) return;
        if (nr <= 64) {
            settle(b0, b0 + nr);
            if (!status) status = launch_diag_solve(c, b0, (int)nr, a);
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
        const int64_t h = nb;  // rows of the next diagonal block
        if (!lookahead || M <= 2 * h) {
            settle(ci0, ci0 + M);
            if (!status) status = launch_gemm_update(c, ci0, M, ak0, K, a);
            return;
        }
        // forward: the next block is at the top of the rows, backward at the bottom
        const int64_t head0 = c.forward ? ci0 : ci0 + M - h;
        const int64_t tail0 = c.forward ? ci0 + h : ci0;
        const int64_t tailM = M - h;
        // the head's rows may still be pending in an older tail
        settle(head0, head0 + h);
        if (status) return;
        // tail on the second stream, after everything issued so far
        if ((status = check(cudaEventRecord(ev_fork, c.stream)))) return;
        if ((status = check(cudaStreamWaitEvent(side, ev_fork, 0)))) return;
        Canon<T> cs = c;
        cs.stream = side;
        if ((status = launch_gemm_update(cs, tail0, tailM, ak0, K, a))) return;
        if ((status = check(cudaEventRecord(ev_tail, side)))) return;
        // the tail covers rows the fork already ordered; any earlier pending
        // tail is ordered before this one on the second stream
        pend_lo = pend_hi > pend_lo ? std::min(pend_lo, tail0) : tail0;
        pend_hi = std::max(pend_hi, tail0 + tailM);
        // head on the caller's stream: disjoint from the new tail's rows, and
        // ordered after any older tail that wrote them (settled above)
        status = launch_gemm_update(c, head0, h, ak0, K, a);
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
    // lookahead where a split update can overlap the next diagonal block:
    // the blocked and recursive models on more than four blocks of rows
    if (g_lookahead.load() && p.driver != GB_DRIVER_ITERATIVE && k > 4 * p.nb)
        GB_TRY(e.enable_lookahead());
    drive_plan(e, p.driver, k, p.nb, p.depth, alpha, c.forward);
    if (e.status) {
        e.join();  // leave no work of this call on the second stream unordered
        return e.status;
    }
    return e.join();
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

int gb_set_lookahead(int on)
{
    const int old = gb::g_lookahead.load();
    if (on == 0 || on == 1) gb::g_lookahead.store(on);
    return old;
}

int gb_version(void) { return 100; }

}  // extern "C"

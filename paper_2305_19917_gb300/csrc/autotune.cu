// Autotuner: measures plans on the GPU with CUDA events.  It is the ground
// truth of the planner (exhaustive search over the standard candidate set)
// and the source of the timings the cost-model network is trained on; it
// replaces the paper's estimation of TS / gemm latencies by compiler
// analysis (Section III) with measurements on the target GPU.
#include <algorithm>
#include <vector>
#include "common.cuh"

namespace gb {
int plan_candidates(int dtype, gb_plan *out, int cap);
}

namespace {

int run_plan(int dtype, int side, int uplo, int trans, int diag, int64_t m, int64_t n, double alpha, const void *A,
             int64_t lda, void *B, int64_t ldb, const gb_plan *p, cudaStream_t s)
{
    if (dtype == 0)
        return gb_dtrsm_plan(side, uplo, trans, diag, m, n, alpha, static_cast<const double *>(A), lda,
                             static_cast<double *>(B), ldb, p, s);
    return gb_strsm_plan(side, uplo, trans, diag, m, n, float(alpha), static_cast<const float *>(A), lda,
                         static_cast<float *>(B), ldb, p, s);
}

}  // namespace

extern "C" {

int gb_autotune_time(int dtype, int side, int uplo, int trans, int diag, int64_t m, int64_t n, double alpha,
                     const void *A, int64_t lda, void *B, int64_t ldb, const gb_plan *plans, int nplans, int reps,
                     double *ms_out, void *stream)
{
    if (dtype != 0 && dtype != 1) return -1;
    if (nplans < 0 || (nplans > 0 && (!plans || !ms_out))) return -14;
    if (reps < 1 || reps > 100) return -16;
    if (m <= 0 || n <= 0 || nplans == 0) return 0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t esz = dtype == 0 ? 8 : 4;
    // B is restored before every run from a copy (the solve overwrites it)
    void *Bsave = nullptr;
    GB_CUDA(cudaMallocAsync(&Bsave, esz * size_t(m) * size_t(n), s));
    int st = gb::check(cudaMemcpy2DAsync(Bsave, esz * m, B, esz * ldb, esz * m, n, cudaMemcpyDeviceToDevice, s));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (!st) st = gb::check(cudaEventCreate(&e0));
    if (!st) st = gb::check(cudaEventCreate(&e1));
    std::vector<float> t(reps);
    for (int p = 0; p < nplans && !st; p++) {
        for (int r = 0; r < reps && !st; r++) {
            st = gb::check(cudaMemcpy2DAsync(B, esz * ldb, Bsave, esz * m, esz * m, n, cudaMemcpyDeviceToDevice, s));
            if (st) break;
            cudaEventRecord(e0, s);
            st = run_plan(dtype, side, uplo, trans, diag, m, n, alpha, A, lda, B, ldb, &plans[p], s);
            cudaEventRecord(e1, s);
            if (!st) st = gb::check(cudaEventSynchronize(e1));
            if (!st) st = gb::check(cudaEventElapsedTime(&t[r], e0, e1));
        }
        if (!st) {
            std::sort(t.begin(), t.end());
            ms_out[p] = t[reps / 2];
        }
    }
    cudaMemcpy2DAsync(B, esz * ldb, Bsave, esz * m, esz * m, n, cudaMemcpyDeviceToDevice, s);
    cudaFreeAsync(Bsave, s);
    cudaStreamSynchronize(s);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return st;
}

int gb_autotune(int dtype, int side, int uplo, int trans, int diag, int64_t m, int64_t n, double alpha, const void *A,
                int64_t lda, void *B, int64_t ldb, gb_plan *best, double *best_ms, void *stream)
{
    if (!best) return -13;
    gb_plan cand[64];
    const int nc = gb::plan_candidates(dtype, cand, 64);
    std::vector<double> ms(nc, 0.0);
    const int st = gb_autotune_time(dtype, side, uplo, trans, diag, m, n, alpha, A, lda, B, ldb, cand, nc, 3,
                                    ms.data(), stream);
    if (st) return st;
    int bi = 0;
    for (int i = 1; i < nc; i++)
        if (ms[i] < ms[bi]) bi = i;
    *best = cand[bi];
    if (best_ms) *best_ms = ms[bi];
    return 0;
}

}  // extern "C"

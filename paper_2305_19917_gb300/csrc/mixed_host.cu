// gb_dtrsm_mixed_host: the mixed-precision solve for operands in host memory.
//
// The library copies in only the referenced triangle of A (in 128-column
// panels, about half of A's bytes), then the right-hand sides on a second
// stream while the kernels that need only A (row exponents, digit slices,
// BF16 copy, diagonal-block inverses) already run; the solution is copied
// back into B.  Device copies come from the library's memory pool.  The
// transfers overlap computation only when the host buffers are page-locked
// (cudaHostAlloc / cudaHostRegister); with pageable buffers the result is
// the same, the copies are just not overlapped.
#include <mutex>
#include "common.cuh"
#include "mixed.cuh"

namespace gb {
namespace {

std::mutex g_cs_mu;
cudaStream_t g_copy_stream[64] = {nullptr};

int copy_stream(cudaStream_t *out)
{
    int dev = 0;
    GB_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return GB_STATUS_CUDA_ERROR;
    std::lock_guard<std::mutex> lk(g_cs_mu);
    if (!g_copy_stream[dev]) GB_CUDA(cudaStreamCreateWithFlags(&g_copy_stream[dev], cudaStreamNonBlocking));
    *out = g_copy_stream[dev];
    return 0;
}

}  // namespace

// Bytes of A that gb_dtrsm_mixed_host copies for an order-k triangle.
int64_t host_a_bytes(int64_t k, int uplo)
{
    int64_t b = 0;
    for (int64_t j0 = 0; j0 < k; j0 += 128) {
        const int64_t w = (k - j0) < 128 ? (k - j0) : 128;
        b += (uplo == GB_LOWER ? (k - j0) : (j0 + w)) * w * 8;
    }
    return b;
}

}  // namespace gb

extern "C" int64_t gb_mixed_host_bytes(int side, int uplo, int64_t m, int64_t n, int64_t *d2h_bytes)
{
    if (m < 0 || n < 0) return -1;
    const int64_t k = side == GB_LEFT ? m : n;
    if (d2h_bytes) *d2h_bytes = m * n * 8;
    return gb::host_a_bytes(k, uplo) + m * n * 8;
}

extern "C" int gb_dtrsm_mixed_host(int side, int uplo, int trans, int diag, int64_t m, int64_t n, double alpha,
                                   const double *A, int64_t lda, double *B, int64_t ldb, double tol, int prec,
                                   int max_iter, int *iters_out, double *est_err_out, void *stream)
{
    if (iters_out) *iters_out = 0;
    if (est_err_out) *est_err_out = 0;
    const int v = gb::mixed_validate(side, uplo, trans, diag, m, n, alpha, A, lda, B, ldb, tol, prec, max_iter);
    if (v) return v;
    if (m == 0 || n == 0) return 0;
    if (alpha == 0.0) {  // B = 0 (A is not read)
        for (int64_t j = 0; j < n; j++)
            for (int64_t i = 0; i < m; i++) B[i + j * ldb] = 0.0;
        return 0;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaStream_t cs = nullptr;
    GB_TRY(gb::copy_stream(&cs));
    const int64_t k = side == GB_LEFT ? m : n;
    cudaMemPool_t pool = gb::mixed_pool();
    if (!pool) return GB_STATUS_CUDA_ERROR;
    const gb::MixedLayout L = gb::mixed_layout(side, m, n, prec);
    const size_t a_bytes = size_t(k) * size_t(k) * 8, b_bytes = size_t(m) * size_t(n) * 8;
    char *mem = nullptr;
    const size_t a_off = (L.total + 255) / 256 * 256, b_off = a_off + (a_bytes + 255) / 256 * 256;
    GB_CUDA(cudaMallocFromPoolAsync(reinterpret_cast<void **>(&mem), b_off + b_bytes, pool, s));
    char *ws = mem;
    double *Ad = reinterpret_cast<double *>(mem + a_off);
    double *Bd = reinterpret_cast<double *>(mem + b_off);
    cudaEvent_t ev_a = nullptr, ev_b = nullptr;
    int st = 0;
    do {
        if ((st = gb::check(cudaEventCreateWithFlags(&ev_a, cudaEventDisableTiming)))) break;
        if ((st = gb::check(cudaEventCreateWithFlags(&ev_b, cudaEventDisableTiming)))) break;
        // the referenced triangle, 128 columns at a time (the rest of Ad is
        // never read: the kernels touch only the referenced triangle)
        for (int64_t j0 = 0; j0 < k && !st; j0 += 128) {
            const int64_t w = (k - j0) < 128 ? (k - j0) : 128;
            const int64_t r0 = uplo == GB_LOWER ? j0 : 0;
            const int64_t rows = uplo == GB_LOWER ? (k - j0) : (j0 + w);
            st = gb::check(cudaMemcpy2DAsync(Ad + r0 + j0 * k, size_t(k) * 8, A + r0 + j0 * lda, size_t(lda) * 8,
                                              size_t(rows) * 8, size_t(w), cudaMemcpyHostToDevice, s));
        }
        if (st) break;
        // B on the copy stream once A is in (the link is then B's alone),
        // while the A-only kernels run on s
        if ((st = gb::check(cudaEventRecord(ev_a, s)))) break;
        if ((st = gb::check(cudaStreamWaitEvent(cs, ev_a, 0)))) break;
        if ((st = gb::check(cudaMemcpy2DAsync(Bd, size_t(m) * 8, B, size_t(ldb) * 8, size_t(m) * 8, size_t(n),
                                              cudaMemcpyHostToDevice, cs))))
            break;
        if ((st = gb::check(cudaEventRecord(ev_b, cs)))) break;
        const int r = gb::mixed_core(side, uplo, trans, diag, m, n, alpha, Ad, k, Bd, m, tol, prec, max_iter,
                                     iters_out, est_err_out, s, ws, nullptr, true, ev_b);
        if (r != 0 && r != GB_STATUS_NOT_CONVERGED) {
            st = r;
            break;
        }
        if ((st = gb::check(cudaMemcpy2DAsync(B, size_t(ldb) * 8, Bd, size_t(m) * 8, size_t(m) * 8, size_t(n),
                                              cudaMemcpyDeviceToHost, s))))
            break;
        if ((st = gb::check(cudaStreamSynchronize(s)))) break;
        st = r;
    } while (0);
    // the copy stream must be done with Bd before the memory goes back
    if (ev_b) cudaStreamWaitEvent(s, ev_b, 0);
    cudaFreeAsync(mem, s);
    if (st == 0 || st == GB_STATUS_NOT_CONVERGED) {
        const int c = gb::check(cudaStreamSynchronize(s));
        if (c) st = c;
    }
    if (ev_a) cudaEventDestroy(ev_a);
    if (ev_b) cudaEventDestroy(ev_b);
    return st;
}

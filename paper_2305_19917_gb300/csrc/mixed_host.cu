// gb_dtrsm_mixed_host: the mixed-precision solve for operands in host memory.
//
// The host link (about 210 GB/s each way on this class of machine, slower
// when both directions run at once) moves A, B and X in about a third of the
// time the solve itself takes, so the transfers are pipelined with the
// computation over column blocks of the right-hand sides, which are
// independent problems:
//
//   link:    A | B_0 | B_1 ...          X_0 ...          X_last
//   kernels:     prep(A) | solve(B_0) | solve(B_1) ... |
//
// Only the referenced triangle of A is copied (in 128-column panels, about
// half of A's bytes); the kernels that need only A run while B_0 arrives;
// block j + 1 arrives while block j is solved, and X_j goes back while block
// j + 1 is solved.  X of every block but the last goes to a separate device
// buffer, so B's original values stay on the device until the end: when a
// later block fails (e.g. GB_STATUS_RANGE), the columns already copied back
// are restored and B is left as it was.  Device memory is the library's
// cached per-device work space (see gb_mixed_workspace_release).  The transfers overlap computation only when the host
// buffers are page-locked (cudaHostAlloc / cudaHostRegister); with pageable
// buffers the result is the same, the copies are just not overlapped.
#include <algorithm>
#include <cstdlib>
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

namespace gb {
namespace {

// Column blocks of the pipelined host solve.  Two halves hide half of B's
// upload and half of X's download under computation; more blocks would hide
// more of the link but make every launch of the low-precision solve narrower
// (its leaf kernel runs one CTA per 128 columns, and a leaf takes as long
// at half the width).  Below about a gigabyte of
// right-hand sides the launches' fixed costs outweigh what the overlap
// saves, so one block is used.  GB_MIXED_HOST_BLOCKS (1..64) overrides the
// choice; the blocks are whole multiples of 128 columns.
int host_blocks(int64_t k, int64_t ncols)
{
    if (const char *e = std::getenv("GB_MIXED_HOST_BLOCKS")) {
        const int v = std::atoi(e);
        if (v >= 1 && v <= 64) return v;
    }
    return (k * ncols >= (int64_t(1) << 27) && ncols >= 8192) ? 2 : 1;
}

// One block of the canonical columns [c0, c0 + w): its place in a
// column-major m x n matrix with leading dimension ld (columns of the matrix
// for side = left, rows for right) and the 2D copy shape (bytes per line,
// lines).
struct BlockSpan {
    int64_t off;    // element offset of the block
    size_t width;   // bytes per line
    size_t height;  // lines
};
BlockSpan block_span(bool left, int64_t m, int64_t n, int64_t ld, int64_t c0, int64_t w)
{
    if (left) return {c0 * ld, size_t(m) * 8, size_t(w)};
    return {c0, size_t(w) * 8, size_t(n)};
}

}  // namespace
}  // namespace gb

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
    const bool left = side == GB_LEFT;
    const int64_t k = left ? m : n;
    const int64_t ncols = left ? n : m;
    const int nb_req = gb::host_blocks(k, ncols);
    // block width: a multiple of 128 canonical columns (the padded width of
    // the work space), the last block possibly narrower
    int64_t cw = (ncols + nb_req - 1) / nb_req;
    cw = std::min<int64_t>(ncols, (cw + 127) / 128 * 128);
    const int nblk = int((ncols + cw - 1) / cw);
    const gb::MixedLayout L = left ? gb::mixed_layout(side, m, cw, prec) : gb::mixed_layout(side, cw, n, prec);
    // device: work space | A | B | X of the blocks before the last
    const int64_t xcols = int64_t(nblk - 1) * cw;
    const int64_t ldx = left ? m : std::max<int64_t>(xcols, 1);
    const size_t a_bytes = size_t(k) * size_t(k) * 8, b_bytes = size_t(m) * size_t(n) * 8;
    const size_t x_bytes = size_t(k) * size_t(xcols) * 8;
    const size_t a_off = (L.total + 255) / 256 * 256, b_off = a_off + (a_bytes + 255) / 256 * 256;
    const size_t x_off = b_off + (b_bytes + 255) / 256 * 256;
    // the device's cached work space (kept between calls, so that the
    // captured low-precision graphs are found again); held until the end
    std::lock_guard<std::recursive_mutex> lk(gb::mixed_device_mutex());
    char *mem = nullptr;
    GB_TRY(gb::mixed_workspace(x_off + x_bytes, s, &mem));
    char *ws = mem;
    double *Ad = reinterpret_cast<double *>(mem + a_off);
    double *Bd = reinterpret_cast<double *>(mem + b_off);
    double *Xd = reinterpret_cast<double *>(mem + x_off);
    cudaEvent_t ev_a = nullptr, ev_b[64] = {nullptr}, ev_x = nullptr, ev_done = nullptr;
    int st = 0, worst = 0, it_max = 0, ndone = 0;
    double est_max = 0;
    do {
        if ((st = gb::check(cudaEventCreateWithFlags(&ev_a, cudaEventDisableTiming)))) break;
        if ((st = gb::check(cudaEventCreateWithFlags(&ev_x, cudaEventDisableTiming)))) break;
        if ((st = gb::check(cudaEventCreateWithFlags(&ev_done, cudaEventDisableTiming)))) break;
        for (int j = 0; j < nblk && !st; j++) st = gb::check(cudaEventCreateWithFlags(&ev_b[j], cudaEventDisableTiming));
        if (st) break;
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
        // the blocks of B on the copy stream once A is in (the link is then
        // B's alone), while the A-only kernels run on s
        if ((st = gb::check(cudaEventRecord(ev_a, s)))) break;
        if ((st = gb::check(cudaStreamWaitEvent(cs, ev_a, 0)))) break;
        for (int j = 0; j < nblk && !st; j++) {
            const int64_t c0 = j * cw, w = std::min(cw, ncols - c0);
            const gb::BlockSpan d = gb::block_span(left, m, n, m, c0, w), h = gb::block_span(left, m, n, ldb, c0, w);
            st = gb::check(cudaMemcpy2DAsync(Bd + d.off, size_t(m) * 8, B + h.off, size_t(ldb) * 8, d.width, d.height,
                                              cudaMemcpyHostToDevice, cs));
            if (!st) st = gb::check(cudaEventRecord(ev_b[j], cs));
        }
        if (st) break;
        if ((st = gb::mixed_prep_a(side, uplo, trans, diag, k, Ad, k, prec, L, ws, s))) break;
        for (int j = 0; j < nblk; j++) {
            const int64_t c0 = j * cw, w = std::min(cw, ncols - c0);
            const bool last = j == nblk - 1;
            const gb::BlockSpan d = gb::block_span(left, m, n, m, c0, w), h = gb::block_span(left, m, n, ldb, c0, w);
            const gb::BlockSpan x = gb::block_span(left, m, n, ldx, c0, w);
            double *out = last ? Bd + d.off : Xd + x.off;
            const int64_t ldo = last ? m : ldx;
            int it = 0;
            double est = 0;
            const int r = gb::mixed_solve_b(side, uplo, trans, k, w, alpha, Bd + d.off, m, out, ldo, tol, prec,
                                            max_iter, &it, &est, s, ws, L, true, ev_b[j], j > 0);
            it_max = std::max(it_max, it);
            est_max = std::max(est_max, est);
            if (r != 0 && r != GB_STATUS_NOT_CONVERGED) {
                st = r;
                break;
            }
            if (r) worst = r;
            // X_j back to the host while the next block is solved
            if ((st = gb::check(cudaEventRecord(ev_x, s)))) break;
            if ((st = gb::check(cudaStreamWaitEvent(cs, ev_x, 0)))) break;
            if ((st = gb::check(cudaMemcpy2DAsync(B + h.off, size_t(ldb) * 8, out, size_t(ldo) * 8, d.width, d.height,
                                                  cudaMemcpyDeviceToHost, cs))))
                break;
            ndone = j + 1;
        }
        if (st) {
            // a block failed after earlier ones went back: restore their
            // columns of B from the device copy of the original values
            if (ndone > 0 && gb::check(cudaStreamSynchronize(cs)) == 0) {
                const gb::BlockSpan d = gb::block_span(left, m, n, m, 0, std::min(ncols, ndone * cw));
                const gb::BlockSpan h = gb::block_span(left, m, n, ldb, 0, std::min(ncols, ndone * cw));
                cudaMemcpy2DAsync(B + h.off, size_t(ldb) * 8, Bd + d.off, size_t(m) * 8, d.width, d.height,
                                  cudaMemcpyDeviceToHost, cs);
            }
            break;
        }
    } while (0);
    if (iters_out) *iters_out = it_max;
    if (est_err_out) *est_err_out = est_max;
    // the copy stream must be done with the device buffers before the work
    // space is used again
    if (ev_done && cudaEventRecord(ev_done, cs) == cudaSuccess) cudaStreamWaitEvent(s, ev_done, 0);
    const int c = gb::check(cudaStreamSynchronize(s));
    if (!st && c) st = c;
    if (ev_a) cudaEventDestroy(ev_a);
    if (ev_x) cudaEventDestroy(ev_x);
    if (ev_done) cudaEventDestroy(ev_done);
    for (int j = 0; j < 64; j++)
        if (ev_b[j]) cudaEventDestroy(ev_b[j]);
    return st ? st : worst;
}

// gb_dtrsm_mixed_noalloc: the mixed-precision solve of gb_dtrsm_mixed for
// callers that must not allocate device memory.
//
// Who cannot allocate: code that runs where cudaMalloc is unavailable or
// unwelcome -- applications whose device memory is owned by another
// allocator (a framework that reserved most of the GPU up front, so that a
// driver allocation fails even though its own pool has room), latency- or
// safety-critical loops that must not call the driver's allocator (it may
// synchronise the device and may fail at run time), and plug-ins that are
// only handed buffers.  This entry point takes its work space (and the
// status word of its bounded waits) from a fixed array that is part of the
// library image instead, and calls no allocating routine.
//
// The scratch array below is a file-scope __device__ object: every GPU that
// loads the library holds its kNoAllocBytes until the process exits.  Host
// code cannot use its name as a device address, so the first call on each
// device (with that device current) looks the address up with
// cudaGetSymbolAddress and keeps it; make that first call before any stream
// capture.  The kept address belongs to the context that was current then:
// calls after cudaDeviceReset are not supported.  All calls share the one
// array and it keeps the last call's contents: everything that must start at
// zero is cleared by each call, and calls that overlap on the GPU (on
// different streams or host threads) race on it -- serialise them.
#include <mutex>
#include "common.cuh"
#include "mixed.cuh"

namespace gb {
namespace {

// 16 MiB: the work space of one solve (the same layout as gb_dtrsm_mixed's,
// status word included).
constexpr size_t kNoAllocBytes = size_t(16) << 20;

static __device__ __align__(256) unsigned char noalloc_scratch[kNoAllocBytes];

std::mutex g_setup_mu;
void *g_scratch_addr[64] = {nullptr};

// Once per device, with that device current: the device address of the
// scratch array.
int scratch_address(char **out)
{
    int dev = 0;
    GB_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return GB_STATUS_CUDA_ERROR;
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        GB_CUDA(cudaGetSymbolAddress(&p, noalloc_scratch));
        g_scratch_addr[dev] = p;
    }
    *out = static_cast<char *>(g_scratch_addr[dev]);
    return 0;
}

}  // namespace
}  // namespace gb

extern "C" int gb_dtrsm_mixed_noalloc(int side, int uplo, int trans, int diag, int64_t m, int64_t n, double alpha,
                                      const double *A, int64_t lda, double *B, int64_t ldb, double tol, int prec,
                                      int max_iter, int *iters_out, double *est_err_out, void *stream)
{
    if (iters_out) *iters_out = 0;
    if (est_err_out) *est_err_out = 0;
    const int v = gb::mixed_validate(side, uplo, trans, diag, m, n, alpha, A, lda, B, ldb, tol, prec, max_iter);
    if (v) return v;
    if (m == 0 || n == 0) return 0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (alpha == 0.0) {  // B = 0 needs no scratch
        gb::Canon<double> c{};
        c.B = B;
        c.ldb = ldb;
        c.left = side == GB_LEFT;
        c.k = side == GB_LEFT ? m : n;
        c.ncols = side == GB_LEFT ? n : m;
        c.stream = s;
        const int st = gb::launch_zero(c);
        if (st) return st;
        return gb::check(cudaStreamSynchronize(s));
    }
    const gb::MixedLayout L = gb::mixed_layout(side, m, n, prec);
    if (L.total > gb::kNoAllocBytes) return GB_STATUS_SCRATCH_TOO_SMALL;
    char *base = nullptr;
    GB_TRY(gb::scratch_address(&base));
    // no graph (capturing and instantiating one allocates); the solve clears
    // and reads its status word itself and returns GB_STATUS_TIMEOUT with B
    // unchanged if a bounded wait gave up
    return gb::mixed_core(side, uplo, trans, diag, m, n, alpha, A, lda, B, ldb, tol, prec, max_iter, iters_out,
                          est_err_out, s, base, false, nullptr);
}

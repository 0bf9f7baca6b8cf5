// Mixed-precision solve: work-space layout and core routine shared by the
// allocating entry point and the no-allocation one (internal header).
#pragma once
#include <mutex>
#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime.h>

namespace gb {

// Byte offsets of the work arrays of one mixed solve (k and the number of
// right-hand sides padded to multiples of 128 as kp, np); `total` bytes.
struct MixedLayout {
    int64_t kp, np;
    size_t o_abf, o_as, o_band, o_binv, o_binv16, o_r, o_t, o_x, o_y, o_ybf, o_zs, o_e, o_f, o_norm, o_dg, o_xm, o_cs;
    size_t o_a8, o_bmax, o_bscale, o_y8, o_sy;  // FP8 variant only (0 otherwise)
    size_t total;
};
MixedLayout mixed_layout(int side, int64_t m, int64_t n, int prec);

// The refinement solve on a caller-provided work space `ws` (layout above,
// 256-byte aligned), with the low-precision solve either replayed from a
// cached CUDA graph (use_graph) or launched directly.  The kernels' bounded
// waits record timeouts in a status word inside the work space, cleared at
// the start of each solve and read back at every refinement step: a timeout
// returns GB_STATUS_TIMEOUT before anything is written to B.  With b_ready,
// the work that reads B waits for that event (the preparation of A does
// not).  Arguments are assumed valid; alpha != 0; m, n > 0.  Synchronous.
int mixed_core(int side, int uplo, int trans, int diag, int64_t m, int64_t n, double alpha, const double *A,
               int64_t lda, double *B, int64_t ldb, double tol, int prec, int max_iter, int *iters_out,
               double *est_err_out, cudaStream_t s, char *ws, bool use_graph, cudaEvent_t b_ready,
               int64_t leaf = 0);
// The two halves of mixed_core, for callers that solve several column blocks
// of one problem against one preparation of A (the work space laid out for
// the widest block, L.np >= every block's ncols):
//  - mixed_prep_a: the work that needs only A (row exponents, digit slices,
//    BF16 copy, diagonal-block inverses);
//  - mixed_solve_b: the refinement solve of one block of ncols right-hand
//    sides read from B (ldb) and written to Bout (ldbo; may be B), given in
//    the user's orientation (columns of B for side = left, rows for right).
//    merge_hist folds this block's refinement history into the previous
//    block's (step-wise maximum) instead of starting a new one.
// leaf: order of the low-precision solve's recursion leaves (a multiple of
// 128; 0 = the form's default, 1024 rows BF16 / 128 rows FP8).
int mixed_prep_a(int side, int uplo, int trans, int diag, int64_t k, const double *A, int64_t lda, int prec,
                 const MixedLayout &L, char *ws, cudaStream_t s);
int mixed_solve_b(int side, int uplo, int trans, int64_t k, int64_t ncols, double alpha, const double *B,
                  int64_t ldb, double *Bout, int64_t ldbo, double tol, int prec, int max_iter, int *iters_out,
                  double *est_err_out, cudaStream_t s, char *ws, const MixedLayout &L, bool use_graph,
                  cudaEvent_t b_ready, bool merge_hist, int64_t leaf = 0);
// The library's stream-ordered memory pool for work space (current device).
cudaMemPool_t mixed_pool();
// Per-device lock of the mixed solves that use cached graphs or the cached
// work space (recursive: held by an entry point around its whole call).
std::recursive_mutex &mixed_device_mutex();
// The cached work space of the current device, at least `bytes` long
// (allocated or regrown from the library's pool on stream s); the caller
// holds mixed_device_mutex() while it uses it.
int mixed_workspace(size_t bytes, cudaStream_t s, char **out);

// Argument checks of gb_dtrsm_mixed (0 or -i).
int mixed_validate(int side, int uplo, int trans, int diag, int64_t m, int64_t n, double alpha, const double *A,
                   int64_t lda, const double *B, int64_t ldb, double tol, int prec, int max_iter);

}  // namespace gb

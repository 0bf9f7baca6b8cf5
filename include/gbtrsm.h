/*
 * gbtrsm -- GB300 (sm_103a) triangular solver with many right-hand sides.
 *
 * The operation is the triangular system solver of arXiv 2305.19917
 * (Section IV: L x = b for a dense lower-triangular L, extended there to n
 * right-hand sides with the same L), exposed with the BLAS ?trsm forms:
 *
 *     side = GB_LEFT :  op(A) * X = alpha * B     A is m x m, B is m x n
 *     side = GB_RIGHT:  X * op(A) = alpha * B     A is n x n, B is m x n
 *
 * op(A) = A (GB_NOTRANS) or A^T (GB_TRANS); A is lower (GB_LOWER) or upper
 * (GB_UPPER) triangular; with GB_UNIT the diagonal is taken as 1 and not
 * read.  Only the triangle named by uplo is read.  X overwrites B.
 *
 * The solve is carried out by the decompositions of Section V: a diagonal
 * block solve (the paper's TS task) plus off-diagonal GEMM updates
 * B2 -= A21 * X1 (the paper's gemm task), arranged as the recursive
 * (Section V-A), iterative (Section V-B) or blocked (Section V-C) model.
 *
 * Conventions common to every entry point
 *   - Matrices are column-major: element (i, j) of A is A[i + j*lda].
 *   - A, B (and every other array unless stated) are DEVICE pointers owned
 *     by the caller; the library never frees them.  Work space the library
 *     needs is taken from the stream-ordered allocator on `stream` and
 *     returned before the call's work completes.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls are asynchronous on that stream unless stated.
 *   - Status codes: 0 = success; -i = argument i (1-based) is invalid,
 *     nothing was launched; GB_STATUS_* below for run-time conditions.
 *   - Quick returns: m == 0 or n == 0 returns 0 and touches nothing.
 *     alpha == 0 sets B to zero and does not read A (BLAS convention).
 *   - A zero on a non-unit diagonal is not checked (BLAS convention): the
 *     result then holds Inf/NaN.
 *   - The device that owns the pointers must be the current device.
 */
#ifndef GBTRSM_H
#define GBTRSM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { GB_LEFT = 0, GB_RIGHT = 1 };
enum { GB_LOWER = 0, GB_UPPER = 1 };
enum { GB_NOTRANS = 0, GB_TRANS = 1 };
enum { GB_NONUNIT = 0, GB_UNIT = 1 };

/* Run-time status codes (positive). */
enum {
    GB_STATUS_OK = 0,
    GB_STATUS_NOT_CONVERGED = 1, /* refinement stopped before reaching tol  */
    GB_STATUS_CUDA_ERROR = 2,    /* a CUDA call failed; see gb_last_cuda_error */
    GB_STATUS_TIMEOUT = 3,       /* a device-side wait hit its iteration cap */
    GB_STATUS_NO_MODEL = 4,      /* no cost model loaded where one is needed */
    GB_STATUS_SCRATCH_TOO_SMALL = 5, /* problem exceeds the fixed scratch of
                                        gb_dtrsm_mixed_noalloc             */
    GB_STATUS_RANGE = 6          /* mixed path: alpha*B, a residual or a
                                    correction left the FP32 range of the
                                    low-precision solve (B is unchanged;
                                    use the FP64 path)                     */
};

/* Decomposition drivers (the paper's three computation models). */
enum {
    GB_DRIVER_BLOCKED = 0,   /* Section V-C: r = ceil(k/nb) diagonal blocks,
                                one trailing GEMM per block column          */
    GB_DRIVER_RECURSIVE = 1, /* Section V-A: halve to `depth` levels (refinement
                                level r = 2^depth), leaves solved blocked    */
    GB_DRIVER_ITERATIVE = 2, /* Section V-B: fixed block size; block row j is
                                updated by one GEMM with all solved blocks
                                0..j-1 (left-looking), then solved           */
    GB_DRIVER_AUTO = -1      /* let the planner choose                       */
};

/* Execution plan for one solve.  nb in {16, 32, 64, 128, 256, 512};
 * depth in 0..12 (recursive driver only). */
typedef struct gb_plan {
    int32_t driver;
    int32_t nb;
    int32_t depth;
    int32_t reserved; /* must be 0 */
} gb_plan;

/*
 * gb_dtrsm / gb_strsm: FP64 / FP32 triangular solve, X overwrites B.
 * Arguments (1-based numbers are the ones a negative status refers to):
 *   1 side, 2 uplo, 3 trans, 4 diag       enum values above
 *   5 m, 6 n                              rows / columns of B (>= 0)
 *   7 alpha                               scalar on B
 *   8 A   device, k x k with k = m (Left) or n (Right); may be NULL only
 *         when alpha == 0 or m*n == 0
 *   9 lda >= max(1, k)
 *  10 B   device, m x n, overwritten by X; may be NULL only when m*n == 0
 *  11 ldb >= max(1, m)
 *  12 stream
 * The plan is picked by the planner (cost model if loaded, else the
 * built-in default).  Asynchronous.
 */
int gb_dtrsm(int side, int uplo, int trans, int diag, int64_t m, int64_t n,
             double alpha, const double *A, int64_t lda, double *B,
             int64_t ldb, void *stream);
int gb_strsm(int side, int uplo, int trans, int diag, int64_t m, int64_t n,
             float alpha, const float *A, int64_t lda, float *B, int64_t ldb,
             void *stream);

/*
 * gb_dtrsm_plan / gb_strsm_plan: as above with an explicit plan
 * (argument 12, host pointer; NULL = planner's choice); stream is argument
 * 13.  A plan with an unknown driver, nb outside the set above, depth out of
 * range or reserved != 0 returns -12.
 */
int gb_dtrsm_plan(int side, int uplo, int trans, int diag, int64_t m,
                  int64_t n, double alpha, const double *A, int64_t lda,
                  double *B, int64_t ldb, const gb_plan *plan, void *stream);
int gb_strsm_plan(int side, int uplo, int trans, int diag, int64_t m,
                  int64_t n, float alpha, const float *A, int64_t lda,
                  float *B, int64_t ldb, const gb_plan *plan, void *stream);

/* Low precision of the mixed-precision solve. */
enum { GB_PREC_BF16 = 0, GB_PREC_FP8 = 1 };

/*
 * gb_dtrsm_mixed: FP64-accurate triangular solve by a low-precision solve
 * plus iterative refinement (X overwrites B, both FP64 as in gb_dtrsm).
 *   X0 = solve in low precision (GEMM updates on the tensor cores in BF16
 *        with FP32 accumulation, FP32 diagonal blocks; recursive model,
 *        Section V-A);
 *   repeat R = alpha*B - op(A)X (split-precision tensor-core products with
 *        exact integer sums, FP64 accumulation), D = low-precision solve of
 *        op(A) D = R, X += D (FP64), until ||D||_F <= tol * ||X||_F.
 * Arguments 1-11 as gb_dtrsm, then
 *  12 tol        >= 0 (e.g. 1e-11 for ~1e-10 forward error)
 *  13 prec       GB_PREC_BF16 (GB_PREC_FP8: see the FP8 entry below)
 *  14 max_iter   1..1000 refinement steps
 *  15 iters_out  host, optional: refinement steps taken
 *  16 est_err_out host, optional: last ||D||_F / ||X||_F
 *  17 stream
 * Returns 0 when converged, GB_STATUS_NOT_CONVERGED (X = last iterate) when
 * max_iter was reached first.  The residual's exact digit sums bound the
 * attainable accuracy near 2^-48 |op(A)||X| (a tol much below 1e-13 is not
 * reached).  Each right-hand side is scaled by an exact power of two (its
 * largest |alpha*B| entry brought near 1) for the low-precision solve and
 * scaled back on output, so the scale of B does not matter; but the scaled
 * solution must stay within the FP32 range of that solve (about 3.4e38 times
 * the column's largest |alpha*B|): beyond it, or with non-finite data, the
 * call returns GB_STATUS_RANGE with B unchanged.
 * The kernels' bounded device waits record a timeout in a status word of
 * the call's own work space, read back at every refinement step: a wait
 * that gave up returns GB_STATUS_TIMEOUT with B unchanged.
 * Synchronous: returns after the solve is complete.  Work space (about
 * 14 k^2 + 42 k n bytes, k and n rounded up to multiples of 128) is a
 * library-owned buffer per device, taken from a stream-ordered pool on first
 * use, kept between calls (so that its address, and the graphs below that
 * name it, stay valid) and regrown when a larger problem needs it;
 * gb_mixed_workspace_release frees it.  The low-precision solve is replayed
 * from a CUDA graph cached per device (the 4 most recently used problem
 * shapes and work spaces); calls on one device from several host threads are
 * serialised.
 */
int gb_dtrsm_mixed(int side, int uplo, int trans, int diag, int64_t m,
                   int64_t n, double alpha, const double *A, int64_t lda,
                   double *B, int64_t ldb, double tol, int prec, int max_iter,
                   int *iters_out, double *est_err_out, void *stream);

/*
 * gb_dtrsm_mixed_leaf: gb_dtrsm_mixed with an explicit plan for its
 * low-precision solve: `leaf` (argument 15, after max_iter; iters_out,
 * est_err_out and stream follow as arguments 16-18) is the order of the
 * recursion's leaves (Section V-A: refinement level ~ k / leaf), a multiple
 * of 128 in [128, 8192], or 0 for the default (1024 rows for BF16, each leaf
 * one tensor-core kernel launch; 128 rows for FP8, larger FP8 leaves are
 * solved blocked in 128-row steps).  Any other value returns -15.  Results
 * and status codes as gb_dtrsm_mixed; the planner's timing sweep uses it.
 */
int gb_dtrsm_mixed_leaf(int side, int uplo, int trans, int diag, int64_t m,
                        int64_t n, double alpha, const double *A, int64_t lda,
                        double *B, int64_t ldb, double tol, int prec,
                        int max_iter, int64_t leaf, int *iters_out,
                        double *est_err_out, void *stream);

/*
 * gb_dtrsm_mixed_noalloc: gb_dtrsm_mixed for callers that cannot allocate
 * device memory (the paper has no counterpart; this is an interface
 * addition).  Same arguments, results and status codes as gb_dtrsm_mixed
 * (GB_STATUS_TIMEOUT included), plus GB_STATUS_SCRATCH_TOO_SMALL; it calls
 * no allocator: its work space and status word are a fixed 16 MiB array
 * inside the library image (held on every GPU that loads the library until
 * the process exits).  That bounds the problem: the padded sizes kp = 128*ceil(k/128),
 * np = 128*ceil(ncols/128) (k = order of A, ncols = right-hand sides) must
 * satisfy roughly 14 kp^2 + 42 kp np + 1550 kp + 20 np + 4 KB <= 16 MiB
 * (e.g. k = ncols = 512); larger problems return GB_STATUS_SCRATCH_TOO_SMALL
 * without touching the GPU.  The first call on a device performs a one-time
 * set-up (it looks up the array's device address and keeps it), so make it
 * before any stream capture; the kept address belongs to that context, so
 * calls after cudaDeviceReset are not supported.  Calls share the array:
 * calls that overlap on the GPU race and must be serialised by the caller.
 * Synchronous, like gb_dtrsm_mixed.
 */
int gb_dtrsm_mixed_noalloc(int side, int uplo, int trans, int diag,
                           int64_t m, int64_t n, double alpha,
                           const double *A, int64_t lda, double *B,
                           int64_t ldb, double tol, int prec, int max_iter,
                           int *iters_out, double *est_err_out, void *stream);

/*
 * gb_dtrsm_mixed_host: gb_dtrsm_mixed with A and B in HOST memory (an
 * interface addition).  Same arguments, results and status codes, except
 * that A (8) and B (10) are host pointers; X overwrites B on the host.  The
 * library copies in only the referenced triangle of A (128-column panels),
 * then the right-hand sides in column blocks (columns of B for side = left,
 * rows for right) on a second stream while the kernels that need only A
 * run; it solves block j on `stream` while block j+1 arrives and block
 * j-1's X goes back.  It uses two blocks once the right-hand sides reach
 * about a gigabyte, else one; the environment variable GB_MIXED_HOST_BLOCKS
 * (1..64) overrides the count.  Blocks are independent problems, so a
 * block's refinement stops on its own criterion; iters_out and est_err_out
 * report the largest over the blocks.  On an error in a later block the
 * columns already copied back are restored: B is unchanged, as for
 * gb_dtrsm_mixed.  Device buffers (work space, A, B and the X blocks) are
 * the library's cached per-device work space of gb_dtrsm_mixed, grown to
 * fit.  For the copies to overlap with
 * computation, A and B should be page-locked (cudaHostAlloc or
 * cudaHostRegister); pageable memory gives the same result, slower.
 * alpha == 0 sets B = 0 on the host without reading A.  Synchronous.
 */
int gb_dtrsm_mixed_host(int side, int uplo, int trans, int diag,
                        int64_t m, int64_t n, double alpha,
                        const double *A, int64_t lda, double *B,
                        int64_t ldb, double tol, int prec, int max_iter,
                        int *iters_out, double *est_err_out, void *stream);

/*
 * gb_mixed_host_bytes: the bytes gb_dtrsm_mixed_host copies host -> device
 * (return value: A's referenced triangle in 128-column panels plus B) and,
 * in *d2h_bytes (may be NULL), device -> host (X), for the given side, uplo
 * and sizes.  Host-only; -1 for negative sizes.
 */
int64_t gb_mixed_host_bytes(int side, int uplo, int64_t m, int64_t n, int64_t *d2h_bytes);

/*
 * gb_set_lookahead: switch the plain solves' lookahead on (1, the default)
 * or off (0) for the whole process; any other value only queries.  With it,
 * an off-diagonal update whose rows extend beyond the next diagonal block is
 * split: the next block's rows are updated first on the caller's stream, so
 * that block's TS task starts at once, while the other rows are updated on a
 * library stream at the same time (the overlap of diagonal solves and
 * updates of Sections V-C and VIII); the solve joins that stream before it
 * returns, so results and stream semantics are unchanged.  Used by the
 * blocked and recursive models when the order exceeds four blocks.  Returns
 * the previous setting.  Host only.
 */
int gb_set_lookahead(int on);

/*
 * gb_gemm_update: the plain path's gemm task on its own (Section IV stage 2,
 * b.low -= L.mid x.up, with many right-hand sides): C = alpha*C - A*B with
 * A (M x K, lda), B (K x N, ldb) and C (M x N, ldc) column-major device
 * arrays of FP64 (dtype 0) or FP32 (dtype 1), alpha converted to the dtype;
 * DFMA / FFMA register-blocked kernel, asynchronous on `stream`.  The
 * planner's analytic model times it (gemm(j) of Section V).  Returns 0, -1
 * for a bad dtype, -2..-4 for negative M, N, K, -5 / -7 / -9 for a NULL
 * operand that is needed, -6 / -8 / -10 for a leading dimension below its
 * operand's row count, or GB_STATUS_CUDA_ERROR.
 */
int gb_gemm_update(int dtype, int64_t M, int64_t N, int64_t K, const void *A,
                   int64_t lda, const void *B, int64_t ldb, void *C,
                   int64_t ldc, double alpha, void *stream);

/*
 * gb_dpotrf / gb_spotrf: Cholesky factorisation on this library's
 * triangular solve -- the use the paper names for its TS machinery (Section
 * VIII, future work), with the recursive computation model of Section V-A:
 * split A's order in two (first part a multiple of 64), factorise the first
 * diagonal block, solve the off-diagonal panel against it with gb_dtrsm /
 * gb_strsm (side Right, Lower, transposed: L21 = A21 L11^-T; or side Left,
 * Upper, transposed: U12 = U11^-T A12), update the trailing block by a SYRK
 * (A22 -= L21 L21^T, or U12^T U12; its triangle only), recurse; leaves of at
 * most 64 columns are factorised by one CTA in shared memory.
 *   1 uplo   GB_LOWER: A = L L^T, L over the lower triangle;
 *            GB_UPPER: A = U^T U, U over the upper triangle
 *   2 n      order of A, >= 0
 *   3 A      device, column-major n x n, symmetric positive definite; only
 *            the named triangle is read and overwritten (the other is not
 *            touched)
 *   4 lda    >= max(1, n)
 *   5 info   host, out: 0 on success, or j (1-based) when the leading
 *            minor of order j is not positive definite (a pivot <= 0 or
 *            NaN; the LAPACK ?potrf convention).  With info > 0 the
 *            factorisation stopped: columns from j on are undefined.
 *   6 stream
 * Returns 0 (then see *info), -i for invalid argument i, or
 * GB_STATUS_CUDA_ERROR.  Synchronous (it reads info); a 4-byte device word
 * for info comes from the library's stream-ordered pool.  Accuracy (FP64):
 * ||A - L L^T|| / ||A|| is a small multiple of n 2^-53.
 */
int gb_dpotrf(int uplo, int64_t n, double *A, int64_t lda, int64_t *info, void *stream);
int gb_spotrf(int uplo, int64_t n, float *A, int64_t lda, int64_t *info, void *stream);

/*
 * gb_mixed_workspace_release: frees the cached work space of gb_dtrsm_mixed
 * and gb_dtrsm_mixed_host on the current device, after `stream` is idle (the
 * next call allocates it again; the cached graphs that name it are then not
 * replayed unless the new buffer lands at the same address with the same
 * layout).  Returns 0 or GB_STATUS_CUDA_ERROR.
 */
int gb_mixed_workspace_release(void *stream);

/*
 * gb_mixed_history: refinement history of the last gb_dtrsm_mixed call made
 * by this host thread.  Writes up to `cap` entries: rho[t] = ||D||_F/||X||_F
 * of correction t+1 and levels[t] = 10 P + P2 for the residual preceding
 * that correction (it formed A digit slices 1..P with the first correction
 * digit and 1..P2 also with the second; either pointer may be NULL).
 * Returns the number of corrections recorded.  Host only.
 */
int gb_mixed_history(double *rho, int *levels, int cap);

/*
 * Batched uneven solves (many independent problems of different order and
 * width, each "n instances of TS" as in Section IV) in one persistent kernel
 * launch driven by a device-side work queue, replayed from a CUDA graph.
 *
 * gb_trsm_batched(dtype, count, side[], uplo[], trans[], diag[], m[], n[],
 *                 alpha[], A[], lda[], B[], ldb[], stream)
 *   1 dtype   0 = FP64 (double), 1 = FP32 (float)
 *   2 count   number of problems (>= 0)
 *   3..13     HOST arrays of `count` entries: the gb_dtrsm arguments of
 *             each problem; alpha[] holds doubles (dtype 0) or floats
 *             (dtype 1); A[i] and B[i] are DEVICE pointers (column-major),
 *             B[i] overwritten by X_i
 *  14 stream
 * A negative status -a names the argument a whose entry is invalid (or
 * whose array is NULL).  Problems of order (m for Left, n for Right) up to
 * 512 are solved in shared memory by the persistent kernel, in chunks of 16
 * (FP64) or 32 (FP32) right-hand sides (the default tile; see
 * gb_batched_plan_create_tiled), largest first; larger problems are
 * solved one after the other by the regular driver on the same stream.
 * Synchronous (returns after the solves completed).
 *
 * gb_batched_plan_create(... same 1-14 ..., void **plan_out) builds the work
 * queue once (device descriptor array, CUDA graph) for the given pointers;
 * gb_batched_plan_run(plan, stream) replays it (asynchronous; the pointed-to
 * data may change between runs, the pointers and sizes may not);
 * gb_batched_plan_destroy(plan) frees it; gb_batched_plan_info reports the
 * number of work units, the persistent grid size, the number of problems
 * handled by the regular driver and the algorithmic flops (sum of k^2 ncols).
 */
int gb_trsm_batched(int dtype, int64_t count, const int8_t *side,
                    const int8_t *uplo, const int8_t *trans,
                    const int8_t *diag, const int64_t *m, const int64_t *n,
                    const void *alpha, const void *const *A,
                    const int64_t *lda, void *const *B, const int64_t *ldb,
                    void *stream);
int gb_batched_plan_create(int dtype, int64_t count, const int8_t *side,
                           const int8_t *uplo, const int8_t *trans,
                           const int8_t *diag, const int64_t *m,
                           const int64_t *n, const void *alpha,
                           const void *const *A, const int64_t *lda,
                           void *const *B, const int64_t *ldb, void *stream,
                           void **plan_out);
/*
 * gb_batched_plan_create_tiled: as gb_batched_plan_create with the tile
 * shape of the kernel's gemm tasks as argument 14 (stream 15, plan_out 16):
 * tile = rows of a 32-row block row per thread, 1 (units of 16 FP64 / 32
 * FP32 right-hand sides, several CTAs per SM) or 2 (units of 32 / 64
 * right-hand sides, twice the multiply-adds per shared-memory load, one CTA
 * per SM); 0 = 1.  Any other value returns -15; a NULL plan_out -17.
 * gb_batched_plan_create is this with tile 1.
 * gb_batched_plan_tile(plan): the plan's tile (or -1 for NULL).
 *
 * gb_batched_autotune(... 1-13 as gb_trsm_batched ..., int reps, stream,
 *   int *tile_out, double *ms_out): the autotuner of the batched kernel's
 *   tile shape: builds a plan with each tile, times `reps` replays of each
 *   (after one warm-up; CUDA events, median) with every B restored from a
 *   device copy before each replay, and returns the fastest tile in
 *   *tile_out and the two medians in ms_out[0..1] (optional).  B is left as
 *   it was.  Synchronous; its copy of the B's comes from the stream-ordered
 *   allocator.  Returns 0, -14 for reps outside 1..100, -16 for a NULL
 *   tile_out, or a plan-creation / CUDA status.
 */
int gb_batched_plan_create_tiled(int dtype, int64_t count, const int8_t *side,
                                 const int8_t *uplo, const int8_t *trans,
                                 const int8_t *diag, const int64_t *m,
                                 const int64_t *n, const void *alpha,
                                 const void *const *A, const int64_t *lda,
                                 void *const *B, const int64_t *ldb, int tile,
                                 void *stream, void **plan_out);
int gb_batched_plan_tile(const void *plan);
int gb_batched_autotune(int dtype, int64_t count, const int8_t *side,
                        const int8_t *uplo, const int8_t *trans,
                        const int8_t *diag, const int64_t *m, const int64_t *n,
                        const void *alpha, const void *const *A,
                        const int64_t *lda, void *const *B, const int64_t *ldb,
                        int reps, void *stream, int *tile_out, double *ms_out);
int gb_batched_plan_run(void *plan, void *stream);
int gb_batched_plan_destroy(void *plan);
int gb_batched_plan_info(const void *plan, int64_t *units, int *grid,
                         int64_t *large_instances, double *flops);

/*
 * Planner, autotuner and cost model (the paper's analytical performance
 * models of Section V -- Comp(i) and the refinement stop rule -- replaced by
 * timings measured on the GPU and a network trained on them).
 *
 * gb_plan_candidates(dtype, out, cap): the standard candidate set (blocked
 *   and iterative with nb in {16..512}, recursive with nb in {16..512} and
 *   depth 1..6); writes up to cap plans, returns the set size (48).
 * gb_plan_features(dtype, side, uplo, trans, m, n, plan, features): the
 *   17 network inputs of (shape, plan): log2 m / 16, log2 n / 16, one-hots of
 *   side, uplo, trans and dtype (0 FP64, 1 FP32, 2 BF16-mixed, 3 FP8-mixed),
 *   log2 nb / 9, depth / 6, one-hot driver.  Returns 17.  Host only.
 * gb_plan_set_model(path): load a trained network ("GBMLP001" file: magic,
 *   int32 in_dim = 17, int32 hidden = 64, int32 parameter count, float mean
 *   and scale of the log-time target, then the parameters); NULL unloads.
 *   Returns 0 or -1 (unreadable / malformed).  While loaded, the planner of
 *   gb_dtrsm / gb_strsm picks the predicted-fastest candidate; the first
 *   call for a new shape runs one inference launch and waits for it.
 * gb_plan_choose(dtype, side, uplo, trans, m, n, plan_out, predicted_ms):
 *   the model's choice (GB_STATUS_NO_MODEL and the built-in default when no
 *   model is loaded).
 * gb_autotune_time(dtype, side, uplo, trans, diag, m, n, alpha, A, lda, B,
 *   ldb, plans, nplans, reps, ms_out, stream): median of `reps` CUDA-event
 *   timings of each plan on the caller's buffers (dtype 0 FP64 / 1 FP32);
 *   B is restored to its input values afterwards.  Synchronous.
 * gb_autotune(..., best, best_ms, stream): exhaustive search over the
 *   candidate set (3 repetitions each), the fastest plan and its time.
 */
int gb_plan_candidates(int dtype, gb_plan *out, int cap);
int gb_plan_features(int dtype, int side, int uplo, int trans, int64_t m,
                     int64_t n, const gb_plan *plan, float *features);
int gb_plan_set_model(const char *path);
int gb_plan_choose(int dtype, int side, int uplo, int trans, int64_t m,
                   int64_t n, gb_plan *plan_out, double *predicted_ms);

/*
 * gb_plan_mixed_candidates: the mixed-precision candidates of the precision
 * decision for an order-k triangle (host only): (prec[i], leaf[i]) for
 * i < 5 -- BF16 with leaves of 512, 1024, 2048 rows, FP8 with 128 and 512 --
 * and plans[i], their encoding for the cost model (driver recursive, nb =
 * leaf, depth = log2(kp / leaf) clamped to 0..6, kp = k rounded up to 128).
 * Any output may be NULL; at most `cap` entries are written.  Returns 5, or
 * -1 for k < 0, -5 for cap < 0.
 *
 * gb_plan_choose_precision: the planner's answer for a solve to FP64-level
 * accuracy: the plain FP64 path with the network's best plan, or one of the
 * mixed candidates above (gb_dtrsm_mixed_leaf with that precision and
 * leaf), whichever the loaded network predicts fastest.  *prec_out = -1
 * (plain FP64), GB_PREC_BF16 or GB_PREC_FP8; *leaf_out = the leaf (0 for
 * plain); plan_out (optional) = the plain plan or the candidate's encoding;
 * predicted_ms (optional).  Arguments 1-5 as gb_plan_choose's 2-6; returns 0,
 * -i for invalid argument i (-6: prec_out or leaf_out NULL), or
 * GB_STATUS_NO_MODEL (then plain FP64 with the built-in default plan).
 */
int gb_plan_mixed_candidates(int64_t k, int *prec, int64_t *leaf, gb_plan *plans, int cap);
int gb_plan_choose_precision(int side, int uplo, int trans, int64_t m, int64_t n, int *prec_out,
                             int64_t *leaf_out, gb_plan *plan_out, double *predicted_ms);
int gb_autotune_time(int dtype, int side, int uplo, int trans, int diag,
                     int64_t m, int64_t n, double alpha, const void *A,
                     int64_t lda, void *B, int64_t ldb, const gb_plan *plans,
                     int nplans, int reps, double *ms_out, void *stream);
int gb_autotune(int dtype, int side, int uplo, int trans, int diag, int64_t m,
                int64_t n, double alpha, const void *A, int64_t lda, void *B,
                int64_t ldb, gb_plan *best, double *best_ms, void *stream);

/*
 * Cost-model network kernels (FP32, 3 hidden layers of 64, GELU), on device
 * arrays; `in_dim` = D inputs per sample (1..64), parameters laid out as
 * W1[64][D], b1[64], W2[64][64], b2[64], W3[64][64], b3[64], w4[64], b4.
 * gb_mlp_param_count(D): number of parameters (-1 if D < 1).
 * gb_mlp_forward(params, D, X[n][D], n, Y[n], Z, stream): predictions; when
 *   Z != NULL also the pre-activations Z[n][3][64] needed by the backward.
 * gb_mlp_backward(params, D, X, Z, dY[n], n, grads, stream): ADDS the
 *   gradient of sum_s dY[s] y_s to grads (zero it first).
 * gb_mlp_loss(Y, T, n, dY, loss, stream): mean squared error; writes
 *   dY = 2 (Y - T) / n and adds the loss to *loss (device scalar, may be
 *   NULL).
 * gb_mlp_adam(params, grads, m, v, np, lr, beta1, beta2, eps, step, stream):
 *   one Adam step with bias correction (step >= 1).
 * All asynchronous; negative status = invalid argument.
 */
int64_t gb_mlp_param_count(int in_dim);
int gb_mlp_forward(const float *params, int in_dim, const float *X, int64_t n,
                   float *Y, float *Z, void *stream);
int gb_mlp_backward(const float *params, int in_dim, const float *X,
                    const float *Z, const float *dY, int64_t n, float *grads,
                    void *stream);
int gb_mlp_loss(const float *Y, const float *T, int64_t n, float *dY,
                float *loss, void *stream);
int gb_mlp_adam(float *params, const float *grads, float *m, float *v,
                int64_t np, float lr, float beta1, float beta2, float eps,
                int step, void *stream);

/*
 * gb_plan_counts: host-only description of the launches a plan issues for a
 * triangle of order k (no GPU work).  Writes the number of diagonal-block
 * solves and of GEMM updates, and the sum over GEMMs of M*N*K / ncols (i.e.
 * the GEMM multiply-adds per right-hand side).  This exposes the task counts
 * of the paper's Section V models: 2^j GEMMs at recursion level j
 * (Section V-A), r(r-1)/2 off-diagonal blocks for r diagonal blocks
 * (Section V-C; r - 1 launches, one per block column).
 * Returns 0, or -1 for an invalid plan, -2 for k < 0.
 */
int gb_plan_counts(const gb_plan *plan, int64_t k, int64_t *n_diag,
                   int64_t *n_gemm, int64_t *n_offdiag_blocks,
                   double *gemm_madds_per_col);

/*
 * Launch accounting (host only, no GPU work).
 * gb_kernel_launches: number of kernels this library has launched in the
 * process so far.
 * gb_profile_enable(on): clear the per-launch records; while on, every
 * launch is bracketed by CUDA events on its stream.
 * gb_profile_read(kind, ...): for kernel kind 0 diagonal solve, 1 CUDA-core
 * GEMM update, 2 tensor-core GEMM update, 3 split residual, 4 conversion /
 * elementwise, 5 batched solve, 6 cost-model network: the number of
 * recorded launches, their summed device time in ms and their summed
 * algorithmic flops and bytes.  Waits for the recorded events.  Returns 0,
 * -1 for an unknown kind, GB_STATUS_CUDA_ERROR if an event failed.
 */
uint64_t gb_kernel_launches(void);
int gb_profile_enable(int on);
int gb_profile_read(int kind, int64_t *launches, double *ms, double *flops,
                    double *bytes);

/*
 * gb_bf16_gemm_update: the tensor-core gemm task of the mixed-precision
 * path (Section IV stage 2, b.low -= L.mid x.up, with many right-hand
 * sides), exposed for testing and reuse:
 *     C = alpha * C - A * B
 *   1 M, 2 N, 3 K       sizes; K must be a multiple of 64 (K == 0: no-op)
 *   4 A   device BF16, M x K row-major (element (i,k) at A[i*lda + k]),
 *         16-byte aligned
 *   5 lda >= max(K, 8), multiple of 8
 *   6 B   device BF16, K x N column-major (element (k,j) at B[k + j*ldb]),
 *         16-byte aligned
 *   7 ldb >= max(K, 8), multiple of 8
 *   8 C   device FP32, M x N column-major
 *   9 ldc >= max(1, M)
 *  10 alpha, 11 stream
 * Products are exact, sums accumulate in FP32 (tcgen05, tensor memory).
 * Asynchronous.  A device-side wait that times out is reported by
 * gb_device_status().
 */
int gb_bf16_gemm_update(int64_t M, int64_t N, int64_t K, const void *A,
                        int64_t lda, const void *B, int64_t ldb, float *C,
                        int64_t ldc, float alpha, void *stream);

/*
 * gb_device_status: synchronises with the current device and returns the
 * library's device-side status word (0 = no error, GB_STATUS_TIMEOUT-class
 * codes 1..3 = a bounded wait of a tensor-core kernel expired); clears it
 * when `clear` is nonzero.  Returns GB_STATUS_CUDA_ERROR if it cannot read.
 */
int gb_device_status(int clear);

/* Message for a status code (static storage). */
const char *gb_status_string(int status);
/* Last CUDA error code seen by the library on this host thread (0 = none). */
int gb_last_cuda_error(void);
/* Library version as major*10000 + minor*100 + patch. */
int gb_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GBTRSM_H */

// Shared definitions of the gbtrsm CUDA library (internal header).
#pragma once
#include <atomic>
#include <cuda_runtime.h>
#include <stdint.h>
#include "../../include/gbtrsm.h"

namespace gb {

// Per-thread record of the last CUDA error the library saw.
void set_cuda_error(cudaError_t e);

// Returns GB_STATUS_CUDA_ERROR (and records it) if e != cudaSuccess.
inline int check(cudaError_t e)
{
    if (e != cudaSuccess) {
        set_cuda_error(e);
        return GB_STATUS_CUDA_ERROR;
    }
    return 0;
}

#define GB_TRY(expr)                 \
    do {                             \
        int _st = (expr);            \
        if (_st != 0) return _st;    \
    } while (0)

#define GB_CUDA(expr) GB_TRY(::gb::check(expr))

// One-time set-up flag per device.  Kernel attributes such as the dynamic
// shared-memory limit belong to a device (its context): a process that
// drives several GPUs must set them on each, so the flag is kept per device
// (a static PerDeviceOnce starts all-clear).
struct PerDeviceOnce {
    std::atomic<int> done[64];
};
// Raise `kernel`'s dynamic shared-memory limit to `bytes` on the current
// device, once per device (repeating it when two threads race is harmless).
template <typename K>
inline int smem_attr_once(PerDeviceOnce &once, K *kernel, size_t bytes)
{
    int dev = 0;
    GB_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return GB_STATUS_CUDA_ERROR;
    if (!once.done[dev].load(std::memory_order_acquire)) {
        GB_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
        once.done[dev].store(1, std::memory_order_release);
    }
    return 0;
}

// Launch with programmatic stream serialisation: the kernel may start while
// the previous kernel of the stream is finishing (it must execute
// griddepcontrol.wait before touching that kernel's data, and it lets the
// next kernel do the same by executing griddepcontrol.launch_dependents).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<Args &&>(args)...);
}

// Canonical ("left view") form of a triangular solve.
//
// Every BLAS form is reduced to   Mv * Xv = alpha * Bv   where Mv is a k x k
// triangular matrix and Bv is k x ncols:
//   Left :  Mv = op(A),    Bv = B   (k = m, ncols = n, Bv column-major)
//   Right:  Mv = op(A)^T,  Bv = B^T (k = n, ncols = m, Bv row-major)
// Mv(i, j) is A(i, j) or A(j, i); `mt` says which.  Mv lower => forward
// substitution, upper => backward.
template <typename T>
struct Canon {
    const T *A;      // base of A
    int64_t lda;
    bool mt;         // Mv(i,j) = A(j,i) when true, A(i,j) when false
    bool forward;    // Mv lower triangular
    bool unit;       // unit diagonal
    T *B;            // base of B
    int64_t ldb;
    bool left;       // Bv column-major (Left) or row-major (Right)
    int64_t k;       // order of Mv
    int64_t ncols;   // columns of Bv
    T alpha;
    cudaStream_t stream;
};

// Pointer to Mv(i, j).
template <typename T>
__host__ __device__ inline const T *mv_ptr(const Canon<T> &c, int64_t i, int64_t j)
{
    return c.mt ? c.A + j + i * c.lda : c.A + i + j * c.lda;
}
// Pointer to Bv(i, j).
template <typename T>
__host__ __device__ inline T *bv_ptr(const Canon<T> &c, int64_t i, int64_t j)
{
    return c.left ? c.B + i + j * c.ldb : c.B + j + i * c.ldb;
}

// ---- launch accounting and optional per-launch event timing (prof.cu) ------
enum KernelKind {
    KK_DIAG = 0,      // diagonal-block solve
    KK_GEMM_SIMT = 1, // CUDA-core GEMM update (FP64 DFMA / FP32 FFMA)
    KK_GEMM_TC = 2,   // tensor-core (tcgen05) GEMM update
    KK_RESIDUAL = 3,  // split-precision residual
    KK_CONVERT = 4,   // precision conversion / slicing / elementwise
    KK_BATCHED = 5,   // persistent batched solve
    KK_MLP = 6,       // cost-model network
    KK_GRAPH = 7,     // a CUDA-graph launch (e.g. a captured low-precision solve)
    KK_COUNT = 8
};
// Every kernel launch of the library is wrapped in a LaunchScope: it counts
// the launch and, while profiling is enabled, brackets it with CUDA events on
// the launching stream and records its algorithmic flops and bytes.
// Launches issued while `s` is being captured into a CUDA graph are counted
// into a per-thread capture counter instead (capture_count()), and the
// graph launch later adds that many kernels (nkernels).
struct LaunchScope {
    int kind;
    int slot;
    cudaStream_t stream;
    LaunchScope(int kind, cudaStream_t s, double flops, double bytes, uint64_t nkernels = 1);
    ~LaunchScope();
};
uint64_t &capture_count();

// ---- kernel launchers (defined in the .cu files) -------------------------

// Solve Mv[r0:r0+nr, r0:r0+nr] * X = alpha * Bv[r0:r0+nr, :] in place,
// nr <= 64.
template <typename T>
int launch_diag_solve(const Canon<T> &c, int64_t r0, int nr, T alpha);

// C = alpha*C - Aop * Bop on the canonical view:
//   C   = Bv[ci0 : ci0+M, :]            (M x ncols)
//   Aop = Mv[ci0 : ci0+M, ak0 : ak0+K]  (M x K)
//   Bop = Bv[ak0 : ak0+K, :]            (K x ncols)
template <typename T>
int launch_gemm_update(const Canon<T> &c, int64_t ci0, int64_t M, int64_t ak0,
                       int64_t K, T alpha);

// Bv = 0 (alpha == 0 quick path).
template <typename T>
int launch_zero(const Canon<T> &c);

}  // namespace gb

// (internal header) Diagonal-block triangular solve: the paper's TS task (Section IV, stages 1
// and 3; the white triangles of Figs. 2-4), for one nr x nr block with
// nr <= 64 and all right-hand sides of the canonical view.
//
// Design (GB300): a CTA solves 64 right-hand sides with 8 warps; warp w
// handles 32 of them (column group w / 4) and the rows i = w % 4 (mod 4) of
// the block, in registers, by column-oriented substitution: at step k the
// warp owning row k forms x_k = t_k / a_kk, publishes it in shared memory
// (a named barrier per column group), and the four warps update their own
// rows.  Splitting each right-hand side's rows over four warps matters on
// this GPU: a warp runs on one SM sub-partition, whose FP64 unit takes about
// 64 clocks per warp instruction (a quarter of the SM's 1.9 DFMA per clock),
// so one warp per column would leave three quarters of the FP64 throughput
// idle and make the serial chain four times longer.  The triangle sits in
// shared memory (broadcast reads), the B panel is staged through shared
// memory with asynchronous copies so that global loads and stores are
// coalesced whichever way B is laid out, and the diagonal is inverted once
// per CTA (nr^2/2 multiply-adds per right-hand side).
#pragma once
#include <cuda_bf16.h>
#include "common.cuh"

namespace gb {
namespace {

// Threads per CTA (8 warps: 2 column groups x 4 row groups); a CTA solves
// CW = 64 right-hand sides.
constexpr int kDiagThreads = 256;

// Asynchronous copy of one 4- or 8-byte element into shared memory; `in`
// false writes zero (the source is not read).
template <typename T>
__device__ __forceinline__ void diag_cp_async(T *dst, const T *src, bool in)
{
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
    const int n = in ? int(sizeof(T)) : 0;
    if (sizeof(T) == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(n) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(n) : "memory");
}

// Shared-memory layout (dynamic):
//   L  [NB][NB]   column form (MT=false): L[k*NB + i] = Mv(i,k)
//                 row form    (MT=true) : L[i*NB + k] = Mv(i,k)
//   inv[NB]       1 / Mv(i,i)  (1 for a unit diagonal or padding rows)
//   Bs [NB][CW + 1]
template <typename T, int NB, int CW>
constexpr size_t diag_smem_bytes()
{
    return sizeof(T) * (size_t(NB) * NB + NB + size_t(NB) * (CW + 1));
}

// The substitution of one warp: rows i = 4 m + RG of right-hand side `col`
// (column group cg).  At step k the warp owning row k forms x_k = t_k / a_kk
// and publishes it in Bs (row k); after the column group's named barrier the
// four warps subtract a_ik x_k from their rows below (forward) or above
// (backward) k.  Fully unrolled with RG fixed, so t stays in registers and
// every row test is a compile-time constant.  The four warps of a column
// group run different instantiations and meet at the same named barrier
// (a counting barrier of 128 threads) from their own code.
template <typename T, int NB, bool FWD, bool MT, int CW, int RG>
__device__ __forceinline__ void diag_rows(const T *L, const T *inv, T *Bs, int nr, int col, int cg, T alpha)
{
    constexpr int BS = CW + 1;
    constexpr int NM = NB / 4;
    T t[NM];
    // a warp reads only its own rows of B, and x_k overwrites row k, owned by
    // the warp that writes it: no barrier needed before the steps
#pragma unroll
    for (int m = 0; m < NM; m++) t[m] = alpha * Bs[(4 * m + RG) * BS + col];
    const uint32_t bar_id = 1u + uint32_t(cg);
#pragma unroll
    for (int s = 0; s < NB; s++) {
        const int k = FWD ? s : NB - 1 - s;
        if (k < nr) {
            if ((k & 3) == RG) {
                const T x = t[k >> 2] * inv[k];
                t[k >> 2] = x;
                Bs[k * BS + col] = x;
            }
            asm volatile("bar.sync %0, 128;" ::"r"(bar_id) : "memory");
            const T x = Bs[k * BS + col];
#pragma unroll
            for (int m = 0; m < NM; m++) {
                const int i = 4 * m + RG;
                if (FWD ? (i > k) : (i < k)) t[m] -= (MT ? L[i * NB + k] : L[k * NB + i]) * x;
            }
        }
    }
}

// FWD: Mv lower (forward substitution); MT: Mv(i,j) = A(j,i); LEFT: Bv
// column-major.  Msub = &A(r0, r0), Bsub = &Bv(r0, 0).
// EMIT: also write a BF16 copy of the solved block to Ebf (column-major,
// ldb), the operand of the tensor-core GEMM updates (LEFT layout only).
template <typename T, int NB, bool FWD, bool MT, bool LEFT, bool EMIT, int CW>
__global__ void __launch_bounds__(kDiagThreads)
diag_solve_kernel(const T *__restrict__ Msub, int64_t lda, T *__restrict__ Bsub,
                  int64_t ldb, int nr, int64_t ncols, T alpha, int unit,
                  __nv_bfloat16 *__restrict__ Ebf)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *L = reinterpret_cast<T *>(smem_raw);
    T *inv = L + NB * NB;
    T *Bs = inv + NB;
    constexpr int BS = CW + 1;

    const int tid = threadIdx.x;
    const int64_t c0 = int64_t(blockIdx.x) * CW;
    const int ncb = (int)((ncols - c0) < CW ? (ncols - c0) : CW);

    // ---- triangle and B panel -> shared memory, as asynchronous copies ----
    // (every copy of the thread in flight at once: a loop of load-then-store
    // would wait out the memory latency once per element).  Global A is
    // column-major; Mv(i,k) = MT ? A(k,i) : A(i,k).  The loop index runs
    // fastest over A's contiguous dimension; entries outside the referenced
    // strict triangle are zero-filled.
    for (int idx = tid; idx < NB * NB; idx += kDiagThreads) {
        int fast = idx % NB, slow = idx / NB;  // fast = row of A, slow = col of A
        int i = MT ? slow : fast;              // row of Mv
        int k = MT ? fast : slow;              // col of Mv
        bool ref = (i < nr) && (k < nr) && (FWD ? (k < i) : (k > i));
        // column form stores Mv(:,k) contiguously, row form Mv(i,:)
        diag_cp_async(&L[MT ? (i * NB + k) : (k * NB + i)], ref ? Msub + fast + int64_t(slow) * lda : Msub, ref);
    }
    // B panel, coalesced
    if (LEFT) {  // Bv(i,c) = Bsub[i + c*ldb]: contiguous in i
        for (int idx = tid; idx < NB * CW; idx += kDiagThreads) {
            int i = idx % NB, c = idx / NB;
            const bool in = i < nr && c < ncb;
            diag_cp_async(&Bs[i * BS + c], in ? Bsub + i + (c0 + c) * ldb : Bsub, in);
        }
    } else {     // Bv(i,c) = Bsub[c + i*ldb]: contiguous in c
        for (int idx = tid; idx < NB * CW; idx += kDiagThreads) {
            int c = idx % CW, i = idx / CW;
            const bool in = i < nr && c < ncb;
            diag_cp_async(&Bs[i * BS + c], in ? Bsub + (c0 + c) + int64_t(i) * ldb : Bsub, in);
        }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    for (int i = tid; i < NB; i += kDiagThreads) {
        T d = T(1);
        if (i < nr && !unit) d = T(1) / Msub[i + int64_t(i) * lda];
        inv[i] = d;
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();

    // ---- substitution: rows split over the four warps of a column group -----
    // Bs holds B on entry; once every thread has its rows in registers it
    // holds the published x_k (row k of the solved block).
    {
        const int warp = tid >> 5, lane = tid & 31;
        const int cg = warp >> 2, rg = warp & 3;
        const int col = cg * 32 + lane;
        // one code path per row group, so that every row test is resolved at
        // compile time (no predicated-off FP64 instructions)
        switch (rg) {
        case 0: diag_rows<T, NB, FWD, MT, CW, 0>(L, inv, Bs, nr, col, cg, alpha); break;
        case 1: diag_rows<T, NB, FWD, MT, CW, 1>(L, inv, Bs, nr, col, cg, alpha); break;
        case 2: diag_rows<T, NB, FWD, MT, CW, 2>(L, inv, Bs, nr, col, cg, alpha); break;
        default: diag_rows<T, NB, FWD, MT, CW, 3>(L, inv, Bs, nr, col, cg, alpha); break;
        }
        // Bs now holds x_k in row k for every k < nr: the solved block
    }
    __syncthreads();

    // ---- write back, coalesced --------------------------------------------
    if (LEFT) {
        for (int idx = tid; idx < NB * CW; idx += kDiagThreads) {
            int i = idx % NB, c = idx / NB;
            if (i < nr && c < ncb) {
                Bsub[i + (c0 + c) * ldb] = Bs[i * BS + c];
                if (EMIT) Ebf[i + (c0 + c) * ldb] = __float2bfloat16_rn(float(Bs[i * BS + c]));
            }
        }
    } else {
        for (int idx = tid; idx < NB * CW; idx += kDiagThreads) {
            int c = idx % CW, i = idx / CW;
            if (i < nr && c < ncb) Bsub[(c0 + c) + int64_t(i) * ldb] = Bs[i * BS + c];
        }
    }
}

// One-time kernel attribute (dynamic shared memory above 48 KB).
template <typename T, int NB, bool FWD, bool MT, bool LEFT, bool EMIT, int CW>
int diag_prepare()
{
    static PerDeviceOnce attr;  // per instantiation and device
    return smem_attr_once(attr, diag_solve_kernel<T, NB, FWD, MT, LEFT, EMIT, CW>, diag_smem_bytes<T, NB, CW>());
}

template <typename T, int NB, bool FWD, bool MT, bool LEFT, bool EMIT, int CW>
int launch_nb_cw(const T *Msub, int64_t lda, T *Bsub, int64_t ldb, int nr, int64_t ncols, T alpha, int unit,
                 cudaStream_t s, __nv_bfloat16 *Ebf)
{
    auto kern = diag_solve_kernel<T, NB, FWD, MT, LEFT, EMIT, CW>;
    constexpr size_t smem = diag_smem_bytes<T, NB, CW>();
    {
        const int pst = diag_prepare<T, NB, FWD, MT, LEFT, EMIT, CW>();
        if (pst) return pst;
    }
    int64_t grid = (ncols + CW - 1) / CW;
    if (grid > 0x7fffffff) return GB_STATUS_CUDA_ERROR;
    LaunchScope ls(KK_DIAG, s, double(nr) * nr * ncols,
                   sizeof(T) * (0.5 * nr * nr + 2.0 * nr * ncols));
    kern<<<(unsigned)grid, kDiagThreads, smem, s>>>(Msub, lda, Bsub, ldb, nr, ncols, alpha, unit, Ebf);
    return check(cudaGetLastError());
}

template <typename T, int NB, bool FWD, bool MT, bool LEFT, bool EMIT = false>
int launch_nb(const T *Msub, int64_t lda, T *Bsub, int64_t ldb, int nr, int64_t ncols,
              T alpha, int unit, cudaStream_t s, __nv_bfloat16 *Ebf = nullptr)
{
    return launch_nb_cw<T, NB, FWD, MT, LEFT, EMIT, 64>(Msub, lda, Bsub, ldb, nr, ncols, alpha, unit, s, Ebf);
}

template <typename T, bool FWD, bool MT, bool LEFT>
int launch_dir(const T *Msub, int64_t lda, T *Bsub, int64_t ldb, int nr, int64_t ncols,
               T alpha, int unit, cudaStream_t s)
{
    if (nr <= 16) return launch_nb<T, 16, FWD, MT, LEFT>(Msub, lda, Bsub, ldb, nr, ncols, alpha, unit, s);
    if (nr <= 32) return launch_nb<T, 32, FWD, MT, LEFT>(Msub, lda, Bsub, ldb, nr, ncols, alpha, unit, s);
    return launch_nb<T, 64, FWD, MT, LEFT>(Msub, lda, Bsub, ldb, nr, ncols, alpha, unit, s);
}

}  // namespace

template <typename T>
int launch_diag_solve(const Canon<T> &c, int64_t r0, int nr, T alpha)
{
    if (nr <= 0 || c.ncols <= 0) return 0;
    if (nr > 64) return GB_STATUS_CUDA_ERROR;  // driver never asks for more
    const T *Msub = c.A + r0 + r0 * c.lda;
    T *Bsub = bv_ptr(c, r0, 0);
    int unit = c.unit ? 1 : 0;
#define GB_DIAG_CASE(F, M, L)                                                             \
    if (c.forward == F && c.mt == M && c.left == L)                                       \
        return launch_dir<T, F, M, L>(Msub, c.lda, Bsub, c.ldb, nr, c.ncols, alpha, unit, \
                                      c.stream);
    GB_DIAG_CASE(true, false, true)
    GB_DIAG_CASE(true, false, false)
    GB_DIAG_CASE(true, true, true)
    GB_DIAG_CASE(true, true, false)
    GB_DIAG_CASE(false, false, true)
    GB_DIAG_CASE(false, false, false)
    GB_DIAG_CASE(false, true, true)
    GB_DIAG_CASE(false, true, false)
#undef GB_DIAG_CASE
    return GB_STATUS_CUDA_ERROR;
}

}  // namespace gb

// Off-diagonal update C = alpha*C - Aop*Bop on CUDA cores: the paper's gemm
// task (Section IV stage 2, b.low -= L.mid x.up; with many right-hand sides
// the gemv becomes a GEMM, Section V-A).  Used by the FP64 path (DFMA: the
// GB300 FP64 rate is set by the DFMA pipe, and tcgen05 has no f64 kind) and
// by the FP32 path (FFMA).
//
// Design: CTA tile BM x BN, k-slices of BK staged in shared memory with a
// register double buffer (global loads of slice k+1 are in flight while
// slice k is multiplied).  Each thread owns a TM x TN micro-tile split in two
// halves (rows ty*TM/2.. and BM/2 + ty*TM/2..) so that its shared-memory
// reads are conflict-free 16-byte vectors.  Global loads run along whichever
// dimension is contiguous (A normal or transposed; B/C column-major for
// side Left, row-major for side Right), and are transposed on the way into
// shared memory.  alpha is applied to C in the epilogue (first touch).
#include "common.cuh"

namespace gb {
namespace {

template <typename T>
struct Cfg;
template <>
struct Cfg<float> {  // FFMA: 128x128 tile, 8x8 per thread, 256 threads
    static constexpr int BM = 128, BN = 128, BK = 8, TM = 8, TN = 8;
};
template <>
struct Cfg<double> {  // DFMA: 64x64 tile, 4x4 per thread, 256 threads
    static constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4;
};

template <typename T, int W>
struct VecT;
template <>
struct VecT<float, 4> {
    using type = float4;
};
template <>
struct VecT<double, 2> {
    using type = double2;
};

// AM: A-operand contiguous along M (Mv(i,k) = A(i,k), i.e. !mt).
// LEFT: Bop/C column-major (contiguous along K / M); else row-major.
template <typename T, bool AM, bool LEFT>
__global__ void __launch_bounds__((Cfg<T>::BM / Cfg<T>::TM) * (Cfg<T>::BN / Cfg<T>::TN))
gemm_update_kernel(int64_t M, int64_t N, int64_t K, const T *__restrict__ A, int64_t lda,
                   const T *__restrict__ B, int64_t ldb, T *__restrict__ C, int64_t ldc, T alpha)
{
    constexpr int BM = Cfg<T>::BM, BN = Cfg<T>::BN, BK = Cfg<T>::BK;
    constexpr int TM = Cfg<T>::TM, TN = Cfg<T>::TN;
    constexpr int NTX = BN / TN, NTY = BM / TM;
    constexpr int NT = NTX * NTY;
    constexpr int VW = TM / 2;  // vector width of one half micro-tile
    static_assert(TM == TN, "square micro-tile");
    static_assert(VW * sizeof(T) == 16, "16-byte shared vectors");
    constexpr int PAD = VW;     // keeps rows 16-byte aligned, spreads banks
    constexpr int LDA_S = BM + PAD, LDB_S = BN + PAD;
    constexpr int A_PER = BM * BK / NT, B_PER = BN * BK / NT;
    static_assert(A_PER * NT == BM * BK && B_PER * NT == BN * BK, "tile split");
    using V = typename VecT<T, VW>::type;

    __shared__ __align__(16) T As[2][BK * LDA_S];
    __shared__ __align__(16) T Bs[2][BK * LDB_S];

    const int tid = threadIdx.x;
    const int tx = tid % NTX, ty = tid / NTX;
    const int64_t m0 = int64_t(blockIdx.y) * BM;
    const int64_t n0 = int64_t(blockIdx.x) * BN;

    T ra[A_PER], rb[B_PER];

    // Global -> registers for k-slice starting at kk.
    auto load_tiles = [&](int64_t kk) {
#pragma unroll
        for (int p = 0; p < A_PER; p++) {
            int idx = tid + p * NT;
            int i, k;
            if (AM) { i = idx % BM; k = idx / BM; }
            else    { k = idx % BK; i = idx / BK; }
            int64_t gi = m0 + i, gk = kk + k;
            T v = T(0);
            if (gi < M && gk < K) v = AM ? A[gi + gk * lda] : A[gk + gi * lda];
            ra[p] = v;
        }
#pragma unroll
        for (int p = 0; p < B_PER; p++) {
            int idx = tid + p * NT;
            int k, j;
            if (LEFT) { k = idx % BK; j = idx / BK; }
            else      { j = idx % BN; k = idx / BN; }
            int64_t gk = kk + k, gj = n0 + j;
            T v = T(0);
            if (gk < K && gj < N) v = LEFT ? B[gk + gj * ldb] : B[gj + gk * ldb];
            rb[p] = v;
        }
    };
    auto store_tiles = [&](int buf) {
#pragma unroll
        for (int p = 0; p < A_PER; p++) {
            int idx = tid + p * NT;
            int i, k;
            if (AM) { i = idx % BM; k = idx / BM; }
            else    { k = idx % BK; i = idx / BK; }
            As[buf][k * LDA_S + i] = ra[p];
        }
#pragma unroll
        for (int p = 0; p < B_PER; p++) {
            int idx = tid + p * NT;
            int k, j;
            if (LEFT) { k = idx % BK; j = idx / BK; }
            else      { j = idx % BN; k = idx / BN; }
            Bs[buf][k * LDB_S + j] = rb[p];
        }
    };

    T acc[TM][TN];
#pragma unroll
    for (int r = 0; r < TM; r++)
#pragma unroll
        for (int c = 0; c < TN; c++) acc[r][c] = T(0);

    const int64_t nk = (K + BK - 1) / BK;
    if (nk > 0) {
        load_tiles(0);
        store_tiles(0);
        __syncthreads();
    }
    for (int64_t kt = 0; kt < nk; kt++) {
        const int cur = int(kt & 1);
        if (kt + 1 < nk) load_tiles((kt + 1) * BK);
#pragma unroll
        for (int k = 0; k < BK; k++) {
            T a[TM], b[TN];
            V a0 = *reinterpret_cast<const V *>(&As[cur][k * LDA_S + ty * VW]);
            V a1 = *reinterpret_cast<const V *>(&As[cur][k * LDA_S + BM / 2 + ty * VW]);
            V b0 = *reinterpret_cast<const V *>(&Bs[cur][k * LDB_S + tx * VW]);
            V b1 = *reinterpret_cast<const V *>(&Bs[cur][k * LDB_S + BN / 2 + tx * VW]);
            const T *pa0 = reinterpret_cast<const T *>(&a0), *pa1 = reinterpret_cast<const T *>(&a1);
            const T *pb0 = reinterpret_cast<const T *>(&b0), *pb1 = reinterpret_cast<const T *>(&b1);
#pragma unroll
            for (int e = 0; e < VW; e++) {
                a[e] = pa0[e]; a[VW + e] = pa1[e];
                b[e] = pb0[e]; b[VW + e] = pb1[e];
            }
#pragma unroll
            for (int r = 0; r < TM; r++)
#pragma unroll
                for (int c = 0; c < TN; c++) acc[r][c] = fma(a[r], b[c], acc[r][c]);
        }
        if (kt + 1 < nk) {
            store_tiles(cur ^ 1);
            __syncthreads();
        }
    }

    // ---- epilogue: C = alpha*C - acc ----------------------------------------
#pragma unroll
    for (int r = 0; r < TM; r++) {
        int64_t gi = m0 + (r < VW ? ty * VW + r : BM / 2 + ty * VW + (r - VW));
        if (gi >= M) continue;
#pragma unroll
        for (int c = 0; c < TN; c++) {
            int64_t gj = n0 + (c < VW ? tx * VW + c : BN / 2 + tx * VW + (c - VW));
            if (gj >= N) continue;
            T *p = LEFT ? &C[gi + gj * ldc] : &C[gj + gi * ldc];
            *p = (alpha == T(1)) ? (*p - acc[r][c]) : (alpha * *p - acc[r][c]);
        }
    }
}

template <typename T, bool AM, bool LEFT>
int launch_cfg(int64_t M, int64_t N, int64_t K, const T *A, int64_t lda, const T *B,
               int64_t ldb, T *C, int64_t ldc, T alpha, cudaStream_t s)
{
    constexpr int BM = Cfg<T>::BM, BN = Cfg<T>::BN;
    constexpr int NT = (BM / Cfg<T>::TM) * (BN / Cfg<T>::TN);
    int64_t gx = (N + BN - 1) / BN, gy = (M + BM - 1) / BM;
    if (gx > 0x7fffffff || gy > 65535) return GB_STATUS_CUDA_ERROR;
    LaunchScope ls(KK_GEMM_SIMT, s, 2.0 * M * N * K,
                   sizeof(T) * (double(M) * K + double(K) * N + 2.0 * M * N));
    gemm_update_kernel<T, AM, LEFT><<<dim3((unsigned)gx, (unsigned)gy), NT, 0, s>>>(
        M, N, K, A, lda, B, ldb, C, ldc, alpha);
    return check(cudaGetLastError());
}

}  // namespace

template <typename T>
int launch_gemm_update(const Canon<T> &c, int64_t ci0, int64_t M, int64_t ak0, int64_t K, T alpha)
{
    if (M <= 0 || c.ncols <= 0) return 0;
    if (K <= 0) {
        if (alpha == T(1)) return 0;
        K = 0;  // still scale C by alpha
    }
    const T *Ap = mv_ptr(c, ci0, ak0);
    const T *Bp = bv_ptr(c, ak0, 0);
    T *Cp = bv_ptr(c, ci0, 0);
    const bool am = !c.mt;
    if (am && c.left) return launch_cfg<T, true, true>(M, c.ncols, K, Ap, c.lda, Bp, c.ldb, Cp, c.ldb, alpha, c.stream);
    if (am && !c.left) return launch_cfg<T, true, false>(M, c.ncols, K, Ap, c.lda, Bp, c.ldb, Cp, c.ldb, alpha, c.stream);
    if (!am && c.left) return launch_cfg<T, false, true>(M, c.ncols, K, Ap, c.lda, Bp, c.ldb, Cp, c.ldb, alpha, c.stream);
    return launch_cfg<T, false, false>(M, c.ncols, K, Ap, c.lda, Bp, c.ldb, Cp, c.ldb, alpha, c.stream);
}

template int launch_gemm_update<double>(const Canon<double> &, int64_t, int64_t, int64_t, int64_t, double);
template int launch_gemm_update<float>(const Canon<float> &, int64_t, int64_t, int64_t, int64_t, float);

}  // namespace gb

// The gemm task on its own, column-major operands: C (M x N, ldc) =
// alpha*C - A (M x K, lda) * B (K x N, ldb), FP64 (dtype 0) or FP32 (1) --
// the kernel every plain solve uses for its off-diagonal updates.
extern "C" int gb_gemm_update(int dtype, int64_t M, int64_t N, int64_t K, const void *A, int64_t lda, const void *B,
                              int64_t ldb, void *C, int64_t ldc, double alpha, void *stream)
{
    if (dtype != 0 && dtype != 1) return -1;
    if (M < 0) return -2;
    if (N < 0) return -3;
    if (K < 0) return -4;
    if (A == nullptr && M * K > 0) return -5;
    if (lda < (M > 1 ? M : 1)) return -6;
    if (B == nullptr && K * N > 0) return -7;
    if (ldb < (K > 1 ? K : 1)) return -8;
    if (C == nullptr && M * N > 0) return -9;
    if (ldc < (M > 1 ? M : 1)) return -10;
    if (M == 0 || N == 0) return 0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (dtype == 0)
        return gb::launch_cfg<double, true, true>(M, N, K, static_cast<const double *>(A), lda,
                                                  static_cast<const double *>(B), ldb, static_cast<double *>(C), ldc,
                                                  alpha, s);
    return gb::launch_cfg<float, true, true>(M, N, K, static_cast<const float *>(A), lda,
                                             static_cast<const float *>(B), ldb, static_cast<float *>(C), ldc,
                                             float(alpha), s);
}

namespace gb {

// ---- alpha == 0: Bv = 0 ------------------------------------------------------
namespace {
template <typename T>
__global__ void zero_kernel(T *B, int64_t ldb, int64_t rows, int64_t cols)
{
    // rows = contiguous extent, cols = strided extent
    int64_t total = rows * cols;
    for (int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; idx < total;
         idx += int64_t(gridDim.x) * blockDim.x) {
        int64_t r = idx % rows, c = idx / rows;
        B[r + c * ldb] = T(0);
    }
}
}  // namespace

template <typename T>
int launch_zero(const Canon<T> &c)
{
    // Bv column-major (Left): k rows contiguous, ncols strided; row-major
    // (Right): ncols contiguous, k strided.
    int64_t rows = c.left ? c.k : c.ncols, cols = c.left ? c.ncols : c.k;
    if (rows <= 0 || cols <= 0) return 0;
    int64_t total = rows * cols;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    LaunchScope ls(KK_CONVERT, c.stream, 0.0, sizeof(T) * double(total));
    zero_kernel<T><<<(unsigned)blocks, 256, 0, c.stream>>>(c.B, c.ldb, rows, cols);
    return check(cudaGetLastError());
}

template int launch_zero<double>(const Canon<double> &);
template int launch_zero<float>(const Canon<float> &);

}  // namespace gb

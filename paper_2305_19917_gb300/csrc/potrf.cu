// Cholesky factorisation on this triangular solver: the use the paper names
// for its TS machinery (Section VIII, future work), built with the same
// recursive computation model (Section V-A) as the solve:
//
//     A = [A11 A21^T; A21 A22]  ->  L11 = chol(A11)             (recursion)
//                                   L21 = A21 L11^-T             (TS task: the
//                                         library's own TRSM, side Right)
//                                   A22 -= L21 L21^T             (gemm task:
//                                         a SYRK update of the lower triangle)
//                                   L22 = chol(A22)              (recursion)
//
// down to leaves of at most 64 columns, each factorised by one CTA in shared
// memory.  The upper form (A = U^T U) is the mirror image: U12 = U11^-T A12
// (TRSM side Left, Upper, transposed) and A22 -= U12^T U12.  Only the named
// triangle of A is read and written.
//
// A non-positive (or NaN) pivot stops the leaf that meets it; the leaf
// records info = (global column + 1) in a device word (the first failure
// wins, leaves run in order) and every later leaf returns without work.  As
// with LAPACK, the contents of A from that column on are then undefined.
#include <cmath>
#include "common.cuh"
#include "driver.cuh"
#include "mixed.cuh"

extern "C" int gb_dtrsm(int side, int uplo, int trans, int diag, int64_t m, int64_t n, double alpha,
                        const double *A, int64_t lda, double *B, int64_t ldb, void *stream);
extern "C" int gb_strsm(int side, int uplo, int trans, int diag, int64_t m, int64_t n, float alpha,
                        const float *A, int64_t lda, float *B, int64_t ldb, void *stream);

namespace gb {
namespace {

constexpr int kLeafNB = 64;
constexpr int kLeafThreads = 256;

// One diagonal block of order nr <= 64 at &A(r0, r0) (A0 points there),
// factorised right-looking in shared memory.  s[i][c] (i >= c) holds the
// block's lower triangle: A(i, c) for the lower form, A(c, i) for the upper.
template <typename T>
__global__ void __launch_bounds__(kLeafThreads)
potrf_leaf_kernel(T *__restrict__ A0, int64_t lda, int nr, int upper, int64_t r0, int *info)
{
    __shared__ T s[kLeafNB][kLeafNB + 1];
    __shared__ int fail;
    if (*static_cast<volatile int *>(info) != 0) return;  // an earlier leaf failed
    const int tid = threadIdx.x;
    // load the named triangle, reading A along its contiguous dimension
    for (int idx = tid; idx < nr * nr; idx += kLeafThreads) {
        const int fast = idx % nr, slow = idx / nr;  // A(fast, slow)
        if (!upper && fast >= slow) s[fast][slow] = A0[fast + int64_t(slow) * lda];
        if (upper && fast <= slow) s[slow][fast] = A0[fast + int64_t(slow) * lda];
    }
    if (tid == 0) fail = -1;
    __syncthreads();
    for (int j = 0; j < nr; j++) {
        if (tid == 0) {
            const T d = s[j][j];
            if (!(d > T(0))) fail = j;
            else s[j][j] = sqrt(d);
        }
        __syncthreads();
        if (fail >= 0) break;
        const T ljj = s[j][j];
        for (int i = j + 1 + tid; i < nr; i += kLeafThreads) s[i][j] = s[i][j] / ljj;
        __syncthreads();
        // trailing update of the lower triangle: s[i][c] -= l_ij l_cj, j < c <= i
        const int w = nr - j - 1;
        for (int idx = tid; idx < w * w; idx += kLeafThreads) {
            const int i = j + 1 + idx % w, c = j + 1 + idx / w;
            if (c <= i) s[i][c] -= s[i][j] * s[c][j];
        }
        __syncthreads();
    }
    if (fail >= 0) {
        if (tid == 0) atomicCAS(info, 0, int(r0 + fail + 1));
        return;
    }
    for (int idx = tid; idx < nr * nr; idx += kLeafThreads) {
        const int fast = idx % nr, slow = idx / nr;
        if (!upper && fast >= slow) A0[fast + int64_t(slow) * lda] = s[fast][slow];
        if (upper && fast <= slow) A0[fast + int64_t(slow) * lda] = s[slow][fast];
    }
}

// ---- SYRK update: C -= P P^T (lower) or C -= P^T P (upper) -----------------
// The gemm task of the factorisation, restricted to the named triangle of
// the symmetric C (order M): lower form, P is M x K (column-major, ldp) and
// C(i, c) -= sum_k P(i, k) P(c, k) for i >= c; upper form, P is K x M and
// C(i, c) -= sum_k P(k, i) P(k, c) for i <= c.  CTA tiles of BM x BM cover
// the triangle only (a 1-D grid over the T (T + 1) / 2 tiles on and below /
// above the diagonal); k-slices of BK are staged in shared memory with a
// register double buffer, each thread owning a TM x TM micro-tile split in
// two halves so that its shared-memory reads are 16-byte vectors (the
// layout of the solve's gemm task).
template <typename T>
struct SyrkCfg;
template <>
struct SyrkCfg<double> {  // DFMA: 64 x 64 tile, 4 x 4 per thread, 256 threads
    static constexpr int BM = 64, BK = 16, TM = 4;
};
template <>
struct SyrkCfg<float> {  // FFMA: 128 x 128 tile, 8 x 8 per thread, 256 threads
    static constexpr int BM = 128, BK = 8, TM = 8;
};
template <typename T, int W>
struct SyrkVec;
template <>
struct SyrkVec<double, 2> {
    using type = double2;
};
template <>
struct SyrkVec<float, 4> {
    using type = float4;
};

template <typename T, bool UP>
__global__ void __launch_bounds__((SyrkCfg<T>::BM / SyrkCfg<T>::TM) * (SyrkCfg<T>::BM / SyrkCfg<T>::TM))
syrk_update_kernel(int64_t M, int64_t K, const T *__restrict__ P, int64_t ldp, T *__restrict__ C, int64_t ldc)
{
    constexpr int BM = SyrkCfg<T>::BM, BK = SyrkCfg<T>::BK, TM = SyrkCfg<T>::TM;
    constexpr int NTX = BM / TM, NT = NTX * NTX;
    constexpr int VW = TM / 2;
    static_assert(VW * sizeof(T) == 16, "16-byte shared vectors");
    constexpr int LDS = BM + VW;
    constexpr int PER = BM * BK / NT;
    static_assert(PER * NT == BM * BK, "tile split");
    using V = typename SyrkVec<T, VW>::type;
    __shared__ __align__(16) T Rs[2][BK * LDS];  // rows operand: R(i, k), tile rows
    __shared__ __align__(16) T Cs[2][BK * LDS];  // columns operand: R(c, k), tile columns

    // tile (ti, tc) of the triangle: linear index t over tc <= ti (lower) or
    // ti <= tc (upper, the same enumeration with the roles swapped)
    const int64_t t = blockIdx.x;
    int64_t a = int64_t((sqrt(8.0 * double(t) + 1.0) - 1.0) / 2.0);
    while (a * (a + 1) / 2 > t) a--;
    while ((a + 1) * (a + 2) / 2 <= t) a++;
    const int64_t b = t - a * (a + 1) / 2;  // 0 <= b <= a
    const int64_t ti = UP ? b : a, tc = UP ? a : b;
    const int64_t i0 = ti * BM, c0 = tc * BM;

    const int tid = threadIdx.x;
    const int tx = tid % NTX, ty = tid / NTX;
    T rr[PER], rc[PER];
    // element (row x, k) of the operand R with R(x, k) = P(x, k) (lower) or
    // P(k, x) (upper), read along P's contiguous dimension
    auto load = [&](int64_t kk) {
#pragma unroll
        for (int p = 0; p < PER; p++) {
            const int idx = tid + p * NT;
            int x, k;
            if (!UP) { x = idx % BM; k = idx / BM; }
            else     { k = idx % BK; x = idx / BK; }
            const int64_t gk = kk + k, gi = i0 + x, gc = c0 + x;
            T vi = T(0), vc = T(0);
            if (gk < K) {
                if (gi < M) vi = UP ? P[gk + gi * ldp] : P[gi + gk * ldp];
                if (gc < M) vc = UP ? P[gk + gc * ldp] : P[gc + gk * ldp];
            }
            rr[p] = vi;
            rc[p] = vc;
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int p = 0; p < PER; p++) {
            const int idx = tid + p * NT;
            int x, k;
            if (!UP) { x = idx % BM; k = idx / BM; }
            else     { k = idx % BK; x = idx / BK; }
            Rs[buf][k * LDS + x] = rr[p];
            Cs[buf][k * LDS + x] = rc[p];
        }
    };
    T acc[TM][TM];
#pragma unroll
    for (int r = 0; r < TM; r++)
#pragma unroll
        for (int c = 0; c < TM; c++) acc[r][c] = T(0);
    const int64_t nk = (K + BK - 1) / BK;
    if (nk > 0) {
        load(0);
        store(0);
        __syncthreads();
    }
    for (int64_t kt = 0; kt < nk; kt++) {
        const int cur = int(kt & 1);
        if (kt + 1 < nk) load((kt + 1) * BK);
#pragma unroll
        for (int k = 0; k < BK; k++) {
            T x[TM], y[TM];
            const V a0 = *reinterpret_cast<const V *>(&Rs[cur][k * LDS + ty * VW]);
            const V a1 = *reinterpret_cast<const V *>(&Rs[cur][k * LDS + BM / 2 + ty * VW]);
            const V b0 = *reinterpret_cast<const V *>(&Cs[cur][k * LDS + tx * VW]);
            const V b1 = *reinterpret_cast<const V *>(&Cs[cur][k * LDS + BM / 2 + tx * VW]);
            const T *pa0 = reinterpret_cast<const T *>(&a0), *pa1 = reinterpret_cast<const T *>(&a1);
            const T *pb0 = reinterpret_cast<const T *>(&b0), *pb1 = reinterpret_cast<const T *>(&b1);
#pragma unroll
            for (int e = 0; e < VW; e++) {
                x[e] = pa0[e];
                x[VW + e] = pa1[e];
                y[e] = pb0[e];
                y[VW + e] = pb1[e];
            }
#pragma unroll
            for (int r = 0; r < TM; r++)
#pragma unroll
                for (int c = 0; c < TM; c++) acc[r][c] = fma(x[r], y[c], acc[r][c]);
        }
        if (kt + 1 < nk) {
            store(cur ^ 1);
            __syncthreads();
        }
    }
#pragma unroll
    for (int r = 0; r < TM; r++) {
        const int64_t gi = i0 + (r < VW ? ty * VW + r : BM / 2 + ty * VW + (r - VW));
        if (gi >= M) continue;
#pragma unroll
        for (int c = 0; c < TM; c++) {
            const int64_t gc = c0 + (c < VW ? tx * VW + c : BM / 2 + tx * VW + (c - VW));
            if (gc >= M || (UP ? gi > gc : gi < gc)) continue;
            T *q = &C[gi + gc * ldc];
            *q = *q - acc[r][c];
        }
    }
}

template <typename T>
int launch_syrk(bool upper, int64_t M, int64_t K, const T *P, int64_t ldp, T *C, int64_t ldc, cudaStream_t s)
{
    if (M <= 0 || K <= 0) return 0;
    constexpr int BM = SyrkCfg<T>::BM, NT = (BM / SyrkCfg<T>::TM) * (BM / SyrkCfg<T>::TM);
    const int64_t tiles = (M + BM - 1) / BM;
    const int64_t grid = tiles * (tiles + 1) / 2;
    if (grid > 0x7fffffffLL) return GB_STATUS_CUDA_ERROR;
    // algorithmic work: the triangle of C (M (M + 1) / 2 entries) x K multiply-adds
    LaunchScope ls(KK_GEMM_SIMT, s, double(M) * double(M + 1) * double(K),
                   sizeof(T) * (double(M) * K + double(M) * double(M + 1)));
    if (upper)
        syrk_update_kernel<T, true><<<(unsigned)grid, NT, 0, s>>>(M, K, P, ldp, C, ldc);
    else
        syrk_update_kernel<T, false><<<(unsigned)grid, NT, 0, s>>>(M, K, P, ldp, C, ldc);
    return check(cudaGetLastError());
}

int trsm_call(int side, int uplo, int trans, int64_t m, int64_t n, const double *A, int64_t lda, double *B,
              int64_t ldb, cudaStream_t s)
{
    return gb_dtrsm(side, uplo, trans, GB_NONUNIT, m, n, 1.0, A, lda, B, ldb, s);
}
int trsm_call(int side, int uplo, int trans, int64_t m, int64_t n, const float *A, int64_t lda, float *B,
              int64_t ldb, cudaStream_t s)
{
    return gb_strsm(side, uplo, trans, GB_NONUNIT, m, n, 1.0f, A, lda, B, ldb, s);
}

// Recursive model (Section V-A) on columns [off, off + n) of the
// factorisation, A pointing at their diagonal block.
template <typename T>
int potrf_rec(int uplo, int64_t n, T *A, int64_t lda, int64_t off, int *info, cudaStream_t s)
{
    if (n <= 0) return 0;
    if (n <= kLeafNB) {
        LaunchScope ls(KK_DIAG, s, double(n) * n * n / 3.0, sizeof(T) * double(n) * (n + 1));
        potrf_leaf_kernel<T><<<1, kLeafThreads, 0, s>>>(A, lda, int(n), uplo == GB_UPPER, off, info);
        return check(cudaGetLastError());
    }
    const int64_t n1 = rec_split(n, kLeafNB), n2 = n - n1;
    GB_TRY(potrf_rec(uplo, n1, A, lda, off, info, s));
    T *A22 = A + n1 + n1 * lda;
    if (uplo == GB_LOWER) {
        T *A21 = A + n1;
        GB_TRY(trsm_call(GB_RIGHT, GB_LOWER, GB_TRANS, n2, n1, A, lda, A21, lda, s));  // L21 = A21 L11^-T
        GB_TRY(launch_syrk<T>(false, n2, n1, A21, lda, A22, lda, s));                   // A22 -= L21 L21^T
    } else {
        T *A12 = A + n1 * lda;
        GB_TRY(trsm_call(GB_LEFT, GB_UPPER, GB_TRANS, n1, n2, A, lda, A12, lda, s));    // U12 = U11^-T A12
        GB_TRY(launch_syrk<T>(true, n2, n1, A12, lda, A22, lda, s));                    // A22 -= U12^T U12
    }
    return potrf_rec(uplo, n2, A22, lda, off + n1, info, s);
}

template <typename T>
int potrf_impl(int uplo, int64_t n, T *A, int64_t lda, int64_t *info_out, void *stream)
{
    if (uplo != GB_LOWER && uplo != GB_UPPER) return -1;
    if (n < 0) return -2;
    if (A == nullptr && n > 0) return -3;
    if (lda < (n > 1 ? n : 1)) return -4;
    if (info_out == nullptr) return -5;
    *info_out = 0;
    if (n == 0) return 0;
    if (n > 0x7ffffffeLL) return -2;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaMemPool_t pool = mixed_pool();
    if (!pool) return GB_STATUS_CUDA_ERROR;
    int *dinfo = nullptr;
    GB_CUDA(cudaMallocFromPoolAsync(reinterpret_cast<void **>(&dinfo), sizeof(int), pool, s));
    int st = check(cudaMemsetAsync(dinfo, 0, sizeof(int), s));
    if (!st) st = potrf_rec<T>(uplo, n, A, lda, 0, dinfo, s);
    int h = 0;
    if (!st) st = check(cudaMemcpyAsync(&h, dinfo, sizeof(int), cudaMemcpyDeviceToHost, s));
    cudaFreeAsync(dinfo, s);
    const int c = check(cudaStreamSynchronize(s));
    if (st) return st;
    if (c) return c;
    *info_out = h;
    return 0;
}

}  // namespace
}  // namespace gb

extern "C" int gb_dpotrf(int uplo, int64_t n, double *A, int64_t lda, int64_t *info, void *stream)
{
    return gb::potrf_impl<double>(uplo, n, A, lda, info, stream);
}

extern "C" int gb_spotrf(int uplo, int64_t n, float *A, int64_t lda, int64_t *info, void *stream)
{
    return gb::potrf_impl<float>(uplo, n, A, lda, info, stream);
}

// Diagonal-block step of the mixed-precision low-precision solve, done by
// inversion: each 128 x 128 lower-triangular diagonal block L_b is inverted
// once per solve (FP32, one CTA per block, triangle in shared memory), and
// every TS task of the refinement then applies X_b = L_b^-1 Y_b as a
// register-tiled FP32 triangular matrix product on CUDA cores, writing the
// FP32 result and its BF16 copy (the operand of the tensor-core updates).
// This turns the serial substitution on the critical path of the recursive
// model (Section V-A, the TS(i) leaves) into a fully parallel product.
//
// Storage ("band"): block b occupies band[(b*128 + c)*128 + i] = L_b(i, c),
// i.e. each block column-major with leading dimension 128.
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include "common.cuh"

namespace gb {
namespace {

constexpr int NBI = 128;

// One CTA (128 threads) per diagonal block: thread j forms column j of L^-1
// by forward substitution on e_j (row form, FP32, two partial sums).
__global__ void __launch_bounds__(NBI) invert_blocks_kernel(const float *__restrict__ band, float *__restrict__ inv)
{
    extern __shared__ __align__(16) float sm[];
    float *L = sm;                // L[i*NBI + k] = L(i,k)   (row-major for the dot form)
    float *X = sm + NBI * NBI;    // X[k*(NBI+1) + j] = Linv(k, j)
    const float *Lb = band + size_t(blockIdx.x) * NBI * NBI;
    float *Ib = inv + size_t(blockIdx.x) * NBI * NBI;
    const int j = threadIdx.x;
    for (int idx = j; idx < NBI * NBI; idx += NBI) {
        const int i = idx % NBI, c = idx / NBI;  // coalesced read of the column-major block
        L[i * NBI + c] = Lb[idx];
    }
    __syncthreads();
    for (int i = 0; i < NBI; i++) {
        float v = 0.f;
        if (i == j) v = 1.0f / L[i * NBI + i];
        else if (i > j) {
            float s0 = 0.f, s1 = 0.f;
            int k = j;
            for (; k + 1 < i; k += 2) {
                s0 = fmaf(L[i * NBI + k], X[k * (NBI + 1) + j], s0);
                s1 = fmaf(L[i * NBI + k + 1], X[(k + 1) * (NBI + 1) + j], s1);
            }
            if (k < i) s0 = fmaf(L[i * NBI + k], X[k * (NBI + 1) + j], s0);
            v = -(s0 + s1) / L[i * NBI + i];
        }
        X[i * (NBI + 1) + j] = v;
    }
    __syncthreads();
    for (int idx = j; idx < NBI * NBI; idx += NBI) {
        const int i = idx % NBI, c = idx / NBI;
        Ib[idx] = X[i * (NBI + 1) + c];
    }
}

// Y[b0:b0+nr, :] = Linv * Y[b0:b0+nr, :] for a block of nr <= 128 rows, in
// place (each CTA reads its whole 128 x 64 column panel before writing it),
// plus the BF16 copy.  256 threads, each an 8 x 4 register tile: rows
// ty*4 .. +3 and 64 + ty*4 .. +3, columns tx*4 .. +3.
constexpr int AC = 64;  // columns per CTA
// FP8 = true: instead of the BF16 copy, an FP8 (E4M3) copy Y8 with one
// power-of-two scale for the CTA's 128 x 64 block (written to *s8 + blockIdx.x).
template <bool FP8>
__global__ void __launch_bounds__(256)
apply_inverse_kernel(const float *__restrict__ Linv, float *__restrict__ Y, int64_t ldy,
                     __nv_bfloat16 *__restrict__ Ybf, int nr, int64_t ncols, uint8_t *__restrict__ Y8,
                     float *__restrict__ s8)
{
    extern __shared__ __align__(16) float sm[];
    float *Ls = sm;                 // Ls[k*NBI + i] = Linv(i, k)   (column k contiguous)
    float *Ys = sm + NBI * NBI;     // Ys[k*(AC+4) + c]            (row k contiguous)
    constexpr int LDY = AC + 4;
    const int tid = threadIdx.x;
    const int64_t c0 = int64_t(blockIdx.x) * AC;
    for (int idx = tid; idx < NBI * NBI / 4; idx += 256)
        reinterpret_cast<float4 *>(Ls)[idx] = reinterpret_cast<const float4 *>(Linv)[idx];
    for (int idx = tid; idx < NBI * AC; idx += 256) {
        const int i = idx % NBI, c = idx / NBI;  // Y column-major: contiguous along i
        float v = 0.f;
        if (i < nr && c0 + c < ncols) v = Y[i + (c0 + c) * ldy];
        Ys[i * LDY + c] = v;
    }
    __syncthreads();
    const int tx = tid & 15, ty = tid >> 4;
    const int r0 = ty * 4, r1 = 64 + ty * 4, cc = tx * 4;
    float acc[8][4];
#pragma unroll
    for (int r = 0; r < 8; r++)
#pragma unroll
        for (int c = 0; c < 4; c++) acc[r][c] = 0.f;
    // Linv is lower triangular: rows < 64 need k <= r0+3, rows >= 64 need all k <= r1+3
    const int kend_hi = r1 + 4;
    for (int k = 0; k < kend_hi; k++) {
        const float4 a0 = *reinterpret_cast<const float4 *>(&Ls[k * NBI + r0]);
        const float4 a1 = *reinterpret_cast<const float4 *>(&Ls[k * NBI + r1]);
        const float4 b = *reinterpret_cast<const float4 *>(&Ys[k * LDY + cc]);
        const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int r = 0; r < 8; r++)
#pragma unroll
            for (int c = 0; c < 4; c++) acc[r][c] = fmaf(av[r], bv[c], acc[r][c]);
    }
    __syncthreads();
    // results back through shared memory for coalesced column-major stores
#pragma unroll
    for (int r = 0; r < 8; r++) {
        const int i = r < 4 ? r0 + r : r1 + (r - 4);
#pragma unroll
        for (int c = 0; c < 4; c++) Ys[i * LDY + cc + c] = acc[r][c];
    }
    __syncthreads();
    float scale_inv = 1.f;
    if (FP8) {
        // block maximum -> power-of-two scale s with amax / s <= 448
        __shared__ float red[8];
        float mx = 0.f;
        for (int idx = tid; idx < NBI * AC; idx += 256) mx = fmaxf(mx, fabsf(Ys[(idx % NBI) * LDY + idx / NBI]));
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if ((tid & 31) == 0) red[tid >> 5] = mx;
        __syncthreads();
        mx = 0.f;
        for (int w = 0; w < 8; w++) mx = fmaxf(mx, red[w]);
        const float sc = mx > 0.f ? exp2f(ceilf(log2f(mx / 448.f))) : 1.f;
        scale_inv = 1.f / sc;
        if (tid == 0) s8[blockIdx.x] = sc;
    }
    for (int idx = tid; idx < NBI * AC; idx += 256) {
        const int i = idx % NBI, c = idx / NBI;
        if (i < nr && c0 + c < ncols) {
            const float v = Ys[i * LDY + c];
            Y[i + (c0 + c) * ldy] = v;
            if (FP8)
                Y8[i + (c0 + c) * ldy] = __nv_cvt_float_to_fp8(v * scale_inv, __NV_SATFINITE, __NV_E4M3);
            else
                Ybf[i + (c0 + c) * ldy] = __float2bfloat16_rn(v);
        }
    }
}

constexpr size_t INV_SMEM = size_t(NBI) * NBI * 4 + size_t(NBI) * (NBI + 1) * 4;
constexpr size_t APPLY_SMEM = size_t(NBI) * NBI * 4 + size_t(NBI) * (AC + 4) * 4;

}  // namespace

int diag_inv_prepare()
{
    static bool done = false;
    if (!done) {
        GB_CUDA(cudaFuncSetAttribute(invert_blocks_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)INV_SMEM));
        GB_CUDA(cudaFuncSetAttribute(apply_inverse_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)APPLY_SMEM));
        GB_CUDA(cudaFuncSetAttribute(apply_inverse_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)APPLY_SMEM));
        done = true;
    }
    return 0;
}

// Invert the nblocks diagonal blocks held in `band` into `inv` (same layout).
int launch_invert_blocks(const float *band, float *inv, int64_t nblocks, cudaStream_t s)
{
    if (nblocks <= 0) return 0;
    GB_TRY(diag_inv_prepare());
    LaunchScope ls(KK_DIAG, s, double(nblocks) * NBI * NBI * NBI / 3.0, 8.0 * nblocks * NBI * NBI);
    invert_blocks_kernel<<<(unsigned)nblocks, NBI, INV_SMEM, s>>>(band, inv);
    return check(cudaGetLastError());
}

// The TS task of one block: Y_b = Linv_b Y_b (+ BF16 copy).
int launch_apply_inverse(const float *Linv_b, float *Yb, int64_t ldy, __nv_bfloat16 *Ybf_b, int nr, int64_t ncols,
                         cudaStream_t s)
{
    if (nr <= 0 || ncols <= 0) return 0;
    if (nr > NBI) return GB_STATUS_CUDA_ERROR;
    GB_TRY(diag_inv_prepare());
    const int64_t grid = (ncols + AC - 1) / AC;
    LaunchScope ls(KK_DIAG, s, double(nr) * nr * ncols, 4.0 * (double(nr) * nr + 2.0 * nr * ncols) + 2.0 * nr * ncols);
    apply_inverse_kernel<false><<<(unsigned)grid, 256, APPLY_SMEM, s>>>(Linv_b, Yb, ldy, Ybf_b, nr, ncols,
                                                                         nullptr, nullptr);
    return check(cudaGetLastError());
}

// As above, emitting the FP8 copy Y8_b (same layout) and the block scales
// s8_b[j] of the 128 x 64 blocks j = 0, 1, ... of this row block.
int launch_apply_inverse_fp8(const float *Linv_b, float *Yb, int64_t ldy, uint8_t *Y8_b, float *s8_b, int nr,
                             int64_t ncols, cudaStream_t s)
{
    if (nr <= 0 || ncols <= 0) return 0;
    if (nr > NBI) return GB_STATUS_CUDA_ERROR;
    GB_TRY(diag_inv_prepare());
    const int64_t grid = (ncols + AC - 1) / AC;
    LaunchScope ls(KK_DIAG, s, double(nr) * nr * ncols, 4.0 * (double(nr) * nr + 2.0 * nr * ncols) + 1.0 * nr * ncols);
    apply_inverse_kernel<true><<<(unsigned)grid, 256, APPLY_SMEM, s>>>(Linv_b, Yb, ldy, nullptr, nr, ncols, Y8_b,
                                                                        s8_b);
    return check(cudaGetLastError());
}

}  // namespace gb

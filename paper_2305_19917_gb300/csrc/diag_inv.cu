// Diagonal-block step of the mixed-precision low-precision solve, done by
// inversion: each 128 x 128 lower-triangular diagonal block L_b is inverted
// once per solve (FP32, one CTA per block, triangle in shared memory) into
// FP32 strips and a two-term BF16 split, and every TS task of the
// refinement then applies X_b = L_b^-1 Y_b as a product: on the tensor cores
// from the BF16 split (apply_tc.cu), or, in the FP8 form, here as a
// register-tiled FP32 triangular product on the CUDA cores that also writes
// the FP8 copy with its block scales.  This turns the serial substitution on
// the critical path of the recursive model (Section V-A, the TS(i) leaves)
// into a fully parallel product.
//
// Storage ("band"): block b occupies band[(b*128 + c)*128 + i] = L_b(i, c),
// i.e. each block column-major with leading dimension 128.  The inverses use
// a packed "strip" layout in the same 128*128-float slot per block: strip g
// (g = 0..31) holds rows 4g..4g+3 of L_b^-1 for the columns k = 0..4g+3 it can
// be nonzero in, element (4g+j, k) at strip_off(g) + 4k + j.  That keeps the
// lower triangle only (33 KB instead of 64 KB in shared memory) and gives
// each thread's four rows of one column as one 16-byte vector.
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include "common.cuh"

namespace gb {
namespace {

constexpr int NBI = 128;

// Ampere-style asynchronous global -> shared copies (no register staging).
__device__ __forceinline__ void cp_async16(float *dst, const float *src)
{
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
// copies 4 bytes, or writes zero when `in` is false (source size 0)
__device__ __forceinline__ void cp_async4_zfill(float *dst, const float *src, bool in)
{
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
    const int n = in ? 4 : 0;
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

constexpr int NSTRIP = NBI / 4;
constexpr int STRIP_FLOATS = 8 * NSTRIP * (NSTRIP + 1);  // 8448
__host__ __device__ constexpr int strip_off(int g) { return 8 * g * (g + 1); }

// One CTA (128 threads) per diagonal block: thread j forms column j of L^-1
// by forward substitution on e_j (row form, FP32, two partial sums).
__global__ void __launch_bounds__(NBI) invert_blocks_kernel(const float *__restrict__ band, float *__restrict__ inv,
                                                            __nv_bfloat16 *__restrict__ inv16, int64_t kp)
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
    // strip layout (the zeros above the diagonal inside each 4 x 4 diagonal
    // piece are stored explicitly)
    for (int g = 0; g < NSTRIP; g++) {
        const int cnt = (4 * g + 4) * 4;
        for (int e = j; e < cnt; e += NBI) Ib[strip_off(g) + e] = X[(4 * g + (e & 3)) * (NBI + 1) + (e >> 2)];
    }
    // two-term BF16 split L^-1 = hi + lo, row-major (K-major for the tensor
    // cores): hi rows at block*128 + i, lo rows at kp + block*128 + i
    if (inv16) {
        const int64_t r0 = int64_t(blockIdx.x) * NBI;
        for (int idx = j; idx < NBI * NBI; idx += NBI) {
            const int i = idx / NBI, k = idx % NBI;
            const float x = X[i * (NBI + 1) + k];
            const __nv_bfloat16 h = __float2bfloat16_rn(x);
            inv16[(r0 + i) * NBI + k] = h;
            inv16[(kp + r0 + i) * NBI + k] = __float2bfloat16_rn(x - __bfloat162float(h));
        }
    }
}

// Y[b0:b0+nr, :] = Linv * Y[b0:b0+nr, :] for a block of nr <= 128 rows, in
// place (each CTA reads its whole 128 x 64 column panel before writing it),
// plus the BF16 (or FP8) copy.  256 threads over a 128 x 64 panel; thread
// (tx, ty) = (tid % 16, tid / 16) owns the columns tx, tx+16, tx+32, tx+48
// and the eight rows 4ty .. 4ty+3 and 124-4ty .. 127-4ty.  Pairing a low and
// a high row group makes every thread's share of the triangle the same: rows
// 4ty.. need k < 4ty+4 and rows 124-4ty.. need k < 128-4ty, so each thread
// does 2112 FMAs, and the two row-group pairs of one warp differ by only
// four iterations.  The panel keeps Y's column-major layout in shared memory
// with an odd column stride: staging stores and operand reads are free of
// bank conflicts (the 16 column owners of a warp hit 16 distinct banks; the
// two row groups share each address).  Results go straight from registers
// to global memory.
constexpr int AC = 64;
constexpr int LDC = NBI + 1;  // shared column stride of the panel
// FP8 = true: instead of the BF16 copy, an FP8 (E4M3) copy
// Y8 with one power-of-two scale for the CTA's 128 x 64 block (written to
// s8[blockIdx.x]).
template <bool FP8>
__global__ void __launch_bounds__(4 * AC)
apply_inverse_kernel(const float *__restrict__ Linv, float *__restrict__ Y, int64_t ldy,
                     __nv_bfloat16 *__restrict__ Ybf, int nr, int64_t ncols, uint8_t *__restrict__ Y8,
                     float *__restrict__ s8)
{
    extern __shared__ __align__(16) float sm[];
    float *Ls = sm;                 // strips of Linv
    float *Ys = sm + STRIP_FLOATS;  // Ys[c*LDC + i]   (column c contiguous)
    constexpr int nthr = 4 * AC;
    const int tid = threadIdx.x;
    const int64_t c0 = int64_t(blockIdx.x) * AC;
    // all staging loads go out as asynchronous copies before the one wait
    for (int idx = tid; idx < STRIP_FLOATS / 4; idx += nthr) cp_async16(Ls + 4 * idx, Linv + 4 * idx);
    // 128 * AC = 32 * nthr elements; consecutive threads take consecutive rows
#pragma unroll 8
    for (int it = 0; it < 32; it++) {
        const int idx = tid + it * nthr;
        const int i = idx & (NBI - 1), c = idx >> 7;
        const bool in = i < nr && c0 + c < ncols;
        cp_async4_zfill(Ys + c * LDC + i, in ? Y + i + (c0 + c) * ldy : Y, in);
    }
    cp_async_wait_all();
    __syncthreads();
    const int tx = tid & 15, ty = tid >> 4;
    const int rlo = 4 * ty, rhi = NBI - 4 - 4 * ty;
    const float *S0 = Ls + strip_off(ty);
    const float *S1 = Ls + strip_off(NSTRIP - 1 - ty);
    const float *yb = Ys + tx * LDC;  // column tx + 16c at yb + 16c*LDC
    float acc[8][4];
#pragma unroll
    for (int r = 0; r < 8; r++)
#pragma unroll
        for (int c = 0; c < 4; c++) acc[r][c] = 0.f;
    int k = 0;
#pragma unroll 2
    for (; k < rlo + 4; k++) {
        const float4 a0 = *reinterpret_cast<const float4 *>(S0 + 4 * k);
        const float4 a1 = *reinterpret_cast<const float4 *>(S1 + 4 * k);
        const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        float bv[4];
#pragma unroll
        for (int c = 0; c < 4; c++) bv[c] = yb[16 * c * LDC + k];
#pragma unroll
        for (int r = 0; r < 8; r++)
#pragma unroll
            for (int c = 0; c < 4; c++) acc[r][c] = fmaf(av[r], bv[c], acc[r][c]);
    }
#pragma unroll 4
    for (; k < rhi + 4; k++) {
        const float4 a1 = *reinterpret_cast<const float4 *>(S1 + 4 * k);
        const float av[4] = {a1.x, a1.y, a1.z, a1.w};
        float bv[4];
#pragma unroll
        for (int c = 0; c < 4; c++) bv[c] = yb[16 * c * LDC + k];
#pragma unroll
        for (int r = 0; r < 4; r++)
#pragma unroll
            for (int c = 0; c < 4; c++) acc[4 + r][c] = fmaf(av[r], bv[c], acc[4 + r][c]);
    }
    float scale_inv = 1.f;
    if (FP8) {
        // block maximum -> power-of-two scale s with amax / s <= 448
        __shared__ float red[nthr / 32];
        float mx = 0.f;
#pragma unroll
        for (int h = 0; h < 2; h++)
#pragma unroll
            for (int r = 0; r < 4; r++)
#pragma unroll
                for (int c = 0; c < 4; c++)
                    if ((h ? rhi : rlo) + r < nr && c0 + tx + 16 * c < ncols)
                        mx = fmaxf(mx, fabsf(acc[4 * h + r][c]));
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if ((tid & 31) == 0) red[tid >> 5] = mx;
        __syncthreads();
        mx = 0.f;
        for (int w = 0; w < nthr / 32; w++) mx = fmaxf(mx, red[w]);
        const float sc = mx > 0.f ? exp2f(ceilf(log2f(mx / 448.f))) : 1.f;
        scale_inv = 1.f / sc;
        if (tid == 0) s8[blockIdx.x] = sc;
    }
#pragma unroll
    for (int c = 0; c < 4; c++) {
        const int64_t col = c0 + tx + 16 * c;
        if (col >= ncols) continue;
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int r0 = h ? rhi : rlo;
            const float *a = acc[4 * h];
            const float v0 = a[0 * 4 + c], v1 = a[1 * 4 + c], v2 = a[2 * 4 + c], v3 = a[3 * 4 + c];
            const int64_t o = r0 + col * ldy;
            if (r0 + 3 < nr) {
                *reinterpret_cast<float4 *>(&Y[o]) = make_float4(v0, v1, v2, v3);
                if (FP8) {
                    const uint32_t q0 = __nv_cvt_float_to_fp8(v0 * scale_inv, __NV_SATFINITE, __NV_E4M3);
                    const uint32_t q1 = __nv_cvt_float_to_fp8(v1 * scale_inv, __NV_SATFINITE, __NV_E4M3);
                    const uint32_t q2 = __nv_cvt_float_to_fp8(v2 * scale_inv, __NV_SATFINITE, __NV_E4M3);
                    const uint32_t q3 = __nv_cvt_float_to_fp8(v3 * scale_inv, __NV_SATFINITE, __NV_E4M3);
                    *reinterpret_cast<uint32_t *>(&Y8[o]) = q0 | (q1 << 8) | (q2 << 16) | (q3 << 24);
                } else {
                    __nv_bfloat162 p0 = __floats2bfloat162_rn(v0, v1), p1 = __floats2bfloat162_rn(v2, v3);
                    uint2 w;
                    w.x = *reinterpret_cast<uint32_t *>(&p0);
                    w.y = *reinterpret_cast<uint32_t *>(&p1);
                    *reinterpret_cast<uint2 *>(&Ybf[o]) = w;
                }
            } else {
                const float vv[4] = {v0, v1, v2, v3};
#pragma unroll
                for (int r = 0; r < 4; r++)
                    if (r0 + r < nr) {
                        Y[o + r] = vv[r];
                        if (FP8) Y8[o + r] = __nv_cvt_float_to_fp8(vv[r] * scale_inv, __NV_SATFINITE, __NV_E4M3);
                        else Ybf[o + r] = __float2bfloat16_rn(vv[r]);
                    }
            }
        }
    }
}

constexpr size_t INV_SMEM = size_t(NBI) * NBI * 4 + size_t(NBI) * (NBI + 1) * 4;
constexpr size_t apply_smem(int ac) { return size_t(STRIP_FLOATS) * 4 + size_t(ac) * LDC * 4; }

}  // namespace

int diag_inv_prepare()
{
    static PerDeviceOnce inv_attr, apply_attr;
    GB_TRY(smem_attr_once(inv_attr, invert_blocks_kernel, INV_SMEM));
    return smem_attr_once(apply_attr, apply_inverse_kernel<true>, apply_smem(AC));
}

// Invert the nblocks diagonal blocks held in `band` into `inv` (strips) and,
// when inv16 is given, into its two-term BF16 split (2 x kp x 128, kp =
// 128 * nblocks rows of 128).
int launch_invert_blocks(const float *band, float *inv, __nv_bfloat16 *inv16, int64_t nblocks, cudaStream_t s)
{
    if (nblocks <= 0) return 0;
    GB_TRY(diag_inv_prepare());
    LaunchScope ls(KK_DIAG, s, double(nblocks) * NBI * NBI * NBI / 3.0, 8.0 * nblocks * NBI * NBI);
    invert_blocks_kernel<<<(unsigned)nblocks, NBI, INV_SMEM, s>>>(band, inv, inv16, int64_t(nblocks) * NBI);
    return check(cudaGetLastError());
}

// The TS task of one block of the FP8 form: Y_b = Linv_b Y_b in FP32 on the
// CUDA cores, plus the FP8 copy Y8_b (same layout) and the block scales
// s8_b[j] of the 128 x 64 blocks j = 0, 1, ... of this row block (the BF16
// form applies the inverse on the tensor cores, apply_tc.cu).
int launch_apply_inverse_fp8(const float *Linv_b, float *Yb, int64_t ldy, uint8_t *Y8_b, float *s8_b, int nr,
                             int64_t ncols, cudaStream_t s)
{
    if (nr <= 0 || ncols <= 0) return 0;
    if (nr > NBI) return GB_STATUS_CUDA_ERROR;
    GB_TRY(diag_inv_prepare());
    if (ldy % 4 || (reinterpret_cast<uintptr_t>(Yb) & 15) || (reinterpret_cast<uintptr_t>(Y8_b) & 3))
        return GB_STATUS_CUDA_ERROR;
    const int64_t grid = (ncols + AC - 1) / AC;
    LaunchScope ls(KK_DIAG, s, double(nr) * nr * ncols, 4.0 * (double(nr) * nr + 2.0 * nr * ncols) + 1.0 * nr * ncols);
    apply_inverse_kernel<true><<<(unsigned)grid, 4 * AC, apply_smem(AC), s>>>(Linv_b, Yb, ldy, nullptr, nr, ncols,
                                                                               Y8_b, s8_b);
    return check(cudaGetLastError());
}

}  // namespace gb

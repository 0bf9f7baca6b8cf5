// Mixed-precision triangular solve with iterative refinement:
//
//   X0  = low-precision solve of Mv X = alpha*Bv   (BF16 tensor-core GEMM
//         updates with FP32 accumulation; the recursive model of Section
//         V-A down to 1024-row leaves, each solved by one tensor-core kernel
//         launch in 128-row blocks with precomputed FP32 block inverses)
//   repeat:  R = alpha*Bv - Mv X  (split-precision products on the tensor
//            cores, exact integer sums, FP64 final accumulation)
//            D = low-precision solve of Mv D = R;   X += D  (FP64)
//   until ||D||_F <= tol ||X||_F.
//
// The residual is carried incrementally: after X += D~ (D~ = D rounded to
// the two 8-bit digits per column that the residual kernel consumes),
// R -= Mv D~, so R stays the residual of the X actually held.  Mv is cut
// without its diagonal into six 8-bit digit slices with a power-of-two
// scale per row (48 bits of the largest off-diagonal entry); the diagonal
// term is applied exactly in FP64;
// the number of slice pairs formed shrinks as the corrections shrink.
//
// Everything is done on a canonical FORWARD problem in column-major layout:
// a backward (upper) problem is index-reversed, a right-side problem is
// transposed, both while copying in, and the result is mapped back at the
// end.  Each right-hand side is scaled by a power of two (exact) that brings
// its largest entry near 1 for the FP32 / BF16 solve, and scaled back when
// written.  Sizes are padded to multiples of 128 (identity on the padded
// diagonal, zero right-hand sides), so every tile is aligned for TMA.
#include <cmath>
#include <cstddef>
#include <algorithm>
#include <mutex>
#include <cstdio>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include "common.cuh"
#include "driver.cuh"
#include "mixed.cuh"

namespace gb {

int launch_tc_gemm_bf16(int64_t M, int64_t N, int64_t K, const void *A, int64_t lda, const void *B,
                        int64_t ldb, float *C, int64_t ldc, float alpha, cudaStream_t s, int *status);
int launch_tc_residual(long long *Tg, int64_t ldr, const void *As, const void *Zs, int64_t kp, int64_t np,
                       int64_t k_lo, int64_t k_hi, int P, int P2, cudaStream_t s, int *status);
int residual_weight(int P, int P2);
int tc_gemm_prepare();
int tc_gemm_fp8_prepare();
int launch_tc_gemm_fp8(int64_t M, int64_t N, int64_t K, const void *A, int64_t lda, const void *B, int64_t ldb,
                       float *C, int64_t ldc, float alpha, const float *sA, int64_t ldsa, const float *sB,
                       int64_t ldsb, cudaStream_t s, int *status);
int launch_apply_inverse_fp8(const float *Linv_b, float *Yb, int64_t ldy, uint8_t *Y8_b, float *s8_b, int nr,
                             int64_t ncols, cudaStream_t s);
int diag_inv_prepare();
int launch_invert_blocks(const float *band, float *inv, __nv_bfloat16 *inv16, int64_t nblocks, cudaStream_t s);
int apply_tc_prepare();
int launch_leaf_tc(const __nv_bfloat16 *Abf, const __nv_bfloat16 *inv16, int64_t kp, int64_t np, int64_t s0,
                   int64_t nr, float *Y, __nv_bfloat16 *Ybf, cudaStream_t s, int *status);
namespace {

constexpr int kSlices = 6;     // digit slices of Mv (8 bits each)
// The corrections of the first kZSlots refinement steps are kept as their
// digit slices (z_1, z_2 and the column exponents) and X = D_0 + D_1 + ... is
// formed only when the solution is written back (their exact sum, rounded
// once); a longer refinement folds them into an FP64 X once and updates X in
// place from then on.
constexpr int kZSlots = 3;
constexpr int kBand = 128;     // FP32 band of diagonal 128-blocks (column-major per block)
constexpr int kLeaf = 1024;    // default leaf order of the BF16 low-precision solve (one leaf kernel launch each)

// Library fallback of the integer-built conversions below, for results
// outside the normal double range.  Kept out of line: inlined, the compiler
// may evaluate it on every element (its int -> double conversion and scaling
// run on the FP64 pipe) and select the result afterwards.
__device__ __noinline__ double ldexp_i64_slow(long long t, int e) { return ldexp(static_cast<double>(t), e); }

// z * 2^e as a double for |z| < 2^31 (exact: no rounding), built with 32-bit
// integer operations (an int -> double conversion runs on the FP64 pipe,
// which retires two operations per clock and SM); results outside the
// normal range take the library path.
__device__ __forceinline__ double scaled_i32_to_f64(int z, int e)
{
    if (z == 0) return 0.0;
    const unsigned sign = z < 0 ? 0x80000000u : 0u;
    const unsigned u = z < 0 ? 0u - unsigned(z) : unsigned(z);
    const int lz = __clz(int(u));
    const int ex = 31 - lz + e;
    if (ex < -1022 || ex > 1023) return ldexp_i64_slow(z, e);
    const unsigned m = (lz == 31) ? 0u : (u << (lz + 1));  // fraction bits below the leading one
    const unsigned hi = sign | (unsigned(ex + 1023) << 20) | (m >> 12);
    const unsigned lo = m << 20;
    return __hiloint2double(int(hi), int(lo));
}

// T * 2^e rounded to the nearest double (ties to even), i.e. the value of
// ldexp((double)T, e), for |T| < 2^63, built with integer operations (the
// FP64 pipe retires two operations per clock and SM); results outside the
// normal exponent range take the library path.
__device__ __forceinline__ double scaled_i64_to_f64(long long T, int e)
{
    if (T == 0) return 0.0;
    const unsigned long long sign = T < 0 ? (1ull << 63) : 0ull;
    const unsigned long long u = T < 0 ? 0ull - static_cast<unsigned long long>(T) : static_cast<unsigned long long>(T);
    const int lz = __clzll(static_cast<long long>(u));
    int msb = 63 - lz;
    const unsigned long long m = u << lz;  // leading one at bit 63
    unsigned long long keep = m >> 11;     // 53 significant bits
    const unsigned long long rem = m & 0x7FFull;
    if (rem > 0x400ull || (rem == 0x400ull && (keep & 1ull))) keep++;
    if (keep >> 53) {  // rounded up to the next power of two
        keep >>= 1;
        msb++;
    }
    const int ex = msb + e;
    if (ex < -1022 || ex > 1023) return ldexp_i64_slow(T, e);
    return __longlong_as_double(static_cast<long long>(sign | (static_cast<unsigned long long>(ex + 1023) << 52) |
                                                       (keep & ((1ull << 52) - 1))));
}

// x rounded to the nearest float (ties to even), as __double2float_rn(x),
// from the bit pattern with integer operations only (no FP64 instruction),
// subnormal, overflowing and non-finite cases included.
__device__ __forceinline__ float f64_to_f32_rn(double x)
{
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
    const unsigned int sign = static_cast<unsigned int>(b >> 32) & 0x80000000u;
    const int E = int((b >> 52) & 0x7FF);
    const unsigned long long mant = b & ((1ull << 52) - 1);
    if (E >= 1023 - 126) {  // a normal float or beyond
        if (E == 0x7FF) return __uint_as_float(sign | 0x7F800000u | (mant ? 0x00400000u : 0u));
        if (E > 1023 + 127) return __uint_as_float(sign | 0x7F800000u);
        unsigned int keep = static_cast<unsigned int>(mant >> 29);
        const unsigned long long rem = mant & ((1ull << 29) - 1);
        if (rem > (1ull << 28) || (rem == (1ull << 28) && (keep & 1u))) keep++;
        // a carry out of the mantissa moves into the exponent field, as it must
        return __uint_as_float((sign | (static_cast<unsigned int>(E - 1023 + 127) << 23)) + keep);
    }
    // a subnormal float: round(M 2^(E - 1075 + 149)) units of 2^-149, M the
    // 53-bit significand (zero below a quarter unit; double subnormals too)
    const int r = 926 - E;
    if (E == 0 || r >= 55) return __uint_as_float(sign);
    const unsigned long long M = mant | (1ull << 52);
    unsigned long long q = M >> r;
    const unsigned long long rem = M & ((1ull << r) - 1), half = 1ull << (r - 1);
    if (rem > half || (rem == half && (q & 1ull))) q++;
    return __uint_as_float(sign | static_cast<unsigned int>(q));
}

// Canonical forward view of the user problem (device-side description).
struct View {
    const double *A;
    int64_t lda;
    bool mt;       // Mv(i,c) = A(c,i)
    bool rev;      // index reversal (backward problem)
    bool unit;
    int64_t k;     // order of Mv
};

// Mv'(i,c) of the forward view: lower triangle (c <= i), 1 on a unit or
// padded diagonal, 0 elsewhere.
__device__ __forceinline__ double mvp(const View &v, int64_t i, int64_t c)
{
    if (c > i) return 0.0;
    if (i >= v.k || c >= v.k) return (i == c) ? 1.0 : 0.0;
    if (i == c && v.unit) return 1.0;
    int64_t r = v.rev ? v.k - 1 - i : i;
    int64_t s = v.rev ? v.k - 1 - c : c;
    return v.mt ? v.A[s + r * v.lda] : v.A[r + s * v.lda];
}
// Which index of Mv' runs along A's contiguous dimension: true = i.
__device__ __forceinline__ bool contig_i(const View &v) { return !v.mt; }

// The 16 entries of the 64 x 64 tile (i0.., c0..) of Mv' that thread tid of
// 256 reads along A's contiguous dimension: entry u is (li, lc) with the
// fast index tid & 63 and the slow one (tid >> 6) + 4u (li fast when
// contig_i).  All 16 loads are issued before any is used.
__device__ __forceinline__ void load_vals(const View &v, int64_t i0, int64_t c0, double (&val)[16])
{
    const int tid = threadIdx.x;
    const bool ci = contig_i(v);
    if (c0 + 63 < i0 && i0 + 63 < v.k) {
        // a tile strictly below the diagonal and inside the matrix: entry
        // (fast, slow) sits at base + s fast + s lda slow (s = -1 reversed),
        // with the contiguous index of A along fast
        const int64_t x0 = ci ? i0 : c0, y0 = ci ? c0 : i0;
        const int64_t sg = v.rev ? -1 : 1;
        const int64_t base = v.rev ? (v.k - 1 - x0) + (v.k - 1 - y0) * v.lda : x0 + y0 * v.lda;
        const double *p = v.A + base + sg * ((tid & 63) + int64_t(tid >> 6) * v.lda);
        const int64_t step = 4 * sg * v.lda;
#pragma unroll
        for (int u = 0; u < 16; u++) val[u] = p[u * step];
        return;
    }
#pragma unroll
    for (int u = 0; u < 16; u++) {
        const int fast = tid & 63, slow = (tid >> 6) + 4 * u;
        val[u] = mvp(v, i0 + (ci ? fast : slow), c0 + (ci ? slow : fast));
    }
}

// Load the 64 x 64 tile (i0.., c0..) of Mv' into shared memory t[64][65],
// reading A along its contiguous dimension.
__device__ void load_tile(const View &v, int64_t i0, int64_t c0, double (*t)[65])
{
    const int tid = threadIdx.x;  // 256 threads
    const bool ci = contig_i(v);
    double val[16];
    load_vals(v, i0, c0, val);
#pragma unroll
    for (int u = 0; u < 16; u++) {
        const int fast = tid & 63, slow = (tid >> 6) + 4 * u;
        t[ci ? fast : slow][ci ? slow : fast] = val[u];
    }
}

// Tiles that are needed: every 64x64 tile with c0 < end of the 128-row
// diagonal block of i0 (the residual kernel reads up to that column).
__device__ __forceinline__ bool tile_needed(int64_t i0, int64_t c0) { return c0 < ((i0 >> 7) << 7) + 128; }

// Biased binary exponent field of a double (0 for zero / subnormal).
__device__ __forceinline__ int bexp(double a)
{
    return int((static_cast<unsigned long long>(__double_as_longlong(a)) >> 52) & 0x7FF);
}

// Pass 1: row exponents.  e_i = E + 2 where 2^E <= max_{c<i} |Mv'(i,c)| <
// 2^(E+1), so every strictly-lower entry satisfies |a| < 2^(e_i - 1): the
// strictly lower part only, so that small off-diagonal entries keep all their
// digits when the diagonal is much larger (the diagonal is applied exactly in
// FP64 by the residual kernel).  Integer arithmetic on the exponent fields.
// With bmax != nullptr also the maxima |a| of the strictly-lower 128 x 128
// blocks (as FP32 bit patterns, which order like the values), for the FP8
// block scales.
__global__ void __launch_bounds__(256) rowexp_kernel(View v, int64_t kp, int *e_row, unsigned *bmax)
{
    __shared__ int rmax[64];
    __shared__ float red[8];
    const int64_t i0 = int64_t(blockIdx.y) * 64, c0 = int64_t(blockIdx.x) * 64;
    if (c0 > i0 + 63) return;
    const int tid = threadIdx.x;
    if (tid < 64) rmax[tid] = 0;
    double val[16];
    load_vals(v, i0, c0, val);
    __syncthreads();
    const int fast = tid & 63;
    if (contig_i(v)) {  // the thread's 16 entries share row fast
        int mx = 0;
#pragma unroll
        for (int u = 0; u < 16; u++)
            if (c0 + (tid >> 6) + 4 * u != i0 + fast) mx = max(mx, bexp(val[u]));
        if (mx > 0) atomicMax(&rmax[fast], mx);
    } else {
#pragma unroll
        for (int u = 0; u < 16; u++) {
            const int li = (tid >> 6) + 4 * u;
            const int b = bexp(val[u]);
            if (c0 + fast != i0 + li && b > 0) atomicMax(&rmax[li], b);
        }
    }
    __syncthreads();
    if (tid < 64 && rmax[tid] > 0) atomicMax(&e_row[i0 + tid], rmax[tid] - 1023 + 2);
    if (bmax && (c0 >> 7) < (i0 >> 7)) {
        float m = 0.f;
#pragma unroll
        for (int u = 0; u < 16; u++) m = fmaxf(m, fabsf(float(val[u])));
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if ((tid & 31) == 0) red[tid >> 5] = m;
        __syncthreads();
        if (tid == 0) {
            for (int w = 1; w < 8; w++) m = fmaxf(m, red[w]);
            atomicMax(&bmax[(i0 >> 7) * (kp >> 7) + (c0 >> 7)], __float_as_uint(m));
        }
    }
}

// Power-of-two FP8 block scales s = 2^ceil(log2(amax / 448)) (1 for zero
// blocks), so that every scaled entry fits E4M3's largest finite value.
__global__ void block_scales_kernel(const unsigned *bmax, float *bscale, int64_t nb)
{
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < nb; i += int64_t(gridDim.x) * blockDim.x) {
        const float m = __uint_as_float(bmax[i]);
        bscale[i] = m > 0.f ? exp2f(ceilf(log2f(m / 448.f))) : 1.f;
    }
}

// The 48-bit fixed-point value N = round(a 2^(48-e)) of |a| < 2^(e-1)
// (|N| <= 2^47), computed from the bit pattern with integer operations.
__device__ __forceinline__ long long fixed48(double a, int e)
{
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(a));
    const int E = int((b >> 52) & 0x7FF);
    if (E == 0) return 0;  // zero (subnormals are far below 2^-48 of any row scale)
    const unsigned long long mant = (b & ((1ull << 52) - 1)) | (1ull << 52);  // a = mant 2^(E-1075)
    // a 2^(48-e) = mant 2^(E - 1075 + 48 - e): right shift by r = 1027 + e - E
    const int r = 1027 + e - E;
    long long n;
    if (r >= 63) n = 0;
    else if (r <= 0) n = (long long)(mant << (-r));  // cannot happen for |a| < 2^(e-1)
    else n = (long long)((mant + (1ull << (r - 1))) >> r);
    return (b >> 63) ? -n : n;
}

// Balanced base-256 digit of x: the d in [-128, 127] with d = x (mod 256).
__device__ __forceinline__ int bal8(int x) { return ((x + 128) & 255) - 128; }
// The FP32 bit pattern of an integer |d| < 2^22, exactly: d added to the
// integer bits of 1.5 2^23 adds d to that value, which is then subtracted.
__device__ __forceinline__ uint32_t small_int_f32bits(int d)
{
    return __float_as_uint(__int_as_float(0x4B400000 + d) - 12582912.0f);
}
// Two BF16 in one word from FP32 patterns whose low 16 bits are zero (the
// high halves are then the BF16 values exactly): lo_elem first.
__device__ __forceinline__ uint32_t pack_hi16(uint32_t lo_elem, uint32_t hi_elem)
{
    return __byte_perm(lo_elem, hi_elem, 0x7632);
}
// Round-to-nearest-even BF16 bit pattern of a double, from the two 32-bit
// halves of its bit pattern (as d2bf16: results below the BF16 normal range
// flush to zero, overflow gives infinity, NaN stays NaN).
__device__ __forceinline__ uint32_t d2bf16_bits(double a)
{
    const uint32_t hi = uint32_t(__double2hiint(a)), lo = uint32_t(__double2loint(a));
    const uint32_t s = (hi >> 16) & 0x8000u;
    const int E = int((hi >> 20) & 0x7FFu);
    if (E == 0x7FF) return s | 0x7F80u | (((hi & 0xFFFFFu) | lo) ? 0x40u : 0u);
    const int e = E - 1023 + 127;
    if (E == 0 || e <= 0) return s;
    uint32_t m7 = (hi >> 13) & 0x7Fu;        // mantissa bits 51..45
    const uint32_t rem = hi & 0x1FFFu;       // bits 44..32 (bits 31..0 in lo)
    if (rem > 0x1000u || (rem == 0x1000u && (lo != 0u || (m7 & 1u)))) m7++;
    uint32_t r = (uint32_t(e) << 7) + m7;    // a carry out of m7 raises the exponent
    if (r >= 0x7F80u) r = 0x7F80u;
    return s | r;
}

// Pass 2: BF16 copy (round to nearest), the 6 digit slices of the strictly
// lower part, the FP64 diagonal and the FP32 band of diagonal 64-blocks.
// Thread tid takes 8 consecutive columns (8 (tid & 7) ..) of rows
// (tid >> 3) and (tid >> 3) + 32 of the tile, so that every row-major output
// is written 16 bytes at a time.
__global__ void __launch_bounds__(256)
prepA_kernel(View v, int64_t kp, const int *e_row, __nv_bfloat16 *Abf, __nv_bfloat16 *As, float *band,
             double *dg, uint8_t *A8, const float *bscale)
{
    __shared__ double t[64][65];
    const int64_t i0 = int64_t(blockIdx.y) * 64, c0 = int64_t(blockIdx.x) * 64;
    if (!tile_needed(i0, c0)) return;
    load_tile(v, i0, c0, t);
    __syncthreads();
    const int tid = threadIdx.x;
    const size_t slice = size_t(kp) * size_t(kp);
    const int lc0 = (tid & 7) * 8;
    const int64_t c8 = c0 + lc0;
#pragma unroll 1
    for (int pass = 0; pass < 2; pass++) {
        const int li = (tid >> 3) + 32 * pass;
        const int64_t i = i0 + li;
        const int e = e_row[i];
        const size_t off = size_t(i) * size_t(kp) + size_t(c8);
        uint32_t wbf[4], wd[kSlices][4];
        uint32_t w8[2] = {0u, 0u};
        const bool fp8 = A8 && (c8 >> 7) < (i >> 7);
        const float sc = fp8 ? bscale[(i >> 7) * (kp >> 7) + (c8 >> 7)] : 1.f;
#pragma unroll
        for (int u = 0; u < 8; u += 2) {
            uint32_t hb[2], dig[2][kSlices];
#pragma unroll
            for (int v2 = 0; v2 < 2; v2++) {
                const int64_t c = c8 + u + v2;
                const double a = t[li][lc0 + u + v2];
                hb[v2] = d2bf16_bits(a);
                if (fp8) {
                    const unsigned q = __nv_cvt_float_to_fp8(f64_to_f32_rn(a) / sc, __NV_SATFINITE, __NV_E4M3);
                    w8[(u + v2) >> 2] |= q << (8 * ((u + v2) & 3));
                }
                // balanced base-256 digits of N = round(a 2^(48-e)): N = sum_p q_p 256^(5-p),
                // q_p in [-128, 127] for p >= 1 (least significant first), the top one
                // q_0 in [-128, 128]; in 32-bit halves: the low 24 bits give q_5..q_3
                // and a carry into the high part, which gives q_2..q_0
                const long long N = (c == i) ? 0 : fixed48(a, e);
                if (c == i) dg[i] = a;
                int x = int(uint32_t(N) & 0xFFFFFFu);
#pragma unroll
                for (int p = kSlices - 1; p >= 3; p--) {
                    const int d = bal8(x);
                    dig[v2][p] = small_int_f32bits(d);
                    x = (x - d) >> 8;
                }
                int y = int(N >> 24) + x;
#pragma unroll
                for (int p = 2; p >= 1; p--) {
                    const int d = bal8(y);
                    dig[v2][p] = small_int_f32bits(d);
                    y = (y - d) >> 8;
                }
                dig[v2][0] = small_int_f32bits(y);  // top digit, |y| <= 128
                if (c / kBand == i / kBand) band[size_t(c) * kBand + (i % kBand)] = f64_to_f32_rn(a);
            }
            wbf[u >> 1] = hb[0] | (hb[1] << 16);
#pragma unroll
            for (int p = 0; p < kSlices; p++) wd[p][u >> 1] = pack_hi16(dig[0][p], dig[1][p]);
        }
        *reinterpret_cast<uint4 *>(Abf + off) = make_uint4(wbf[0], wbf[1], wbf[2], wbf[3]);
#pragma unroll
        for (int p = 0; p < kSlices; p++)
            *reinterpret_cast<uint4 *>(As + p * slice + off) = make_uint4(wd[p][0], wd[p][1], wd[p][2], wd[p][3]);
        if (fp8) *reinterpret_cast<uint2 *>(A8 + off) = make_uint2(w8[0], w8[1]);
    }
}

// R = alpha * Bv' (forward view of the right-hand sides), zero padded.
// Left: Bv(i,j) = B(i,j); Right: Bv(i,j) = B(j,i); reversal on i.
// ---- right-hand sides: R = alpha B, scaled per column ------------------------
// Every canonical column j of alpha B is scaled by the power of two 2^-c_j
// that brings its largest entry near 1 (exact in FP64), so that the FP32 /
// BF16 low-precision solve sees neither underflow nor overflow from the
// scale of B; X is scaled back by 2^c_j when written.  With alpha = a 2^ea
// (1 <= |a| < 2) and eb the exponent of max_i |B(i,j)| (clamped to
// [-1000, 1000], so that both factors are normal doubles), c_j = ea + eb and
// R(:,j) = B(:,j) * (a 2^-eb), one rounding, as alpha B(:,j) 2^-c_j.
// Columns with a non-finite entry are left unscaled (the range check then
// reports them).
__device__ __forceinline__ int column_eb(int maxfield)
{
    if (maxfield == 0x7FF) return 0;  // not finite
    return max(-1000, min(1000, maxfield - 1023));  // zero / subnormal columns: 2^1000 up
}
__device__ __forceinline__ double pow2(int e)  // 2^e, -1022 <= e <= 1023
{
    return __longlong_as_double(static_cast<long long>(static_cast<unsigned long long>(e + 1023) << 52));
}

// Side = left (canonical columns = columns of B, rows reversed for a
// backward problem), kp <= NT * VPT: one CTA of NT threads per column holds
// the column in registers (VPT lane-contiguous values per thread), finds its
// exponent, and writes R and Y = float(R) in one pass over B.
template <int NT, int VPT>
__global__ void __launch_bounds__(NT)
prepB_cols_kernel(const double *B, int64_t ldb, bool rev, int64_t k, int64_t ncols, double am, int ea, double *R,
                  float *Y, int *cs, int64_t kp)
{
    constexpr int NW = NT / 32;
    __shared__ int red[NW];
    const int64_t j = blockIdx.x;
    double b[VPT];
    int mf = 0;
#pragma unroll
    for (int q = 0; q < VPT; q++) {
        const int64_t i = threadIdx.x + int64_t(q) * NT;
        b[q] = (i < k && j < ncols) ? B[(rev ? k - 1 - i : i) + j * ldb] : 0.0;
    }
#pragma unroll
    for (int q = 0; q < VPT; q++) mf = max(mf, bexp(b[q]));
    mf = __reduce_max_sync(0xffffffffu, mf);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mf;
    __syncthreads();
    for (int w = 0; w < NW; w++) mf = max(mf, red[w]);
    const int eb = column_eb(mf);
    const double g = am * pow2(-eb);  // exact: a normal power of two times |a| in [1, 2)
    if (threadIdx.x == 0) cs[j] = ea + eb;
#pragma unroll
    for (int q = 0; q < VPT; q++) {
        const int64_t i = threadIdx.x + int64_t(q) * NT;
        if (i < kp) {
            const double v = b[q] * g;
            R[i + j * kp] = v;
            Y[i + j * kp] = f64_to_f32_rn(v);
        }
    }
}

// General case, pass 1: the largest exponent field of every canonical
// column (atomic maximum into cmax, zero-initialised), 64 x 64 tiles read
// along B's contiguous dimension.
__global__ void __launch_bounds__(256)
colexp_kernel(const double *B, int64_t ldb, bool left, bool rev, int64_t k, int64_t ncols, int *cmax)
{
    __shared__ int t[64];
    const int64_t i0 = int64_t(blockIdx.y) * 64, j0 = int64_t(blockIdx.x) * 64;
    const int tid = threadIdx.x;
    if (tid < 64) t[tid] = 0;
    __syncthreads();
    for (int idx = tid; idx < 64 * 64; idx += 256) {
        int fast = idx & 63, slow = idx >> 6;
        int li = left ? fast : slow, lj = left ? slow : fast;
        int64_t i = i0 + li, j = j0 + lj;
        if (i < k && j < ncols) {
            int64_t r = rev ? k - 1 - i : i;
            const int f = bexp(left ? B[r + j * ldb] : B[j + r * ldb]);
            if (f > 0) atomicMax(&t[lj], f);
        }
    }
    __syncthreads();
    if (tid < 64 && t[tid] > 0) atomicMax(&cmax[j0 + tid], t[tid]);
}

// General case, pass 2: R = alpha B 2^-c (canonical layout, zero padding)
// and Y = float(R) through a 64 x 64 shared-memory tile.
__global__ void __launch_bounds__(256)
prepB_kernel(const double *B, int64_t ldb, bool left, bool rev, int64_t k, int64_t ncols, double am, int ea,
             double *R, float *Y, const int *cmax, int64_t kp)
{
    __shared__ double t[64][65];
    __shared__ double gcol[64];
    const int64_t i0 = int64_t(blockIdx.y) * 64, j0 = int64_t(blockIdx.x) * 64;
    const int tid = threadIdx.x;
    if (tid < 64) {
        const int eb = column_eb(cmax[j0 + tid]);
        gcol[tid] = am * pow2(-eb);
    }
    __syncthreads();
    for (int idx = tid; idx < 64 * 64; idx += 256) {
        int fast = idx & 63, slow = idx >> 6;
        int li = left ? fast : slow, lj = left ? slow : fast;
        int64_t i = i0 + li, j = j0 + lj;
        double val = 0.0;
        if (i < k && j < ncols) {
            int64_t r = rev ? k - 1 - i : i;
            val = (left ? B[r + j * ldb] : B[j + r * ldb]) * gcol[lj];
        }
        t[li][lj] = val;
    }
    __syncthreads();
    for (int idx = tid; idx < 64 * 64; idx += 256) {
        int li = idx & 63, lj = idx >> 6;
        R[(i0 + li) + (j0 + lj) * kp] = t[li][lj];
        Y[(i0 + li) + (j0 + lj) * kp] = f64_to_f32_rn(t[li][lj]);
    }
}

// Pass 3: the column maxima become the exponents c_j, in place, once every
// tile of pass 2 has read them.
__global__ void colexp_finish_kernel(int *cs, int ea, int64_t np)
{
    const int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (j < np) cs[j] = ea + column_eb(cs[j]);
}

int launch_prepB(const double *B, int64_t ldb, bool left, bool rev, int64_t k, int64_t ncols, double am, int ea,
                 double *R, float *Y, int *cs, int64_t kp, int64_t np, cudaStream_t s)
{
    const dim3 g((unsigned)np);
    if (left && kp <= 2048)
        prepB_cols_kernel<256, 8><<<g, 256, 0, s>>>(B, ldb, rev, k, ncols, am, ea, R, Y, cs, kp);
    else if (left && kp <= 8192)
        prepB_cols_kernel<512, 16><<<g, 512, 0, s>>>(B, ldb, rev, k, ncols, am, ea, R, Y, cs, kp);
    else if (left && kp <= 16384)
        prepB_cols_kernel<1024, 16><<<g, 1024, 0, s>>>(B, ldb, rev, k, ncols, am, ea, R, Y, cs, kp);
    else {
        GB_CUDA(cudaMemsetAsync(cs, 0, size_t(np) * 4, s));
        const dim3 tg((unsigned)(np / 64), (unsigned)(kp / 64));
        colexp_kernel<<<tg, 256, 0, s>>>(B, ldb, left, rev, k, ncols, cs);
        GB_CUDA(cudaGetLastError());
        prepB_kernel<<<tg, 256, 0, s>>>(B, ldb, left, rev, k, ncols, am, ea, R, Y, cs, kp);
        GB_CUDA(cudaGetLastError());
        colexp_finish_kernel<<<(unsigned)((np + 255) / 256), 256, 0, s>>>(cs, ea, np);
    }
    return check(cudaGetLastError());
}

// The kept corrections of column j: D_t = N_t 2^(f_t(j) - 16), N_t = 256 z_1 +
// z_2 from the digit slices (|N_t| <= 2^15 + 2^7).  With f_min the smallest
// f_t, X = (sum_t N_t 2^(f_t - f_min)) 2^(f_min - 16): when every shift is at
// most 46 the sum is exact in an int64 and X is its one correct rounding (the
// FP64 sum D_0 + D_1 + ... in order gives the same value whenever its first
// additions are exact, the usual case); wider spreads add in FP64 in order.
struct SlotCol {
    int e;               // f_min - 16 + c_j (c_j: the column's scale exponent)
    int sh[kZSlots];     // f_t - f_min
    bool exact;          // the int64 sum applies
    bool small;          // every shift <= 36: |sum| < 2^53, a double holds it unrounded
};

__device__ __forceinline__ SlotCol slot_col(const int *fz, int nz, int64_t np, int64_t j, int cj)
{
    SlotCol c;
    int f[kZSlots];
    int fmin = 0x7fffffff;
#pragma unroll
    for (int t = 0; t < kZSlots; t++) {
        f[t] = t < nz ? fz[size_t(t) * np + j] : 0;
        if (t < nz) fmin = min(fmin, f[t]);
    }
    c.e = fmin - 16 + cj;
    c.exact = true;
    c.small = true;
#pragma unroll
    for (int t = 0; t < kZSlots; t++) {
        c.sh[t] = t < nz ? f[t] - fmin : 0;
        c.exact = c.exact && c.sh[t] <= 46;  // 3 (2^15 + 2^7) 2^46 < 2^63
        c.small = c.small && c.sh[t] <= 36;  // 3 (2^15 + 2^7) 2^36 < 2^53
    }
    return c;
}

// 256 z_1 + z_2 for integer-valued BF16 digits (|z| <= 128): exact in FP32,
// read back as an integer through the 1.5 * 2^23 offset (|n| < 2^22).
__device__ __forceinline__ int digit_pair(__nv_bfloat16 z1, __nv_bfloat16 z2)
{
    const float n = fmaf(__bfloat162float(z1), 256.0f, __bfloat162float(z2));
    return __float_as_int(n + 12582912.0f) - 0x4B400000;
}

// S 2^e as a double for |S| < 2^53 (exact: no rounding), from the bit
// pattern with integer operations; results outside the normal range take the
// library path.
__device__ __forceinline__ double scaled_i53_to_f64(long long S, int e)
{
    if (S == 0) return 0.0;
    const unsigned long long sign = S < 0 ? (1ull << 63) : 0ull;
    const unsigned long long u = S < 0 ? 0ull - static_cast<unsigned long long>(S) : static_cast<unsigned long long>(S);
    const int lz = __clzll(static_cast<long long>(u));  // >= 11
    const int ex = 63 - lz + e;
    if (ex < -1022 || ex > 1023) return ldexp_i64_slow(S, e);
    // leading one moved to bit 52 (the implicit bit, removed by the add
    // of the exponent field minus one)
    return __longlong_as_double(static_cast<long long>(
        sign | ((u << (lz - 11)) + (static_cast<unsigned long long>(ex + 1022) << 52))));
}

// The FP64 sum of the corrections in order, for columns whose spread of
// exponents is too wide for the int64 sum (out of line: rarely taken).
__device__ __noinline__ double x_sum_f64(int n0, int n1, int n2, int nz, int e, int s0, int s1, int s2)
{
    double x = scaled_i32_to_f64(n0, e + s0);
    if (nz > 1) x += scaled_i32_to_f64(n1, e + s1);
    if (nz > 2) x += scaled_i32_to_f64(n2, e + s2);
    return x;
}

// X of one element (column parameters c) from its digits z[2t], z[2t+1] of
// the first nz corrections.
__device__ __forceinline__ double x_from_digits(const __nv_bfloat16 (&z)[2 * kZSlots], int nz, const SlotCol &c)
{
    static_assert(kZSlots == 3, "x_sum_f64 takes three corrections");
    int N[kZSlots];
#pragma unroll
    for (int t = 0; t < kZSlots; t++) N[t] = t < nz ? digit_pair(z[2 * t], z[2 * t + 1]) : 0;
    if (!c.exact) return x_sum_f64(N[0], N[1], N[2], nz, c.e, c.sh[0], c.sh[1], c.sh[2]);
    long long S = 0;
#pragma unroll
    for (int t = 0; t < kZSlots; t++)
        if (t < nz) S += static_cast<long long>(N[t]) << c.sh[t];
    return c.small ? scaled_i53_to_f64(S, c.e) : scaled_i64_to_f64(S, c.e);
}

// The digits of element o (slot t at Zs + 2 t kn: z_1 plane, then z_2 plane).
__device__ __forceinline__ void load_digits(__nv_bfloat16 (&z)[2 * kZSlots], const __nv_bfloat16 *Zs, int nz,
                                            size_t kn, size_t o, bool in)
{
#pragma unroll
    for (int u = 0; u < 2 * kZSlots; u++)
        z[u] = (in && (u >> 1) < nz) ? Zs[size_t(u >> 1) * 2 * kn + size_t(u & 1) * kn + o] : __ushort_as_bfloat16(0);
}

__device__ __forceinline__ double x_from_slots(const __nv_bfloat16 *Zs, int nz, size_t kn, size_t o,
                                               const SlotCol &c)
{
    __nv_bfloat16 z[2 * kZSlots];
    load_digits(z, Zs, nz, kn, o, true);
    return x_from_digits(z, nz, c);
}

// X = the sum of the kept corrections (when the refinement outgrows the slots).
__global__ void __launch_bounds__(256)
fold_slots_kernel(double *X, const __nv_bfloat16 *Zs, const int *fz, int nz, int64_t kp, int64_t np)
{
    const int64_t i = int64_t(blockIdx.y) * 256 + threadIdx.x, j = blockIdx.x;
    const SlotCol c = slot_col(fz, nz, np, j, 0);  // X stays in the scaled units of the refinement
    if (i < kp) X[i + j * kp] = x_from_slots(Zs, nz, size_t(kp) * size_t(np), size_t(i) + size_t(j) * size_t(kp), c);
}

// x 2^c for the column scale exponents c (|c| <= 2074): three factors, each
// a normal power of two (only a product that leaves the normal range rounds).
__device__ __forceinline__ double unscale(double x, int c)
{
    const int h = c / 3;
    return x * pow2(h) * pow2(h) * pow2(c - 2 * h);
}

// B(user) = X' 2^c_j mapped back (only the m x n user entries); X' is read
// from X (nz == 0) or formed from the digit slices of the first nz
// corrections.  Side = right: B's contiguous index is the canonical column,
// so 64 x 64 tiles pass through shared memory.
__global__ void __launch_bounds__(256)
writeback_kernel(double *B, int64_t ldb, bool left, bool rev, int64_t k, int64_t ncols, const double *X,
                 int64_t kp, int64_t np, const __nv_bfloat16 *Zs, const int *fz, int nz, const int *cs)
{
    __shared__ double t[64][65];
    const int64_t i0 = int64_t(blockIdx.y) * 64, j0 = int64_t(blockIdx.x) * 64;
    const int tid = threadIdx.x;
    const size_t kn = size_t(kp) * size_t(np);
    for (int idx = tid; idx < 64 * 64; idx += 256) {
        int li = idx & 63, lj = idx >> 6;
        const size_t o = size_t(i0 + li) + size_t(j0 + lj) * size_t(kp);
        const int cj = cs[j0 + lj];
        t[li][lj] = nz ? x_from_slots(Zs, nz, kn, o, slot_col(fz, nz, np, j0 + lj, cj)) : unscale(X[o], cj);
    }
    __syncthreads();
    for (int idx = tid; idx < 64 * 64; idx += 256) {
        int fast = idx & 63, slow = idx >> 6;
        int li = left ? fast : slow, lj = left ? slow : fast;
        int64_t i = i0 + li, j = j0 + lj;
        if (i < k && j < ncols) {
            int64_t r = rev ? k - 1 - i : i;
            if (left) B[r + j * ldb] = t[li][lj];
            else B[j + r * ldb] = t[li][lj];
        }
    }
}

// Side = left: B's columns are the canonical columns (rows reversed for a
// backward problem; X' 2^c_j as above), so no transpose: one column per CTA row of the grid,
// each warp 128 rows, four consecutive rows per thread: one 8-byte load per
// digit plane (or two 16-byte loads of X), and 16-byte stores of B when the
// destination is aligned (scalar stores otherwise).
__global__ void __launch_bounds__(256)
writeback_left_kernel(double *B, int64_t ldb, bool rev, int64_t k, const double *X, int64_t kp, int64_t np,
                      const __nv_bfloat16 *Zs, const int *fz, int nz, const int *cs)
{
    const int64_t j = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t ib = (int64_t(blockIdx.y) * 8 + warp) * 128 + 4 * lane;
    if (ib >= k) return;  // ib < k <= kp, and kp is a multiple of 128: rows ib .. ib + 3 are in the buffers
    const size_t kn = size_t(kp) * size_t(np), o0 = size_t(ib) + size_t(j) * size_t(kp);
    const int cj = cs[j];
    double x[4];
    if (nz == 0) {
        const double2 a = *reinterpret_cast<const double2 *>(X + o0);
        const double2 b = *reinterpret_cast<const double2 *>(X + o0 + 2);
        x[0] = unscale(a.x, cj);
        x[1] = unscale(a.y, cj);
        x[2] = unscale(b.x, cj);
        x[3] = unscale(b.y, cj);
    } else {
        const SlotCol c = slot_col(fz, nz, np, j, cj);
        uint2 zz[2 * kZSlots];
#pragma unroll
        for (int u = 0; u < 2 * kZSlots; u++)
            zz[u] = (u >> 1) < nz ? *reinterpret_cast<const uint2 *>(Zs + size_t(u >> 1) * 2 * kn + size_t(u & 1) * kn + o0)
                                  : make_uint2(0u, 0u);
#pragma unroll
        for (int q = 0; q < 4; q++) {
            __nv_bfloat16 z[2 * kZSlots];
#pragma unroll
            for (int u = 0; u < 2 * kZSlots; u++) {
                const uint32_t w = (q < 2) ? zz[u].x : zz[u].y;
                z[u] = __ushort_as_bfloat16((unsigned short)((q & 1) ? (w >> 16) : (w & 0xFFFFu)));
            }
            x[q] = x_from_digits(z, nz, c);
        }
    }
    double *bc = B + j * ldb;
    if (ib + 3 < k) {
        // rows ib .. ib + 3 of X: B rows ib .. ib + 3, or k - 4 - ib .. k - 1 - ib reversed
        double *d = rev ? bc + (k - 4 - ib) : bc + ib;
        if ((reinterpret_cast<uintptr_t>(d) & 15) == 0) {
            if (rev) {
                reinterpret_cast<double2 *>(d)[0] = make_double2(x[3], x[2]);
                reinterpret_cast<double2 *>(d)[1] = make_double2(x[1], x[0]);
            } else {
                reinterpret_cast<double2 *>(d)[0] = make_double2(x[0], x[1]);
                reinterpret_cast<double2 *>(d)[1] = make_double2(x[2], x[3]);
            }
            return;
        }
    }
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const int64_t i = ib + q;
        if (i < k) bc[rev ? k - 1 - i : i] = x[q];
    }
}

// Per column j: f_j = E + 2 with 2^E <= max_k |Y(k,j)| < 2^(E+1); the
// 16-bit value N = round(Y 2^(16-f_j)) (|N| <= 2^15, FP32 arithmetic, exact
// scaling) split into balanced base-256 digits z_1, z_2 (N = 256 z_1 + z_2,
// |z_q| <= 128, exact in BF16); X += D~ with D~ = N 2^(f_j-16) (exact in
// FP32, added in FP64).
// Accumulates sum D~^2 into norms[0] (FP32 partial sums), and, on the first
// call, sum X^2 into norms[1] and the column maxima of |X| into xmax; the
// largest column ratio max|D~| / max|X| goes to norms[2] (as bits); a column
// whose maximum is not a finite FP32 value (the low-precision solve left
// the FP32 range, or the data are not finite) counts into norms[3].
// One CTA of NT threads per column; with VPT > 0 (kp <= NT * VPT) the column
// is read once into registers (VPT lane-contiguous values per thread),
// otherwise (VPT = 0) it is read again for the second pass.
template <int NT, int VPT>
__global__ void __launch_bounds__(NT)
slice_cols_kernel(const float *Y, int64_t kp, int64_t np, int64_t ncols, __nv_bfloat16 *Zs, int *f_col,
                  double *X, float *xmax, double *norms, int first)
{
    constexpr int NW = NT / 32;
    const int64_t j = blockIdx.x;
    const float *y = Y + j * kp;
    __shared__ float red[NW];
    __shared__ float redd[2][NW];
    float v[VPT > 0 ? VPT : 1];
    float mx = 0.f;
    int bad = 0;  // a value that is not a finite FP32 number (fmaxf would skip a NaN)
    if constexpr (VPT > 0) {
#pragma unroll
        for (int q = 0; q < VPT; q++) {
            const int64_t i = threadIdx.x + int64_t(q) * NT;
            v[q] = i < kp ? y[i] : 0.f;
        }
#pragma unroll
        for (int q = 0; q < VPT; q++) {
            const float a = fabsf(v[q]);
            mx = fmaxf(mx, a);
            bad |= !(a <= 3.4028235e38f);
        }
    } else {
        for (int64_t i = threadIdx.x; i < kp; i += NT) {
            const float a = fabsf(y[i]);
            mx = fmaxf(mx, a);
            bad |= !(a <= 3.4028235e38f);
        }
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    bad = __syncthreads_or(bad);
    mx = 0.f;
    for (int w = 0; w < NW; w++) mx = fmaxf(mx, red[w]);
    const int be = int((__float_as_uint(mx) >> 23) & 0xFF);
    const int f = (be > 0) ? be - 127 + 2 : 0;
    if (threadIdx.x == 0) f_col[j] = f;
    const float up = ldexpf(1.0f, 16 - f), down = ldexpf(1.0f, f - 16);
    __nv_bfloat16 *z1 = Zs + j * kp;
    __nv_bfloat16 *z2 = Zs + np * kp + j * kp;
    double *x = X ? X + j * kp : nullptr;
    float sd = 0.f, sx = 0.f;
    auto digits = [&](int64_t i, float yi) {
        const int N = (be > 0) ? __float2int_rn(yi * up) : 0;
        const int q2 = ((N + 128) & 255) - 128;
        const int q1 = (N - q2) >> 8;
        // |q1|, |q2| <= 128: the BF16 patterns are the top halves of the exact FP32 values
        z1[i] = __ushort_as_bfloat16((unsigned short)(small_int_f32bits(q1) >> 16));
        z2[i] = __ushort_as_bfloat16((unsigned short)(small_int_f32bits(q2) >> 16));
        const float d = float(N) * down;  // exact
        if (x) {
            const double dd = scaled_i32_to_f64(N, f - 16);  // the same value as a double
            if (first) x[i] = dd;
            else x[i] += dd;
        }
        sd = fmaf(d, d, sd);
    };
    if constexpr (VPT > 0) {
#pragma unroll
        for (int q = 0; q < VPT; q++) {
            const int64_t i = threadIdx.x + int64_t(q) * NT;
            if (i < kp) digits(i, v[q]);
        }
    } else {
        for (int64_t i = threadIdx.x; i < kp; i += NT) digits(i, y[i]);
    }
    if (first) sx = sd;
    for (int o = 16; o > 0; o >>= 1) {
        sd += __shfl_xor_sync(0xffffffffu, sd, o);
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
    }
    if ((threadIdx.x & 31) == 0) {
        redd[0][threadIdx.x >> 5] = sd;
        redd[1][threadIdx.x >> 5] = sx;
    }
    __syncthreads();
    if (threadIdx.x == 0 && j < ncols && bad) atomicAdd(&norms[3], 1.0);
    if (threadIdx.x == 0 && j < ncols) {
        float a = 0.f, b = 0.f;
        for (int w = 0; w < NW; w++) {
            a += redd[0][w];
            b += redd[1][w];
        }
        const float dmax = float((be > 0) ? mx : 0.f);
        if (first) xmax[j] = dmax;
        const float xm = first ? dmax : xmax[j];
        const double ratio = (xm > 0.f) ? double(dmax) / double(xm) : (dmax > 0.f ? 1.0 : 0.0);
        atomicAdd(&norms[0], double(a));
        if (first) atomicAdd(&norms[1], double(b));
        // non-negative doubles order like their bit patterns
        atomicMax(reinterpret_cast<unsigned long long *>(&norms[2]),
                  static_cast<unsigned long long>(__double_as_longlong(ratio)));
    }
}

void launch_slice_cols(const float *Y, int64_t kp, int64_t np, int64_t ncols, __nv_bfloat16 *Zs, int *f_col,
                       double *X, float *xmax, double *norms, int first, cudaStream_t s)
{
    const dim3 g((unsigned)np);
    if (kp <= 1024)
        slice_cols_kernel<256, 4><<<g, 256, 0, s>>>(Y, kp, np, ncols, Zs, f_col, X, xmax, norms, first);
    else if (kp <= 2048)
        slice_cols_kernel<256, 8><<<g, 256, 0, s>>>(Y, kp, np, ncols, Zs, f_col, X, xmax, norms, first);
    else if (kp <= 4096)
        slice_cols_kernel<256, 16><<<g, 256, 0, s>>>(Y, kp, np, ncols, Zs, f_col, X, xmax, norms, first);
    else if (kp <= 8192)
        slice_cols_kernel<256, 32><<<g, 256, 0, s>>>(Y, kp, np, ncols, Zs, f_col, X, xmax, norms, first);
    else if (kp <= 16384)
        slice_cols_kernel<1024, 16><<<g, 1024, 0, s>>>(Y, kp, np, ncols, Zs, f_col, X, xmax, norms, first);
    else if (kp <= 32768)
        slice_cols_kernel<1024, 32><<<g, 1024, 0, s>>>(Y, kp, np, ncols, Zs, f_col, X, xmax, norms, first);
    else
        slice_cols_kernel<256, 0><<<g, 256, 0, s>>>(Y, kp, np, ncols, Zs, f_col, X, xmax, norms, first);
}

// ---- residual: FP64 application of the exact sums ------------------------------

// R(i,j) -= T(i,j) 2^(e_i + f_j - W) for the rows i >= row_lo the tensor-core
// launch over K range [k_lo, k_hi) reached; for the rows of that range it
// also subtracts the diagonal part Mv(i,i) D(i,j), D(i,j) = z(i,j) 2^(f_j-16)
// with z = 256 z_1 + z_2 the correction digits (exact), in one FMA, and
// writes Y = float(R) for the next low-precision solve (the launch holding
// row i is the last to touch it).  One column per CTA row of the grid, each
// warp 128 rows, 4 lane-contiguous rows per thread (coalesced, with four
// independent element updates in flight per thread).
__global__ void __launch_bounds__(256, 5)
residual_apply_kernel(double *R, const long long *Tg, const int *e_row, const int *f_col, int W, const double *dg,
                      const __nv_bfloat16 *Zs, float *Y, int64_t kp, int64_t np, int64_t row_lo, int64_t k_lo,
                      int64_t k_hi)
{
    const int64_t j = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t ib = row_lo + (int64_t(blockIdx.y) * 8 + warp) * 128 + lane;
    const int fj = f_col[j];
    const int64_t o0 = ib + j * kp;
    // every load of the thread first
    double r[4], d[4];
    long long tv[4];
    int e[4];
    __nv_bfloat16 z1[4], z2[4];
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const int64_t i = ib + 32 * q, o = o0 + 32 * q;
        const bool in = i < kp, ink = in && i >= k_lo && i < k_hi;
        r[q] = in ? R[o] : 0.0;
        tv[q] = in ? Tg[o] : 0ll;
        e[q] = in ? e_row[i] : 0;
        d[q] = ink ? dg[i] : 0.0;
        z1[q] = ink ? Zs[o] : __ushort_as_bfloat16(0);
        z2[q] = ink ? Zs[np * kp + o] : __ushort_as_bfloat16(0);
    }
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const int64_t i = ib + 32 * q, o = o0 + 32 * q;
        if (i < kp) {
            double v = r[q] - scaled_i64_to_f64(tv[q], e[q] - W + fj);
            if (i >= k_lo && i < k_hi) {
                v = fma(-d[q], scaled_i32_to_f64(digit_pair(z1[q], z2[q]), fj - 16), v);
                Y[o] = f64_to_f32_rn(v);
            }
            R[o] = v;
        }
    }
}

// ---- workspace --------------------------------------------------------------
struct Workspace {
    char *base = nullptr;
    size_t bytes = 0;
};

cudaMemPool_t library_pool()
{
    static cudaMemPool_t pool[64] = {nullptr};
    static std::mutex mu;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(mu);
    if (!pool[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p;
        if (cudaMemPoolCreate(&p, &props) != cudaSuccess) return nullptr;
        uint64_t thr = ~0ull;  // keep freed blocks cached in the pool
        cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &thr);
        pool[dev] = p;
    }
    return pool[dev];
}

// Executor of the low-precision forward solve on the padded canonical view.
struct LowExec {
    float *Y;
    __nv_bfloat16 *Ybf;
    const __nv_bfloat16 *Abf;
    const float *binv;  // inverses of the diagonal kBand-blocks
    int64_t kp, np;
    cudaStream_t s;
    int *status_word;   // device word for wait timeouts
    bool fp8 = false;   // FP8 E4M3 updates with block scales instead of BF16
    const uint8_t *A8 = nullptr;
    const float *sA = nullptr;   // (kp/128)^2 block scales of A8
    uint8_t *Y8 = nullptr;
    float *sY = nullptr;         // (kp/128) x (np/64) block scales of Y8
    const __nv_bfloat16 *binv16 = nullptr;  // two-term BF16 split of the inverses (tensor-core TS task)
    int64_t leaf = 0;   // leaf order of the recursion (0 = the form's default)
    int status = 0;
    bool ok() const { return status == 0; }
    void ts(int64_t b0, int64_t nr, float a)
    {
        if (status) return;
        if (!fp8) {
            // BF16 form: a leaf (kLeaf rows by default), left-looking, in one
            // launch: each 128-row block takes its update from the solved
            // blocks of the leaf and its TS task
            status = launch_leaf_tc(Abf, binv16, kp, np, b0, nr, Y, Ybf, s, status_word);
            return;
        }
        if (nr > kBand) {
            drive_blocked(*this, b0, b0 + nr, (int64_t)kBand, a, true);
            return;
        }
        // TS task: X_b = L_b^-1 Y_b with the precomputed inverse of the block
        status = launch_apply_inverse_fp8(binv + b0 * kBand, Y + b0, kp, Y8 + b0, sY + (b0 / 128) * (np / 64),
                                          (int)nr, np, s);
    }
    void gemm(int64_t ci0, int64_t M, int64_t ak0, int64_t K, float a)
    {
        if (status) return;
        if (fp8)
            status = launch_tc_gemm_fp8(M, np, K, A8 + ci0 * kp + ak0, kp, Y8 + ak0, kp, Y + ci0, kp, a,
                                        sA + (ci0 / 128) * (kp / 128) + ak0 / 128, kp / 128,
                                        sY + (ak0 / 128) * (np / 64), np / 64, s, status_word);
        else
            status = launch_tc_gemm_bf16(M, np, K, Abf + ci0 * kp + ak0, kp, Ybf + ak0, kp, Y + ci0, kp, a, s,
                                         status_word);
    }
};

// Recursive model (Section V-A) down to leaves of e.leaf rows, by default
// kLeaf (BF16 form: each leaf solved left-looking by one leaf kernel launch)
// or kBand (FP8 form: larger leaves are solved blocked in kBand steps).
int low_solve(LowExec &e, int64_t kp)
{
    const int64_t leaf = e.leaf > 0 ? e.leaf : (e.fp8 ? kBand : kLeaf);
    drive_recursive(e, 0, kp, 24, leaf, 1.0f, true);
    return e.status;
}

// Which digit pairs the residual must form for a correction Z whose size
// relative to X is rho.  Pair (p, q) has weight 2^-(8p + 8q), i.e. it sits
// 2^-(8p + 8q - 16) below the leading pair (1, 1), and the leading pair is
// about rho |Mv||X|; every pair above 2^-target |Mv||X| is formed, with
// target = log2(1/tol) + 2 (a factor 4 under the requested tolerance).
// Returns P (slices paired with z_1) and P2 (slices also paired with z_2).
void pairs_for(double rho, double tol, int *P, int *P2)
{
    const double target = -std::log2(tol > 0 ? tol : 1e-16) + 2.0;
    const double b = rho > 0 ? -std::log2(rho) : 1e9;
    const double budget = target - b + 16.0;
    int p1 = int(std::floor((budget - 8.0) / 8.0));
    int p2 = int(std::floor((budget - 16.0) / 8.0));
    // the int64 sums of the residual hold 2^(W+8) per 1024-chunk, 16 chunks a
    // launch: W = max(8 P + 8, 8 P2 + 16) <= 48 keeps them below 2^61 (this
    // bounds the attainable residual accuracy near 2^-48 |Mv||X|: a tol much
    // below 1e-13 is not reached and is reported as not converged)
    if (p1 > kSlices - 1) p1 = kSlices - 1;
    if (p2 > kSlices - 2) p2 = kSlices - 2;
    if (p1 < 1) p1 = 1;
    if (p2 > p1) p2 = p1;
    if (p2 < 0) p2 = 0;
    *P = p1;
    *P2 = p2;
}

// One tensor-core launch per K range of at most 16384 (the int64 sums stay
// below 2^63; inside, chunks of 1024 keep every tensor-core sum exact:
// |a| <= 128, |z| <= 128: 1024 * 128 * 128 = 2^24), each followed by the FP64
// application of its sums.
int residual_update(double *R, long long *Tg, const __nv_bfloat16 *As, const __nv_bfloat16 *Zs, const int *e_row,
                    const int *f_col, const double *dg, float *Y, int64_t kp, int64_t np, int P, int P2,
                    cudaStream_t s, int *status_word)
{
    const int W = residual_weight(P, P2);
    for (int64_t lo = 0; lo < kp; lo += 16384) {
        int64_t hi = lo + 16384 < kp ? lo + 16384 : kp;
        GB_TRY(launch_tc_residual(Tg, kp, As, Zs, kp, np, lo, hi, P, P2, s, status_word));
        LaunchScope ls(KK_CONVERT, s, 0, 30.0 * double(kp - lo) * double(np));
        const dim3 grid((unsigned)np, (unsigned)((kp - lo + 1023) / 1024));
        residual_apply_kernel<<<grid, 256, 0, s>>>(R, Tg, e_row, f_col, W, dg, Zs, Y, kp, np, lo, lo, hi);
        GB_TRY(check(cudaGetLastError()));
    }
    return 0;
}

// The low-precision solve is a fixed sequence of launches on fixed buffers:
// it is captured once into a CUDA graph (on a library stream) and replayed
// on the caller's stream at every refinement step.  The last few graphs are
// kept per device (least recently used first out), keyed by work-space
// address and sizes, so that callers alternating between problems or entry
// points (device buffers, host buffers in column blocks) do not recapture.
struct LowGraph {
    cudaGraphExec_t exec = nullptr;
    const void *ws = nullptr;
    int64_t kp = 0, np = 0;
    bool fp8 = false;
    int64_t leaf = 0;
    uint64_t nkernels = 0;
    uint64_t used = 0;  // last use (LRU clock)
};
constexpr int kGraphs = 4;

}  // namespace

// Solves that replay cached graphs or use the cached work space on one
// device are serialised: a graph in use must not be evicted (destroyed), nor
// the work space regrown, by another host thread's solve.  Recursive, so that
// an entry point can hold it around the whole call.
std::recursive_mutex &mixed_device_mutex()
{
    static std::recursive_mutex mu[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
    return mu[dev];
}

// The allocating entry points' work space: one buffer per device from the
// library's pool, kept between calls and regrown when a larger problem needs
// more (the old buffer is released once the stream is idle).  A stable
// address means the captured low-precision graphs, which name the work
// space's buffers, are found again on the next call instead of being
// captured anew.  The caller holds mixed_device_mutex().
struct DeviceWorkspace {
    char *base = nullptr;
    size_t size = 0;
};
static DeviceWorkspace g_ws[64];

int mixed_workspace(size_t bytes, cudaStream_t s, char **out)
{
    int dev = 0;
    GB_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return GB_STATUS_CUDA_ERROR;
    DeviceWorkspace &w = g_ws[dev];
    if (w.size < bytes) {
        cudaMemPool_t pool = library_pool();
        if (!pool) return GB_STATUS_CUDA_ERROR;
        if (w.base) {
            GB_CUDA(cudaStreamSynchronize(s));
            GB_CUDA(cudaFreeAsync(w.base, s));
            w.base = nullptr;
            w.size = 0;
        }
        // some headroom, so that slightly larger problems do not regrow it
        const size_t want = bytes + bytes / 16;
        char *p = nullptr;
        GB_CUDA(cudaMallocFromPoolAsync(reinterpret_cast<void **>(&p), want, pool, s));
        w.base = p;
        w.size = want;
    }
    *out = w.base;
    return 0;
}

}  // namespace gb

extern "C" int gb_mixed_workspace_release(void *stream)
{
    std::lock_guard<std::recursive_mutex> lk(gb::mixed_device_mutex());
    int dev = 0;
    GB_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return GB_STATUS_CUDA_ERROR;
    gb::DeviceWorkspace &w = gb::g_ws[dev];
    if (!w.base) return 0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    GB_CUDA(cudaStreamSynchronize(s));
    GB_CUDA(cudaFreeAsync(w.base, s));
    w.base = nullptr;
    w.size = 0;
    return gb::check(cudaStreamSynchronize(s));
}

namespace gb {
namespace {

int low_graph(LowExec &le, const void *ws, LowGraph **out)
{
    static LowGraph cache[64][kGraphs];
    static uint64_t clock[64] = {0};
    static cudaStream_t cap_stream[64] = {nullptr};
    int dev = 0;
    GB_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return GB_STATUS_CUDA_ERROR;
    int victim = 0;
    for (int i = 0; i < kGraphs; i++) {
        LowGraph &c = cache[dev][i];
        if (c.exec && c.ws == ws && c.kp == le.kp && c.np == le.np && c.fp8 == le.fp8 && c.leaf == le.leaf) {
            c.used = ++clock[dev];
            *out = &c;
            return 0;
        }
        if (!c.exec || (cache[dev][victim].exec && c.used < cache[dev][victim].used)) victim = i;
    }
    LowGraph &g = cache[dev][victim];
    if (g.exec) {
        cudaGraphExecDestroy(g.exec);
        g.exec = nullptr;
    }
    if (!cap_stream[dev]) GB_CUDA(cudaStreamCreateWithFlags(&cap_stream[dev], cudaStreamNonBlocking));
    // everything that allocates or sets attributes happens before capture
    GB_TRY(tc_gemm_prepare());
    GB_TRY(tc_gemm_fp8_prepare());
    GB_TRY(diag_inv_prepare());
    GB_TRY(apply_tc_prepare());
    cudaStream_t user = le.s;
    le.s = cap_stream[dev];
    le.status = 0;
    const uint64_t before = capture_count();
    GB_CUDA(cudaStreamBeginCapture(le.s, cudaStreamCaptureModeThreadLocal));
    int st = low_solve(le, le.kp);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(le.s, &graph);
    le.s = user;
    if (st) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    GB_CUDA(e);
    e = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    GB_CUDA(e);
    g.ws = ws;
    g.kp = le.kp;
    g.np = le.np;
    g.fp8 = le.fp8;
    g.leaf = le.leaf;
    g.nkernels = capture_count() - before;
    g.used = ++clock[dev];
    *out = &g;
    return 0;
}

}  // namespace

// Per-thread record of the last mixed solve's refinement history:
// rho_t = ||D_t||_F / ||X||_F for t = 1, 2, ... and the digit levels used.
static thread_local double tl_rho[64];
static thread_local int tl_levels[64];
static thread_local int tl_nhist = 0;

MixedLayout mixed_layout(int side, int64_t m, int64_t n, int prec)
{
    MixedLayout L;
    const int64_t k = side == GB_LEFT ? m : n;
    const int64_t ncols = side == GB_LEFT ? n : m;
    L.kp = (k + 127) / 128 * 128;
    L.np = (ncols + 127) / 128 * 128;
    const size_t kk = size_t(L.kp) * size_t(L.kp), kn = size_t(L.kp) * size_t(L.np);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += (bytes + 255) & ~size_t(255);
        return o;
    };
    L.o_abf = take(kk * 2);
    L.o_as = take(kk * 2 * kSlices);
    L.o_band = take(size_t(L.kp) * kBand * 4);
    L.o_binv = take(size_t(L.kp) * kBand * 4);
    L.o_binv16 = take(size_t(L.kp) * kBand * 4);
    L.o_r = take(kn * 8);
    L.o_t = take(kn * 8);
    L.o_x = take(kn * 8);
    L.o_y = take(kn * 4);
    L.o_ybf = take(kn * 2);
    L.o_zs = take(kn * 4 * kZSlots);
    L.o_e = take(size_t(L.kp) * 4);
    L.o_f = take(size_t(L.np) * 4 * kZSlots);
    L.o_norm = take(64);  // 4 FP64 norms, then the solve's device status word (byte 32)
    L.o_dg = take(size_t(L.kp) * 8);
    L.o_xm = take(size_t(L.np) * 4);
    L.o_cs = take(size_t(L.np) * 4);
    if (prec == GB_PREC_FP8) {
        const size_t nbk = size_t(L.kp / 128);
        L.o_a8 = take(kk);
        L.o_bmax = take(nbk * nbk * 4);
        L.o_bscale = take(nbk * nbk * 4);
        L.o_y8 = take(kn);
        L.o_sy = take(nbk * size_t(L.np / 64) * 4);
    } else {
        L.o_a8 = L.o_bmax = L.o_bscale = L.o_y8 = L.o_sy = 0;
    }
    L.total = off;
    return L;
}

// Pointers into a work space laid out by mixed_layout.
struct MixedBufs {
    __nv_bfloat16 *Abf, *As, *binv16, *Ybf, *Zs;
    float *band, *binv, *Y, *xmax;
    double *R, *X, *norms, *dg;
    long long *Tg;
    int *e_row, *f_col, *cs;
    int *status;  // device word of this solve's bounded waits (beside the norms)
    uint8_t *A8, *Y8;
    unsigned *bmax;
    float *bscale, *sY;
};

static MixedBufs mixed_bufs(const MixedLayout &L, char *ws, bool fp8)
{
    MixedBufs b;
    b.Abf = reinterpret_cast<__nv_bfloat16 *>(ws + L.o_abf);
    b.As = reinterpret_cast<__nv_bfloat16 *>(ws + L.o_as);
    b.binv16 = fp8 ? nullptr : reinterpret_cast<__nv_bfloat16 *>(ws + L.o_binv16);
    b.Ybf = reinterpret_cast<__nv_bfloat16 *>(ws + L.o_ybf);
    b.Zs = reinterpret_cast<__nv_bfloat16 *>(ws + L.o_zs);
    b.band = reinterpret_cast<float *>(ws + L.o_band);
    b.binv = reinterpret_cast<float *>(ws + L.o_binv);
    b.Y = reinterpret_cast<float *>(ws + L.o_y);
    b.xmax = reinterpret_cast<float *>(ws + L.o_xm);
    b.cs = reinterpret_cast<int *>(ws + L.o_cs);
    b.R = reinterpret_cast<double *>(ws + L.o_r);
    b.X = reinterpret_cast<double *>(ws + L.o_x);
    b.norms = reinterpret_cast<double *>(ws + L.o_norm);
    b.status = reinterpret_cast<int *>(ws + L.o_norm + 32);
    b.dg = reinterpret_cast<double *>(ws + L.o_dg);
    b.Tg = reinterpret_cast<long long *>(ws + L.o_t);
    b.e_row = reinterpret_cast<int *>(ws + L.o_e);
    b.f_col = reinterpret_cast<int *>(ws + L.o_f);
    b.A8 = fp8 ? reinterpret_cast<uint8_t *>(ws + L.o_a8) : nullptr;
    b.Y8 = fp8 ? reinterpret_cast<uint8_t *>(ws + L.o_y8) : nullptr;
    b.bmax = fp8 ? reinterpret_cast<unsigned *>(ws + L.o_bmax) : nullptr;
    b.bscale = fp8 ? reinterpret_cast<float *>(ws + L.o_bscale) : nullptr;
    b.sY = fp8 ? reinterpret_cast<float *>(ws + L.o_sy) : nullptr;
    return b;
}

// forward = the canonical view is a forward (lower) substitution
static bool mixed_forward(int side, int uplo, int trans)
{
    const bool mt = side == GB_LEFT ? (trans == GB_TRANS) : (trans == GB_NOTRANS);
    return (uplo == GB_LOWER) != mt;
}

int mixed_prep_a(int side, int uplo, int trans, int diag, int64_t k, const double *A, int64_t lda, int prec,
                 const MixedLayout &L, char *ws, cudaStream_t s)
{
    const bool mt = side == GB_LEFT ? (trans == GB_TRANS) : (trans == GB_NOTRANS);
    const bool forward = mixed_forward(side, uplo, trans);
    const bool fp8 = prec == GB_PREC_FP8;
    const int64_t kp = L.kp;
    const MixedBufs bf = mixed_bufs(L, ws, fp8);
    View v{A, lda, mt, !forward, diag == GB_UNIT, k};
    GB_CUDA(cudaMemsetAsync(bf.e_row, 0x80, size_t(kp) * 4, s));  // very negative
    dim3 tgrid((unsigned)(kp / 64), (unsigned)(kp / 64));
    {
        LaunchScope ls(KK_CONVERT, s, 0, 8.0 * double(k) * double(k) / 2);
        if (fp8) GB_CUDA(cudaMemsetAsync(bf.bmax, 0, size_t(kp / 128) * (kp / 128) * 4, s));
        rowexp_kernel<<<tgrid, 256, 0, s>>>(v, kp, bf.e_row, bf.bmax);
        GB_CUDA(cudaGetLastError());
    }
    {
        LaunchScope ls(KK_CONVERT, s, 0, (8.0 + 2.0 * (1 + kSlices)) * double(kp) * double(kp) / 2);
        if (fp8) {
            const int64_t nbb = (kp / 128) * (kp / 128);
            block_scales_kernel<<<(unsigned)((nbb + 255) / 256), 256, 0, s>>>(bf.bmax, bf.bscale, nbb);
            GB_CUDA(cudaGetLastError());
        }
        prepA_kernel<<<tgrid, 256, 0, s>>>(v, kp, bf.e_row, bf.Abf, bf.As, bf.band, bf.dg, bf.A8, bf.bscale);
        GB_CUDA(cudaGetLastError());
    }
    return launch_invert_blocks(bf.band, bf.binv, bf.binv16, kp / kBand, s);
}

int mixed_solve_b(int side, int uplo, int trans, int64_t k, int64_t ncols, double alpha, const double *B,
                  int64_t ldb, double *Bout, int64_t ldbo, double tol, int prec, int max_iter, int *iters_out,
                  double *est_err_out, cudaStream_t s, char *ws, const MixedLayout &L, bool use_graph,
                  cudaEvent_t b_ready, bool merge_hist, int64_t leaf)
{
    const bool forward = mixed_forward(side, uplo, trans);
    const int64_t kp = L.kp, np = L.np;
    const bool fp8 = prec == GB_PREC_FP8;
    const size_t kn = size_t(kp) * size_t(np);
    const MixedBufs bf = mixed_bufs(L, ws, fp8);
    auto *Abf = bf.Abf;
    auto *As = bf.As;
    auto *binv = bf.binv;
    auto *R = bf.R;
    auto *Tg = bf.Tg;
    auto *X = bf.X;
    auto *Y = bf.Y;
    auto *Ybf = bf.Ybf;
    auto *Zs = bf.Zs;
    auto *e_row = bf.e_row;
    auto *f_col = bf.f_col;
    auto *norms = bf.norms;
    auto *dg = bf.dg;
    auto *xmax = bf.xmax;
    int *status_word = bf.status;
    // history of this solve: from scratch, or merged (step-wise maximum)
    // into that of the previous column block of the same problem
    const int hist0 = merge_hist ? tl_nhist : 0;
    int hist = 0;
    if (!merge_hist) tl_nhist = 0;
    std::unique_lock<std::recursive_mutex> graph_lock(mixed_device_mutex(), std::defer_lock);

    int st = 0;
    // the norms of a step and the status word, read back together
    struct StepRead {
        double norm[4];
        int status;
    } h = {{0, 0, 0, 0}, 0};
    static_assert(offsetof(StepRead, status) == 32, "status word follows the four norms");
    double *h_norm = h.norm;
    int iters = 0;
    double est = 0;
    do {
        // the bounded waits of this solve's kernels record timeouts here
        if ((st = check(cudaMemsetAsync(status_word, 0, sizeof(int), s)))) break;
        // the right-hand sides may still be arriving on another stream
        if (b_ready && (st = check(cudaStreamWaitEvent(s, b_ready, 0)))) break;
        {
            LaunchScope ls(KK_CONVERT, s, 0, 16.0 * double(kp) * double(np));
            int ea = 0;
            const double am = 2.0 * std::frexp(alpha, &ea);  // alpha = am 2^(ea - 1), 1 <= |am| < 2
            ea -= 1;
            if ((st = launch_prepB(B, ldb, side == GB_LEFT, !forward, k, ncols, am, ea, R, Y, bf.cs, kp, np, s)))
                break;
            if ((st = check(cudaGetLastError()))) break;
        }
        LowExec le{Y, Ybf, Abf, binv, kp, np, s, status_word};
        le.binv16 = bf.binv16;
        le.fp8 = fp8;
        le.A8 = bf.A8;
        le.sA = bf.bscale;
        le.Y8 = bf.Y8;
        le.sY = bf.sY;
        le.leaf = leaf;
        LowGraph *lg = nullptr;
        if (use_graph) {
            graph_lock.lock();  // held until the solve returns
            if ((st = low_graph(le, ws, &lg))) break;
        }
        const int64_t nel = int64_t(kn);
        __nv_bfloat16 *Zc = Zs;  // digit slot of the current correction
        int *fc = f_col;
        bool folded = false;
        int nz = 0;              // corrections held in slots (0: X holds the sum)
        int Lmax = 76;
        double nx = 0, prev_rho = 0;
        for (int t = 0;; t++) {
            // Y = float(R) was written by prepB (t = 0) or by the residual kernel
            if (use_graph) {
                LaunchScope ls(KK_GRAPH, s, double(kp) * double(kp) * double(np), 0.0, lg->nkernels);
                if ((st = check(cudaGraphLaunch(lg->exec, s)))) break;
            } else {
                le.status = 0;
                if ((st = low_solve(le, kp))) break;
            }
            if ((st = check(cudaMemsetAsync(norms, 0, 4 * sizeof(double), s)))) break;
            // this step's digit slot; the first kZSlots corrections stay in
            // their slots (X untouched), later ones fold them into X first
            const int slot = t % kZSlots;
            Zc = Zs + size_t(slot) * 2 * kn;
            fc = f_col + size_t(slot) * np;
            if (t == kZSlots) {
                LaunchScope ls(KK_CONVERT, s, 0, (8.0 + 4.0 * kZSlots) * double(nel));
                fold_slots_kernel<<<dim3((unsigned)np, (unsigned)((kp + 255) / 256)), 256, 0, s>>>(X, Zs, f_col, kZSlots,
                                                                                             kp, np);
                if ((st = check(cudaGetLastError()))) break;
                folded = true;
            }
            {
                LaunchScope ls(KK_CONVERT, s, 0, (folded ? 24.0 : 8.0) * double(nel));
                launch_slice_cols(Y, kp, np, ncols, Zc, fc, folded ? X : nullptr, xmax, norms, t == 0, s);
                if ((st = check(cudaGetLastError()))) break;
            }
            nz = folded ? 0 : t + 1;
            if ((st = check(cudaMemcpyAsync(&h, norms, offsetof(StepRead, status) + sizeof(int),
                                            cudaMemcpyDeviceToHost, s))))
                break;
            if ((st = check(cudaStreamSynchronize(s)))) break;
            if (h.status != 0) {  // a bounded wait gave up: B is left as it was
                st = GB_STATUS_TIMEOUT;
                break;
            }
            if (h_norm[3] != 0.0) {  // out of the low-precision range: B is left as it was
                st = GB_STATUS_RANGE;
                break;
            }
            const double nd = std::sqrt(h_norm[0]);
            if (t == 0) nx = std::sqrt(h_norm[1]);
            const double rho = nx > 0 ? nd / nx : 0.0;
            if (t > 0 && hist < 64) {
                if (hist < hist0) {
                    tl_rho[hist] = std::max(tl_rho[hist], rho);
                    tl_levels[hist] = std::max(tl_levels[hist], Lmax);
                } else {
                    tl_rho[hist] = rho;
                    tl_levels[hist] = Lmax;
                    tl_nhist = hist + 1;
                }
                hist++;
            }
            if (t > 0) {
                iters = t;
                est = rho;
                if (rho <= tol) break;
                // Predicted error after this update: rho times the observed
                // contraction, when the iteration contracts well.
                if (t >= 2 && prev_rho > 0) {
                    const double c = rho / prev_rho;
                    if (c <= 0.1 && rho * c <= tol) {
                        est = rho * c;
                        break;
                    }
                }
                if (t >= max_iter) break;
                prev_rho = rho;
            }
            int P = kSlices, P2 = kSlices - 1;
            pairs_for(t == 0 ? 1.0 : h_norm[2], tol, &P, &P2);
            Lmax = P * 10 + P2;  // recorded in the history as 10*P + P2
            if ((st = residual_update(R, Tg, As, Zc, e_row, fc, dg, Y, kp, np, P, P2, s, status_word))) break;
        }
        if (st) break;
        {
            LaunchScope ls(KK_CONVERT, s, 0, 16.0 * double(k) * double(ncols));
            if (side == GB_LEFT)
                writeback_left_kernel<<<dim3((unsigned)ncols, (unsigned)((k + 1023) / 1024)), 256, 0, s>>>(
                    Bout, ldbo, !forward, k, X, kp, np, Zs, f_col, nz, bf.cs);
            else
                writeback_kernel<<<dim3((unsigned)(np / 64), (unsigned)(kp / 64)), 256, 0, s>>>(
                    Bout, ldbo, false, !forward, k, ncols, X, kp, np, Zs, f_col, nz, bf.cs);
            if ((st = check(cudaGetLastError()))) break;
        }
    } while (0);
    if (st == 0) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = check(e);
    }
    if (iters_out) *iters_out = iters;
    if (est_err_out) *est_err_out = est;
    if (st) return st;
    return (est <= tol) ? 0 : GB_STATUS_NOT_CONVERGED;
}


int mixed_core(int side, int uplo, int trans, int diag, int64_t m, int64_t n, double alpha, const double *A,
               int64_t lda, double *B, int64_t ldb, double tol, int prec, int max_iter, int *iters_out,
               double *est_err_out, cudaStream_t s, char *ws, bool use_graph, cudaEvent_t b_ready, int64_t leaf)
{
    const int64_t k = side == GB_LEFT ? m : n;
    const int64_t ncols = side == GB_LEFT ? n : m;
    const MixedLayout L = mixed_layout(side, m, n, prec);
    tl_nhist = 0;
    if (iters_out) *iters_out = 0;
    if (est_err_out) *est_err_out = 0;
    GB_TRY(mixed_prep_a(side, uplo, trans, diag, k, A, lda, prec, L, ws, s));
    return mixed_solve_b(side, uplo, trans, k, ncols, alpha, B, ldb, B, ldb, tol, prec, max_iter, iters_out,
                         est_err_out, s, ws, L, use_graph, b_ready, false, leaf);
}

cudaMemPool_t mixed_pool() { return library_pool(); }

int dtrsm_mixed_impl(int side, int uplo, int trans, int diag, int64_t m, int64_t n, double alpha, const double *A,
                     int64_t lda, double *B, int64_t ldb, double tol, int prec, int max_iter, int *iters_out,
                     double *est_err_out, cudaStream_t s, int64_t leaf)
{
    const MixedLayout L = mixed_layout(side, m, n, prec);
    std::lock_guard<std::recursive_mutex> lk(mixed_device_mutex());
    char *ws = nullptr;
    GB_TRY(mixed_workspace(L.total, s, &ws));
    return mixed_core(side, uplo, trans, diag, m, n, alpha, A, lda, B, ldb, tol, prec, max_iter, iters_out,
                      est_err_out, s, ws, true, nullptr, leaf);
}

}  // namespace gb

extern "C" int gb_mixed_history(double *rho, int *levels, int cap)
{
    const int n = gb::tl_nhist < cap ? gb::tl_nhist : cap;
    for (int i = 0; i < n; i++) {
        if (rho) rho[i] = gb::tl_rho[i];
        if (levels) levels[i] = gb::tl_levels[i];
    }
    return gb::tl_nhist;
}

namespace gb {
int mixed_validate(int side, int uplo, int trans, int diag, int64_t m, int64_t n, double alpha, const double *A,
                   int64_t lda, const double *B, int64_t ldb, double tol, int prec, int max_iter)
{
    if (side != GB_LEFT && side != GB_RIGHT) return -1;
    if (uplo != GB_LOWER && uplo != GB_UPPER) return -2;
    if (trans != GB_NOTRANS && trans != GB_TRANS) return -3;
    if (diag != GB_NONUNIT && diag != GB_UNIT) return -4;
    if (m < 0) return -5;
    if (n < 0) return -6;
    const int64_t k = side == GB_LEFT ? m : n;
    const bool empty = (m == 0 || n == 0);
    if (A == nullptr && !empty && alpha != 0.0) return -8;
    if (lda < (k > 1 ? k : 1)) return -9;
    if (B == nullptr && !empty) return -10;
    if (ldb < (m > 1 ? m : 1)) return -11;
    if (!(tol >= 0.0)) return -12;
    if (prec != GB_PREC_BF16 && prec != GB_PREC_FP8) return -13;
    if (max_iter < 1 || max_iter > 1000) return -14;
    return 0;
}
}  // namespace gb

static int dtrsm_mixed_entry(int side, int uplo, int trans, int diag, int64_t m, int64_t n, double alpha,
                             const double *A, int64_t lda, double *B, int64_t ldb, double tol, int prec,
                             int max_iter, int64_t leaf, int *iters_out, double *est_err_out, void *stream)
{
    if (iters_out) *iters_out = 0;
    if (est_err_out) *est_err_out = 0;
    const int v = gb::mixed_validate(side, uplo, trans, diag, m, n, alpha, A, lda, B, ldb, tol, prec, max_iter);
    if (v) return v;
    if (m == 0 || n == 0) return 0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (alpha == 0.0) {
        gb::Canon<double> c{};
        c.B = B;
        c.ldb = ldb;
        c.left = side == GB_LEFT;
        c.k = side == GB_LEFT ? m : n;
        c.ncols = side == GB_LEFT ? n : m;
        c.stream = s;
        int st = gb::launch_zero(c);
        if (st) return st;
        return gb::check(cudaStreamSynchronize(s));
    }
    return gb::dtrsm_mixed_impl(side, uplo, trans, diag, m, n, alpha, A, lda, B, ldb, tol, prec, max_iter, iters_out,
                                est_err_out, s, leaf);
}

extern "C" int gb_dtrsm_mixed(int side, int uplo, int trans, int diag, int64_t m, int64_t n, double alpha,
                              const double *A, int64_t lda, double *B, int64_t ldb, double tol, int prec,
                              int max_iter, int *iters_out, double *est_err_out, void *stream)
{
    return dtrsm_mixed_entry(side, uplo, trans, diag, m, n, alpha, A, lda, B, ldb, tol, prec, max_iter, 0,
                             iters_out, est_err_out, stream);
}

extern "C" int gb_dtrsm_mixed_leaf(int side, int uplo, int trans, int diag, int64_t m, int64_t n, double alpha,
                                   const double *A, int64_t lda, double *B, int64_t ldb, double tol, int prec,
                                   int max_iter, int64_t leaf, int *iters_out, double *est_err_out, void *stream)
{
    if (leaf != 0 && (leaf < 128 || leaf > 8192 || leaf % 128 != 0)) {
        if (iters_out) *iters_out = 0;
        if (est_err_out) *est_err_out = 0;
        return -15;
    }
    return dtrsm_mixed_entry(side, uplo, trans, diag, m, n, alpha, A, lda, B, ldb, tol, prec, max_iter, leaf,
                             iters_out, est_err_out, stream);
}

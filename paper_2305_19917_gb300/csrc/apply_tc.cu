// Leaf step of the mixed-precision low-precision solve on the tensor cores.
// Each 128-row block b of a leaf (the TS(i) leaves of Section V-A, solved
// left-looking inside the leaf) takes
//
//     Y_b -= L(b, s0:b0) X(s0:b0)        (BF16 products, FP32 in tensor memory)
//     X_b  = L_b^-1 Y_b                  (precomputed 128 x 128 inverse)
//
// in one kernel, in place on the FP32 Y and its BF16 copy.  A plain BF16
// product with the inverse would add a 2^-9 relative error to every block
// solve; instead both factors are split into two BF16 terms, L^-1 = Lh + Ll
// and Y = Yh + Yl, and the three products Lh Yh + Lh Yl + Ll Yh accumulate
// in FP32: the dropped Ll Yl term and the splitting leave about 2^-16
// relative error, below that of the BF16 trailing updates around it.
#include <cuda_bf16.h>
#include "common.cuh"
#include "tc_common.cuh"

namespace gb {

int *device_status_word();

namespace {

constexpr int TB = 128;                    // rows of the block = K = panel width
constexpr uint32_t HALF_BYTES = TB * 128;  // 128 rows x 64 BF16 (one 128-byte swizzle column)
constexpr uint32_t OP_BYTES = 2 * HALF_BYTES;
constexpr uint32_t PANEL_BYTES = TB * TB * 4;  // FP32 staging of the panel, [column][row]

// Byte offset of element (row r, k) of a K-major BF16 operand with K = 128
// stored as two 64-wide halves of 128-byte rows in the 128-byte swizzle
// (16-byte chunk c of row r sits at chunk position c ^ (r mod 8)).
__device__ __forceinline__ uint32_t sw128_off(int r, int k)
{
    const int h = k >> 6, c = (k & 63) >> 3;
    return uint32_t(h) * HALF_BYTES + uint32_t(r) * 128u + uint32_t((c ^ (r & 7)) << 4) + uint32_t(k & 7) * 2u;
}

__device__ __forceinline__ void cp_async16_zfill(void *dst, const void *src, bool in)
{
    const int n = in ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(tc::smem_u32(dst)), "l"(src), "r"(n)
                 : "memory");
}

constexpr int NTH = 256;

// One leaf of the low-precision solve, left-looking, in one launch: for its
// blocks b = 0, 1, ..., nblk-1 (rows b0 = s0 + 128 b .. b0 + 127)
//     Y_b -= L(b, s0:b0) X(s0:b0)          (BF16 tensor cores, FP32 in TMEM)
//     X_b  = L_b^-1 Y_b                    (two-term BF16 split, as above)
// One CTA per 128-column panel walks the blocks in order: the columns of
// the right-hand side are independent, so a panel needs only its own X of
// the earlier blocks, which it wrote itself (stores, then a proxy fence
// before the tensor-memory-access reads of them) -- no launch, prologue or
// grid-wide wait between blocks.  Per block: the GEMM operands stream
// through a 3-stage TMA ring (A rows of the BF16 copy of Mv, X's BF16 copy;
// the ring position runs on across blocks), the FP32 panel and the
// inverse's two terms arrive meanwhile, the ring then holds the split panel.
// While a block's X is stored, the next block's FP32 panel, inverse and
// first k-tiles (those not needing that X) are already on their way.
// Thread 0 issues TMA, thread 32 the MMAs; all 8 warps do the subtraction,
// the split and the stores (warps w, w+4 share TMEM lanes 32(w%4).. and
// split the columns).
constexpr int LST = 3;                                  // ring stages
constexpr uint32_t LA_BYTES = TB * 64 * 2;              // 128 rows x 64 K of A
constexpr uint32_t LB_BYTES = TB * 64 * 2;              // 128 columns x 64 K of X
constexpr uint32_t LSTAGE = LA_BYTES + LB_BYTES;
static_assert(LST * LSTAGE >= 2 * OP_BYTES, "the ring holds the split panel afterwards");
constexpr size_t LEAF_SMEM = 1024 + LST * size_t(LSTAGE) + PANEL_BYTES + 2 * size_t(OP_BYTES) + 256;

__global__ void __launch_bounds__(NTH, 1)
leaf_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmX,
               const __grid_constant__ CUtensorMap tmL, int s0, int nblk, int kp, float *__restrict__ Y,
               int64_t ldy, __nv_bfloat16 *__restrict__ Ybf, int64_t ncols, int *status)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *ring = base;                                         // LST stages, later the split panel
    float *sP = reinterpret_cast<float *>(base + LST * LSTAGE);   // FP32 panel, [column][row]
    uint8_t *sLh = base + LST * LSTAGE + PANEL_BYTES, *sLl = sLh + OP_BYTES;
    uint8_t *sYh = ring, *sYl = ring + OP_BYTES;
    __shared__ uint64_t full[LST], empty[LST], bar_g, bar_l, bar_x;
    __shared__ uint32_t tslot;
    __shared__ int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t c0 = int64_t(blockIdx.x) * TB;
    tc::pdl_launch_dependents();

    if (tid == 0) {
        for (int i = 0; i < LST; i++) {
            tc::mbar_init(&full[i], 1);
            tc::mbar_init(&empty[i], 1);
        }
        tc::mbar_init(&bar_g, 1);
        tc::mbar_init(&bar_l, 1);
        tc::mbar_init(&bar_x, 1);
        abort_flag = 0;
        tc::fence_barrier_init();
    }
    if (warp == 0) tc::tmem_alloc(&tslot, 2 * TB);  // [0,128): L(b,.) X,  [128,256): L_b^-1 Y_b
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = tslot;
    volatile int *ab = &abort_flag;
    tc::pdl_wait();  // Y, its BF16 copy: the previous kernel's until it completes
    const int q = warp & 3, half = warp >> 2;
    const int r = q * 32 + lane;
    uint32_t g = 0;  // ring position (k-tiles issued so far)
    int pre = 0;     // thread 0: k-tiles of the current block issued during the previous one

    // the FP32 panel of Y_b (rows b0..), every copy in flight at once
    auto load_panel = [&](int b0) {
        for (int idx = tid; idx < TB * TB / 4; idx += NTH) {
            const int j = idx >> 5, k4 = (idx & 31) * 4;
            const int64_t col = c0 + j;
            const bool in = col < ncols;
            cp_async16_zfill(sP + j * TB + k4, in ? Y + b0 + k4 + col * ldy : Y, in);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    // thread 0: the inverse's two terms for block b0
    auto load_inverse = [&](int b0) {
        tc::mbar_arrive_expect_tx(&bar_l, 2 * OP_BYTES);
        tc::tma_load_2d(&tmL, &bar_l, sLh, 0, b0);
        tc::tma_load_2d(&tmL, &bar_l, sLh + HALF_BYTES, 64, b0);
        tc::tma_load_2d(&tmL, &bar_l, sLl, 0, kp + b0);
        tc::tma_load_2d(&tmL, &bar_l, sLl + HALF_BYTES, 64, kp + b0);
    };
    // thread 0: k-tile kt of the GEMM of block b0 into ring position gi
    auto load_ktile = [&](uint32_t gi, int kt, int b0) -> bool {
        const int st = int(gi % LST);
        const uint32_t phs = (gi / LST) & 1u;
        if (!tc::mbar_wait(&empty[st], phs ^ 1, ab, status, tc::TC_TIMEOUT_PRODUCER)) return false;
        tc::mbar_arrive_expect_tx(&full[st], LSTAGE);
        tc::tma_load_2d(&tmA, &full[st], ring + st * LSTAGE, s0 + kt * 64, b0);
        tc::tma_load_2d(&tmX, &full[st], ring + st * LSTAGE + LA_BYTES, s0 + kt * 64, int(c0));
        return true;
    };
    load_panel(s0);
    if (tid == 0) {
        tc::tma_prefetch_desc(&tmL);
        load_inverse(s0);
    }

    for (int blk = 0; blk < nblk; blk++) {
        const int b0 = s0 + blk * TB, nk = blk * (TB / 64);
        const uint32_t ph = uint32_t(blk) & 1u;
        if (tid == 0) {
            for (int kt = pre; kt < nk; kt++)
                if (!load_ktile(g + uint32_t(kt), kt, b0)) break;
        } else if (tid == 32) {
            constexpr uint32_t idesc = tc::idesc_bf16_f32(TB, TB);
            for (int kt = 0; kt < nk; kt++) {
                const uint32_t gi = g + uint32_t(kt);
                const int st = int(gi % LST);
                const uint32_t phs = (gi / LST) & 1u;
                if (!tc::mbar_wait(&full[st], phs, ab, status, tc::TC_TIMEOUT_MMA)) break;
                tc::tc_fence_after();
                // descriptors in 16-byte units: a 32-byte K step adds 2
                const uint32_t a0 = tc::smem_u32(ring + st * LSTAGE);
                const uint64_t da = tc::desc_kmajor_sw128(a0), dx = tc::desc_kmajor_sw128(a0 + LA_BYTES);
                tc::mma_f16(tmem, da, dx, idesc, kt != 0);
#pragma unroll
                for (int kk = 1; kk < 4; kk++) tc::mma_f16(tmem, da + uint64_t(2 * kk), dx + uint64_t(2 * kk), idesc, 1);
                tc::mma_commit(&empty[st]);
            }
            tc::mma_commit(&bar_g);  // also when nk == 0: arrives once the earlier MMAs are done
        }
        g += uint32_t(nk);
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncthreads();
        // Y_b - L(b, s0:b0) X(s0:b0), in place in the panel
        const bool ok_g = tc::mbar_wait(&bar_g, ph, ab, status, tc::TC_TIMEOUT_EPILOGUE);
        if (ok_g && nk > 0) {
            tc::tc_fence_after();
#pragma unroll 1
            for (int cc = half * (TB / 2); cc < (half + 1) * (TB / 2); cc += 32) {
                uint32_t x[32];
                tc::tmem_ld32(tmem + (uint32_t(q * 32) << 16) + uint32_t(cc), x);
                tc::tmem_ld_wait();
#pragma unroll
                for (int e = 0; e < 32; e++) sP[(cc + e) * TB + r] -= __uint_as_float(x[e]);
            }
        }
        tc::tc_fence_before();
        __syncthreads();  // the panel is complete and the ring is free (all MMAs of the GEMM are done)
        for (int task = tid; task < TB * 16; task += NTH) {
            const int j = task >> 4, k0 = (task & 15) * 8;
            const float4 a = *reinterpret_cast<const float4 *>(sP + j * TB + k0);
            const float4 b = *reinterpret_cast<const float4 *>(sP + j * TB + k0 + 4);
            const float v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
            uint32_t hw[4], lw[4];
#pragma unroll
            for (int e = 0; e < 8; e += 2) {
                const __nv_bfloat162 h = __floats2bfloat162_rn(v[e], v[e + 1]);
                const __nv_bfloat162 l = __floats2bfloat162_rn(v[e] - __low2float(h), v[e + 1] - __high2float(h));
                hw[e / 2] = *reinterpret_cast<const uint32_t *>(&h);
                lw[e / 2] = *reinterpret_cast<const uint32_t *>(&l);
            }
            const uint32_t off = sw128_off(j, k0);
            *reinterpret_cast<uint4 *>(sYh + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
            *reinterpret_cast<uint4 *>(sYl + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (blk + 1 < nblk) load_panel(b0 + TB);  // the panel is free again: the next block's
        if (tid == 32) {
            if (ok_g && tc::mbar_wait(&bar_l, ph, ab, status, tc::TC_TIMEOUT_MMA)) {
                tc::tc_fence_after();
                constexpr uint32_t idesc = tc::idesc_bf16_f32(TB, TB);
                const uint8_t *As[3] = {sLh, sLh, sLl};
                const uint8_t *Bs[3] = {sYh, sYl, sYh};
                uint32_t acc = 0;
#pragma unroll
                for (int pr = 0; pr < 3; pr++) {
                    const uint64_t da = tc::desc_kmajor_sw128(tc::smem_u32(As[pr]));
                    const uint64_t dy = tc::desc_kmajor_sw128(tc::smem_u32(Bs[pr]));
#pragma unroll
                    for (int kk = 0; kk < TB / 16; kk++) {
                        const uint64_t o = uint64_t(((kk >> 2) * HALF_BYTES + (kk & 3) * 32u) >> 4);
                        tc::mma_f16(tmem + TB, da + o, dy + o, idesc, acc);
                        acc = 1;
                    }
                }
            }
            tc::mma_commit(&bar_x);
        }
        const bool ok_x = tc::mbar_wait(&bar_x, ph, ab, status, tc::TC_TIMEOUT_EPILOGUE);
        pre = 0;
        if (ok_x && tid == 0 && blk + 1 < nblk) {
            // the split panel and the inverse are consumed: the next block's
            // inverse, and its first k-tiles that do not need this block's X
            // (rows below b0), go out while this block's X is stored
            load_inverse(b0 + TB);
            const int nkn = (blk + 1) * (TB / 64);
            pre = min(LST, nkn - TB / 64);
            for (int kt = 0; kt < pre; kt++)
                if (!load_ktile(g + uint32_t(kt), kt, b0 + TB)) {
                    pre = nkn;  // stop issuing: the wait has timed out and set the abort flag
                    break;
                }
        }
        if (ok_x && !*ab) {
            tc::tc_fence_after();
#pragma unroll 1
            for (int cc = half * (TB / 2); cc < (half + 1) * (TB / 2); cc += 32) {
                uint32_t x[32];
                tc::tmem_ld32(tmem + (uint32_t(q * 32) << 16) + uint32_t(TB + cc), x);
                tc::tmem_ld_wait();
#pragma unroll
                for (int e = 0; e < 32; e++) {
                    const int64_t col = c0 + cc + e;
                    if (col < ncols) {
                        const float val = __uint_as_float(x[e]);
                        Y[b0 + r + col * ldy] = val;
                        Ybf[b0 + r + col * ldy] = __float2bfloat16_rn(val);
                    }
                }
            }
        }
        // X_b's BF16 copy is read by the tensor memory accesses of the next blocks
        asm volatile("fence.proxy.async.global;" ::: "memory");
        tc::tc_fence_before();
        __syncthreads();
        if (*ab) break;
    }
    tc::tc_fence_after();
    if (warp == 0) tc::tmem_dealloc(tmem, 2 * TB);
}

}  // namespace

int apply_tc_prepare()
{
    static PerDeviceOnce attr;
    return smem_attr_once(attr, leaf_tc_kernel, LEAF_SMEM);
}

// One leaf of the low-precision solve: rows s0 .. s0 + nr - 1 (s0 and nr
// multiples of 128), every 128-row block updated from the leaf's solved
// blocks and solved with its inverse, over all np columns.  Abf: BF16 Mv,
// row-major, leading dimension kp; Y / Ybf: the FP32 right-hand side and its
// BF16 copy (column-major, kp); inv16: the inverses' high terms in rows
// b*128.., their low terms in rows kp + b*128.. (128 wide).
int launch_leaf_tc(const __nv_bfloat16 *Abf, const __nv_bfloat16 *inv16, int64_t kp, int64_t np, int64_t s0,
                   int64_t nr, float *Y, __nv_bfloat16 *Ybf, cudaStream_t s, int *status)
{
    if (np <= 0 || nr <= 0) return 0;
    if (kp % TB || np % TB || s0 % TB || nr % TB || s0 + nr > kp || 2 * kp > 0x7fffffffLL ||
        (reinterpret_cast<uintptr_t>(Y) & 15) || (reinterpret_cast<uintptr_t>(Abf) & 15) ||
        (reinterpret_cast<uintptr_t>(Ybf) & 15) || (reinterpret_cast<uintptr_t>(inv16) & 15))
        return GB_STATUS_CUDA_ERROR;
    CUtensorMap ta, tx, tl;
    {
        uint64_t dims[2] = {uint64_t(kp), uint64_t(kp)};
        uint64_t strides[1] = {uint64_t(kp) * 2};
        uint32_t box[2] = {64, TB};
        GB_TRY(encode_tmap(&ta, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, Abf, dims, strides, box));
    }
    {
        uint64_t dims[2] = {uint64_t(kp), uint64_t(np)};
        uint64_t strides[1] = {uint64_t(kp) * 2};
        uint32_t box[2] = {64, TB};
        GB_TRY(encode_tmap(&tx, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, Ybf, dims, strides, box));
    }
    {
        uint64_t dims[2] = {uint64_t(TB), uint64_t(2 * kp)};
        uint64_t strides[1] = {uint64_t(TB) * 2};
        uint32_t box[2] = {64, TB};
        GB_TRY(encode_tmap(&tl, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, inv16, dims, strides, box));
    }
    GB_TRY(apply_tc_prepare());
    int *st = status ? status : device_status_word();
    if (!st) return GB_STATUS_CUDA_ERROR;
    const double nrd = double(nr);
    // GEMM flops of the leaf (sum over blocks of 2 * 128 * K * np) plus the 3 split products per block
    LaunchScope ls(KK_DIAG, s, (nrd * (nrd - TB) + 3.0 * 2.0 * TB * nrd) * double(np),
                   nrd * nrd + nrd * (nrd - TB) / TB * double(np) + 10.0 * nrd * double(np));
    return check(launch_pdl(leaf_tc_kernel, dim3((unsigned)(np / TB)), dim3(NTH), LEAF_SMEM, s, ta, tx, tl, int(s0),
                            int(nr / TB), int(kp), Y, kp, Ybf, np, st));
}

}  // namespace gb

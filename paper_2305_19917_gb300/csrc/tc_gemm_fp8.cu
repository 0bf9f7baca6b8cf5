// FP8 (E4M3) tensor-core GEMM update with per-block power-of-two scales:
//     C = alpha*C - sum_kb  sA(I,kb) sB(kb,J) (A8(I,kb) B8(kb,J))
// for the low-precision solve of the mixed-precision path (the paper's gemm
// task, Section IV stage 2).  A8 is M x K row-major FP8 with one scale per
// 128 x 128 block, B8 is K x N column-major FP8 with one scale per 128 (K) x
// 64 (N) block; all scales are powers of two.
//
// A block scale changes at every 128-wide K block, so partial products cannot
// simply accumulate in tensor memory: each K block (one 128-byte swizzle row
// of FP8, 4 MMAs of K = 32) goes to one of two TMEM accumulators, and the
// four epilogue warps read it back, multiply by the block's two scales
// (exact) and add it to FP32 registers while the MMAs of the next block run
// into the other accumulator.  Tile 128 x 128, 6-stage TMA ring.
#include <cuda_fp8.h>
#include "common.cuh"
#include "tc_common.cuh"

namespace gb {

int *device_status_word();

namespace {

constexpr int BM = 128, BN = 128, BK = 128, STAGES = 6;
constexpr uint32_t A_BYTES = BM * BK, B_BYTES = BN * BK;
constexpr uint32_t STAGE_BYTES = A_BYTES + B_BYTES;
constexpr size_t SMEM_BYTES = 1024 + STAGES * size_t(STAGE_BYTES) + 256;

__global__ void __launch_bounds__(192, 1)
tc_gemm_fp8_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   float *__restrict__ C, int64_t ldc, int M, int N, int K, float alpha,
                   const float *__restrict__ sA, int64_t ldsa, const float *__restrict__ sB, int64_t ldsb,
                   int nMt, int nNt, int *status)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *sAm = base;
    uint8_t *sBm = base + STAGES * A_BYTES;
    uint64_t *full = reinterpret_cast<uint64_t *>(sBm + STAGES * B_BYTES);
    uint64_t *empty = full + STAGES;
    uint64_t *accf = empty + STAGES;  // [2]
    uint64_t *acce = accf + 2;        // [2]
    uint32_t *tslot = reinterpret_cast<uint32_t *>(acce + 2);
    __shared__ int abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int m_blk, n_blk;
    tc::raster_grouped(int(blockIdx.x), nMt, nNt, 8, m_blk, n_blk);
    const int nk = K / BK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; s++) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; b++) {
            tc::mbar_init(&accf[b], 1);
            tc::mbar_init(&acce[b], 4);  // one arrival per epilogue warp
        }
        abort_flag = 0;
        tc::fence_barrier_init();
    }
    if (warp == 1) tc::tmem_alloc(tslot, 2 * BN);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tslot;
    volatile int *ab = &abort_flag;

    if (warp == 0) {
        if (lane == 0) {
            tc::tma_prefetch_desc(&tmA);
            tc::tma_prefetch_desc(&tmB);
            for (int kt = 0; kt < nk; kt++) {
                const int s = kt % STAGES;
                const uint32_t ph = (kt / STAGES) & 1;
                if (!tc::mbar_wait(&empty[s], ph ^ 1, ab, status, tc::TC_TIMEOUT_PRODUCER)) break;
                tc::mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
                tc::tma_load_2d(&tmA, &full[s], sAm + s * A_BYTES, kt * BK, m_blk * BM);
                tc::tma_load_2d(&tmB, &full[s], sBm + s * B_BYTES, kt * BK, n_blk * BN);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = tc::idesc_e4m3_f32(BM, BN);
            // descriptors from the ring's base ones (16-byte units: a 32-byte K step adds 2)
            const uint64_t dA0 = tc::desc_kmajor_sw128(tc::smem_u32(sAm)), dB0 = tc::desc_kmajor_sw128(tc::smem_u32(sBm));
            for (int kt = 0; kt < nk; kt++) {
                const int s = kt % STAGES;
                const uint32_t ph = (kt / STAGES) & 1;
                const int buf = kt & 1;
                if (!tc::mbar_wait(&acce[buf], ((kt >> 1) & 1) ^ 1, ab, status, tc::TC_TIMEOUT_MMA)) break;
                if (!tc::mbar_wait(&full[s], ph, ab, status, tc::TC_TIMEOUT_MMA)) break;
                tc::tc_fence_after();
                const uint64_t da = dA0 + uint64_t(uint32_t(s) * (A_BYTES >> 4));
                const uint64_t db = dB0 + uint64_t(uint32_t(s) * (B_BYTES >> 4));
#pragma unroll
                for (int kk = 0; kk < BK / 32; kk++)
                    tc::mma_f8(tmem + uint32_t(buf * BN), da + uint64_t(2 * kk), db + uint64_t(2 * kk), idesc, kk != 0);
                tc::mma_commit(&empty[s]);
                tc::mma_commit(&accf[buf]);
            }
        }
    } else {
        const int q = warp & 3;
        const int row = q * 32 + lane;
        const int64_t gi = int64_t(m_blk) * BM + row;
        float acc[BN];
#pragma unroll
        for (int c = 0; c < BN; c++) acc[c] = 0.f;
        bool ok = true;
        for (int kt = 0; kt < nk; kt++) {
            const int buf = kt & 1;
            if (!tc::mbar_wait(&accf[buf], (kt >> 1) & 1, ab, status, tc::TC_TIMEOUT_EPILOGUE)) {
                ok = false;
                break;
            }
            tc::tc_fence_after();
            const float sa = sA[int64_t(m_blk) * ldsa + kt];
            const float sb0 = sB[int64_t(kt) * ldsb + 2 * n_blk], sb1 = sB[int64_t(kt) * ldsb + 2 * n_blk + 1];
            const float s0 = sa * sb0, s1 = sa * sb1;
            const uint32_t tb = tmem + (uint32_t(q * 32) << 16) + uint32_t(buf * BN);
#pragma unroll
            for (int c0 = 0; c0 < BN; c0 += 32) {
                uint32_t r[32];
                tc::tmem_ld32(tb + c0, r);
                tc::tmem_ld_wait();
                const float sc = c0 < 64 ? s0 : s1;
#pragma unroll
                for (int j = 0; j < 32; j++) acc[c0 + j] = fmaf(sc, __uint_as_float(r[j]), acc[c0 + j]);
            }
            tc::tc_fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&acce[buf]);
        }
        if (ok && gi < M) {
#pragma unroll
            for (int c0 = 0; c0 < BN; c0 += 16) {
                float cv[16];
                const int64_t gj0 = int64_t(n_blk) * BN + c0;
#pragma unroll
                for (int j = 0; j < 16; j++) cv[j] = (gj0 + j < N) ? C[gi + (gj0 + j) * ldc] : 0.f;
#pragma unroll
                for (int j = 0; j < 16; j++)
                    if (gj0 + j < N) C[gi + (gj0 + j) * ldc] = alpha * cv[j] - acc[c0 + j];
            }
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, 2 * BN);
    }
}

}  // namespace

int tc_gemm_fp8_prepare()
{
    static PerDeviceOnce attr;
    return smem_attr_once(attr, tc_gemm_fp8_kernel, SMEM_BYTES);
}

// C (M x N FP32 column-major) = alpha*C - A8*B8 with the block scales above;
// A8 row-major (lda bytes per row), B8 column-major (ldb bytes per column);
// M, K multiples of 128 at 128-aligned block positions, N a multiple of 64;
// sA: scales of the row block of A this call starts at (ldsa per 128 rows,
// one per 128-wide K block), sB: scales of B's first K block (ldsb per K
// block, one per 64 columns).
int launch_tc_gemm_fp8(int64_t M, int64_t N, int64_t K, const void *A, int64_t lda, const void *B, int64_t ldb,
                       float *C, int64_t ldc, float alpha, const float *sA, int64_t ldsa, const float *sB,
                       int64_t ldsb, cudaStream_t s, int *status)
{
    if (M <= 0 || N <= 0) return 0;
    if (K <= 0 || K % BK || N % BN || lda % 16 || ldb % 16 || (reinterpret_cast<uintptr_t>(A) & 15) ||
        (reinterpret_cast<uintptr_t>(B) & 15))
        return GB_STATUS_CUDA_ERROR;
    CUtensorMap ta, tb;
    {
        uint64_t dims[2] = {uint64_t(K), uint64_t(M)};
        uint64_t strides[1] = {uint64_t(lda)};
        uint32_t box[2] = {BK, BM};
        GB_TRY(encode_tmap(&ta, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, A, dims, strides, box));
    }
    {
        uint64_t dims[2] = {uint64_t(K), uint64_t(N)};
        uint64_t strides[1] = {uint64_t(ldb)};
        uint32_t box[2] = {BK, BN};
        GB_TRY(encode_tmap(&tb, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, B, dims, strides, box));
    }
    GB_TRY(tc_gemm_fp8_prepare());
    int *st = status ? status : device_status_word();
    if (!st) return GB_STATUS_CUDA_ERROR;
    const int64_t nM = (M + BM - 1) / BM, nN = (N + BN - 1) / BN;
    if (nM * nN > 0x7fffffffLL) return GB_STATUS_CUDA_ERROR;
    LaunchScope ls(KK_GEMM_TC, s, 2.0 * M * N * K, double(M) * K + double(K) * N + 8.0 * M * N);
    tc_gemm_fp8_kernel<<<(unsigned)(nM * nN), 192, SMEM_BYTES, s>>>(ta, tb, C, ldc, (int)M, (int)N, (int)K, alpha,
                                                                     sA, ldsa, sB, ldsb, (int)nM, (int)nN, st);
    return check(cudaGetLastError());
}

}  // namespace gb

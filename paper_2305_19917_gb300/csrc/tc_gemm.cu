// Tensor-core GEMM update C = alpha*C - A*B on sm_103a (tcgen05 + TMA): the
// paper's gemm task (Section IV stage 2, Section V) in the low-precision
// solve of the mixed-precision path.  A (M x K) and B (K x N) are BF16, the
// product accumulates in FP32 in tensor memory, C is FP32.
//
// Layout: A row-major (K-major), B column-major (K-major as the MMA's B
// operand), C column-major.  One CTA per 128 x BN output tile (BN = 256, 128
// or 64); K advances in 64-element steps (one 128-byte swizzle row) through
// a TMA ring of ~192 KB (4, 5 or 8 stages).
// Warp roles: warp 0 issues TMA loads, warp 1 owns TMEM and issues the MMAs
// (one elected thread), warps 2-5 drain the accumulator (each warp reads the
// 32 TMEM lanes its rank allows) and apply the FP32 epilogue with coalesced
// column-major stores.
#include <cstdio>
#include "common.cuh"
#include "tc_common.cuh"

namespace gb {

// ---- host: tensor-map encoding through the driver entry point ---------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                                  CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                  CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

int encode_tmap(CUtensorMap *map, CUtensorMapDataType dt, int rank, const void *base, const uint64_t *dims,
                const uint64_t *strides_bytes, const uint32_t *box)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return GB_STATUS_CUDA_ERROR;
    cuuint64_t gd[5], gs[4];
    cuuint32_t bx[5], es[5];
    for (int i = 0; i < rank; i++) {
        gd[i] = dims[i];
        bx[i] = box[i];
        es[i] = 1;
        if (i + 1 < rank) gs[i] = strides_bytes[i];
    }
    CUresult r = fn(map, dt, (cuuint32_t)rank, const_cast<void *>(base), gd, gs, bx, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_cuda_error(cudaErrorInvalidValue);
        return GB_STATUS_CUDA_ERROR;
    }
    return 0;
}

// ---- device status word (timeouts of bounded waits) -------------------------
static int *g_status[64] = {nullptr};

int *device_status_word()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    if (!g_status[dev]) {
        int *p = nullptr;
        if (cudaMalloc(&p, sizeof(int)) != cudaSuccess) return nullptr;
        if (cudaMemset(p, 0, sizeof(int)) != cudaSuccess) return nullptr;
        g_status[dev] = p;
    }
    return g_status[dev];
}

namespace {

constexpr int BM = 128, BK = 64;
constexpr uint32_t A_BYTES = BM * BK * 2;

// Tile shape per N-tile width: stages fill ~192 KB of shared memory.
template <int BN>
struct TileCfg {
    static constexpr uint32_t B_BYTES = BN * BK * 2;
    static constexpr uint32_t STAGE_BYTES = A_BYTES + B_BYTES;
    static constexpr int STAGES = (192 * 1024) / STAGE_BYTES > 8 ? 8 : (192 * 1024) / STAGE_BYTES;
    static constexpr size_t SMEM_BYTES = 1024 + STAGES * size_t(STAGE_BYTES) + 256;
    // a short K needs fewer stages; the smaller footprint lets several CTAs
    // share an SM (thin updates are latency-bound)
    static size_t smem_for(int nst) { return 1024 + nst * size_t(STAGE_BYTES) + 256; }
};

template <int BN>
__global__ void __launch_bounds__(192, 1)
tc_gemm_bf16_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                    float *__restrict__ C, int64_t ldc, int M, int N, int K, float alpha, int nMt, int nNt,
                    int STAGES, int *status)
{
    constexpr uint32_t B_BYTES = TileCfg<BN>::B_BYTES;
    constexpr uint32_t STAGE_BYTES = TileCfg<BN>::STAGE_BYTES;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *sA = base;
    uint8_t *sB = base + STAGES * A_BYTES;
    uint64_t *full = reinterpret_cast<uint64_t *>(sB + STAGES * B_BYTES);
    uint64_t *empty = full + STAGES;
    uint64_t *accf = empty + STAGES;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(accf + 1);
    __shared__ int abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int m_blk, n_blk;
    tc::raster_grouped(int(blockIdx.x), nMt, nNt, 8, m_blk, n_blk);
    const int nk = K / BK;
    tc::pdl_launch_dependents();

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; s++) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        tc::mbar_init(accf, 1);
        abort_flag = 0;
        tc::fence_barrier_init();
    }
    if (warp == 1) tc::tmem_alloc(tslot, BN < 32 ? 32 : BN);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tslot;
    volatile int *ab = &abort_flag;
    tc::pdl_wait();  // A, B and C belong to the previous kernel until it completes

    if (warp == 0) {
        if (lane == 0) {
            tc::tma_prefetch_desc(&tmA);
            tc::tma_prefetch_desc(&tmB);
            for (int kt = 0; kt < nk; kt++) {
                const int s = kt % STAGES;
                const uint32_t ph = (kt / STAGES) & 1;
                if (!tc::mbar_wait(&empty[s], ph ^ 1, ab, status, tc::TC_TIMEOUT_PRODUCER)) break;
                tc::mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
                tc::tma_load_2d(&tmA, &full[s], sA + s * A_BYTES, kt * BK, m_blk * BM);
                tc::tma_load_2d(&tmB, &full[s], sB + s * B_BYTES, kt * BK, n_blk * BN);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = tc::idesc_bf16_f32(BM, BN);
            // descriptors from the ring's base ones (16-byte units: a 32-byte K step adds 2)
            const uint64_t dA0 = tc::desc_kmajor_sw128(tc::smem_u32(sA)), dB0 = tc::desc_kmajor_sw128(tc::smem_u32(sB));
            for (int kt = 0; kt < nk; kt++) {
                const int s = kt % STAGES;
                const uint32_t ph = (kt / STAGES) & 1;
                if (!tc::mbar_wait(&full[s], ph, ab, status, tc::TC_TIMEOUT_MMA)) break;
                tc::tc_fence_after();
                const uint64_t da = dA0 + uint64_t(uint32_t(s) * (A_BYTES >> 4));
                const uint64_t db = dB0 + uint64_t(uint32_t(s) * (B_BYTES >> 4));
                tc::mma_f16(tmem, da, db, idesc, kt != 0);
#pragma unroll
                for (int kk = 1; kk < BK / 16; kk++) tc::mma_f16(tmem, da + uint64_t(2 * kk), db + uint64_t(2 * kk), idesc, 1);
                tc::mma_commit(&empty[s]);
            }
            tc::mma_commit(accf);
        }
    } else {
        // epilogue: 4 warps, warp w reads TMEM lanes 32*(w%4) .. +31
        const int q = warp & 3;
        const int row = q * 32 + lane;
        const int64_t gi = int64_t(m_blk) * BM + row;
        if constexpr (BN <= 64) {
            // narrow tiles serve thin updates (small K): the C tile is read
            // while the loads and MMAs run
            float cp[BN];
            const int64_t gj0 = int64_t(n_blk) * BN;
            if (gi < M) {
#pragma unroll
                for (int j = 0; j < BN; j++) cp[j] = (gj0 + j < N) ? C[gi + (gj0 + j) * ldc] : 0.f;
            }
            if (tc::mbar_wait(accf, 0, ab, status, tc::TC_TIMEOUT_EPILOGUE)) {
                tc::tc_fence_after();
#pragma unroll
                for (int c0 = 0; c0 < BN; c0 += 32) {
                    uint32_t r[32];
                    tc::tmem_ld32(tmem + (uint32_t(q * 32) << 16) + uint32_t(c0), r);
                    tc::tmem_ld_wait();
                    if (gi < M) {
#pragma unroll
                        for (int j = 0; j < 32; j++)
                            if (gj0 + c0 + j < N)
                                C[gi + (gj0 + c0 + j) * ldc] = alpha * cp[c0 + j] - __uint_as_float(r[j]);
                    }
                }
            }
        } else if (tc::mbar_wait(accf, 0, ab, status, tc::TC_TIMEOUT_EPILOGUE)) {
            tc::tc_fence_after();
#pragma unroll 1
            for (int c0 = 0; c0 < BN; c0 += 32) {
                uint32_t r[32];
                tc::tmem_ld32(tmem + (uint32_t(q * 32) << 16) + uint32_t(c0), r);
                tc::tmem_ld_wait();
                if (gi < M) {
                    // all 32 loads are issued before any store (the compiler
                    // cannot prove the column addresses distinct)
                    float cv[32];
                    const int64_t gj0 = int64_t(n_blk) * BN + c0;
#pragma unroll
                    for (int j = 0; j < 32; j++) cv[j] = (gj0 + j < N) ? C[gi + (gj0 + j) * ldc] : 0.f;
#pragma unroll
                    for (int j = 0; j < 32; j++)
                        if (gj0 + j < N) C[gi + (gj0 + j) * ldc] = alpha * cv[j] - __uint_as_float(r[j]);
                }
            }
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, BN < 32 ? 32 : BN);
    }
}

// Persistent form: one CTA per SM walks the 128 x PBN tiles t = blockIdx.x,
// blockIdx.x + gridDim.x, ... (grouped rasterisation) with two TMEM
// accumulators (2 x PBN columns), so that the epilogue of one tile runs while
// the MMAs of the next accumulate into the other buffer.  The TMA ring (about
// 192 KB, sized to K when K is short) runs continuously across tiles.  320
// threads: warp 0 TMA, warp 1 MMA, warps 2-9 epilogue (warps w and w+4 share
// TMEM lane quadrant w % 4 and take one half of the tile's columns each).
template <int PBN>
struct PCfg {
    static constexpr uint32_t B_BYTES = PBN * BK * 2, STAGE_BYTES = A_BYTES + B_BYTES;
    static constexpr int STAGES = (192 * 1024) / STAGE_BYTES > 8 ? 8 : (192 * 1024) / STAGE_BYTES;
    static constexpr uint32_t TMEM_COLS = 2 * PBN < 32 ? 32 : 2 * PBN;
    static size_t smem_for(int nst) { return 1024 + nst * size_t(STAGE_BYTES) + 256; }
};

template <int PBN>
__global__ void __launch_bounds__(320, 1)
tc_gemm_bf16_persistent_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                               float *__restrict__ C, int64_t ldc, int M, int N, int K, float alpha, int nMt,
                               int nNt, int PSTAGES, int *status)
{
    constexpr uint32_t P_B_BYTES = PCfg<PBN>::B_BYTES, P_STAGE_BYTES = PCfg<PBN>::STAGE_BYTES;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *sA = base;
    uint8_t *sB = base + PSTAGES * A_BYTES;
    uint64_t *full = reinterpret_cast<uint64_t *>(sB + PSTAGES * P_B_BYTES);
    uint64_t *empty = full + PSTAGES;
    uint64_t *tfull = empty + PSTAGES;  // [2] accumulator ready
    uint64_t *tempty = tfull + 2;       // [2] accumulator drained
    uint32_t *tslot = reinterpret_cast<uint32_t *>(tempty + 2);
    __shared__ int abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nk = K / BK;
    const int ntiles = nMt * nNt;
    tc::pdl_launch_dependents();

    if (threadIdx.x == 0) {
        for (int s = 0; s < PSTAGES; s++) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; b++) {
            tc::mbar_init(&tfull[b], 1);
            tc::mbar_init(&tempty[b], 8);  // one arrival per epilogue warp
        }
        abort_flag = 0;
        tc::fence_barrier_init();
    }
    if (warp == 1) tc::tmem_alloc(tslot, PCfg<PBN>::TMEM_COLS);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tslot;
    volatile int *ab = &abort_flag;
    tc::pdl_wait();  // A, B and C belong to the previous kernel until it completes

    if (warp == 0) {
        if (lane == 0) {
            tc::tma_prefetch_desc(&tmA);
            tc::tma_prefetch_desc(&tmB);
            uint32_t kg = 0;
            for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
                int m_blk, n_blk;
                tc::raster_grouped(t, nMt, nNt, 8, m_blk, n_blk);
                bool ok = true;
                for (int kt = 0; kt < nk; kt++, kg++) {
                    const int s = kg % PSTAGES;
                    const uint32_t ph = (kg / PSTAGES) & 1;
                    if (!tc::mbar_wait(&empty[s], ph ^ 1, ab, status, tc::TC_TIMEOUT_PRODUCER)) {
                        ok = false;
                        break;
                    }
                    tc::mbar_arrive_expect_tx(&full[s], P_STAGE_BYTES);
                    tc::tma_load_2d(&tmA, &full[s], sA + s * A_BYTES, kt * BK, m_blk * BM);
                    tc::tma_load_2d(&tmB, &full[s], sB + s * P_B_BYTES, kt * BK, n_blk * PBN);
                }
                if (!ok) break;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = tc::idesc_bf16_f32(BM, PBN);
            // descriptors from the ring's base ones (16-byte units: a 32-byte K step adds
            // 2), and the ring position kept incrementally (no division per K step)
            const uint64_t dA0 = tc::desc_kmajor_sw128(tc::smem_u32(sA)), dB0 = tc::desc_kmajor_sw128(tc::smem_u32(sB));
            int s = 0;
            uint32_t ph = 0;
            int it = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, it++) {
                const int buf = it & 1;
                const uint32_t use = uint32_t(it >> 1);
                if (!tc::mbar_wait(&tempty[buf], (use & 1) ^ 1, ab, status, tc::TC_TIMEOUT_MMA)) break;
                tc::tc_fence_after();
                const uint32_t d = tmem + uint32_t(buf * PBN);
                for (int kt = 0; kt < nk; kt++) {
                    if (!tc::mbar_wait(&full[s], ph, ab, status, tc::TC_TIMEOUT_MMA)) {
                        ok = false;
                        break;
                    }
                    tc::tc_fence_after();
                    const uint64_t da = dA0 + uint64_t(uint32_t(s) * (A_BYTES >> 4));
                    const uint64_t db = dB0 + uint64_t(uint32_t(s) * (P_B_BYTES >> 4));
                    tc::mma_f16(d, da, db, idesc, kt != 0);
#pragma unroll
                    for (int kk = 1; kk < BK / 16; kk++) tc::mma_f16(d, da + uint64_t(2 * kk), db + uint64_t(2 * kk), idesc, 1);
                    tc::mma_commit(&empty[s]);
                    if (++s == PSTAGES) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
                if (ok) tc::mma_commit(&tfull[buf]);
            }
        }
    } else {
        const int q = warp & 3;                 // TMEM lane quadrant of this warp
        const int half = (warp - 2) >> 2;       // which 128 columns of the tile
        const int row = q * 32 + lane;
        int it = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, it++) {
            int m_blk, n_blk;
            tc::raster_grouped(t, nMt, nNt, 8, m_blk, n_blk);
            const int buf = it & 1;
            const uint32_t use = uint32_t(it >> 1);
            if (!tc::mbar_wait(&tfull[buf], use & 1, ab, status, tc::TC_TIMEOUT_EPILOGUE)) break;
            tc::tc_fence_after();
            const int64_t gi = int64_t(m_blk) * BM + row;
#pragma unroll 1
            for (int c0 = half * (PBN / 2); c0 < (half + 1) * (PBN / 2); c0 += 32) {
                uint32_t r[32];
                tc::tmem_ld32(tmem + (uint32_t(q * 32) << 16) + uint32_t(buf * PBN + c0), r);
                tc::tmem_ld_wait();
                if (gi < M) {
                    float cv[32];
                    const int64_t gj0 = int64_t(n_blk) * PBN + c0;
#pragma unroll
                    for (int j = 0; j < 32; j++) cv[j] = (gj0 + j < N) ? C[gi + (gj0 + j) * ldc] : 0.f;
#pragma unroll
                    for (int j = 0; j < 32; j++)
                        if (gj0 + j < N) C[gi + (gj0 + j) * ldc] = alpha * cv[j] - __uint_as_float(r[j]);
                }
            }
            tc::tc_fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&tempty[buf]);
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, PCfg<PBN>::TMEM_COLS);
    }
}

}  // namespace

template <int BN>
static int prepare_bn()
{
    static PerDeviceOnce attr;
    return smem_attr_once(attr, tc_gemm_bf16_kernel<BN>, TileCfg<BN>::SMEM_BYTES);
}

// One-time per-device set-up (kernel attributes); must run before any
// stream capture that launches the kernel.
template <int PBN>
static int prepare_persistent()
{
    static PerDeviceOnce attr;
    return smem_attr_once(attr, tc_gemm_bf16_persistent_kernel<PBN>, PCfg<PBN>::smem_for(PCfg<PBN>::STAGES));
}

static int num_sms()
{
    static int n[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    if (!n[dev] && cudaDeviceGetAttribute(&n[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return n[dev];
}

int tc_gemm_prepare()
{
    GB_TRY(prepare_persistent<256>());
    GB_TRY(prepare_persistent<128>());
    GB_TRY(prepare_persistent<64>());
    if (num_sms() <= 0) return GB_STATUS_CUDA_ERROR;
    return prepare_bn<64>();
}

template <int BN>
static int launch_bn(int64_t M, int64_t N, int64_t K, const void *A, int64_t lda, const void *B, int64_t ldb,
                     float *C, int64_t ldc, float alpha, cudaStream_t s, int *status)
{
    CUtensorMap ta, tb;
    {
        uint64_t dims[2] = {uint64_t(K), uint64_t(M)};
        uint64_t strides[1] = {uint64_t(lda) * 2};
        uint32_t box[2] = {BK, BM};
        GB_TRY(encode_tmap(&ta, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, A, dims, strides, box));
    }
    {
        uint64_t dims[2] = {uint64_t(K), uint64_t(N)};
        uint64_t strides[1] = {uint64_t(ldb) * 2};
        uint32_t box[2] = {BK, uint32_t(BN)};
        GB_TRY(encode_tmap(&tb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, B, dims, strides, box));
    }
    GB_TRY(prepare_bn<BN>());
    int *st = status ? status : device_status_word();
    if (!st) return GB_STATUS_CUDA_ERROR;
    // 1-D grid (grouped rasterisation)
    const int64_t nM = (M + BM - 1) / BM, nN = (N + BN - 1) / BN;
    if (nM > 65535 || nN > 65535 || nM * nN > 0x7fffffffLL) return GB_STATUS_CUDA_ERROR;
    dim3 grid((unsigned)(nM * nN));
    const int nk = int(K / BK);
    const int nst = nk < TileCfg<BN>::STAGES ? nk : TileCfg<BN>::STAGES;
    LaunchScope ls(KK_GEMM_TC, s, 2.0 * M * N * K, 2.0 * (double(M) * K + double(K) * N) + 8.0 * M * N);
    return check(launch_pdl(tc_gemm_bf16_kernel<BN>, grid, dim3(192), TileCfg<BN>::smem_for(nst), s, ta, tb, C,
                            ldc, (int)M, (int)N, (int)K, alpha, (int)nM, (int)nN, nst, st));
}

template <int PBN>
static int launch_persistent(int64_t M, int64_t N, int64_t K, const void *A, int64_t lda, const void *B,
                             int64_t ldb, float *C, int64_t ldc, float alpha, cudaStream_t s, int *status)
{
    CUtensorMap ta, tb;
    {
        uint64_t dims[2] = {uint64_t(K), uint64_t(M)};
        uint64_t strides[1] = {uint64_t(lda) * 2};
        uint32_t box[2] = {BK, BM};
        GB_TRY(encode_tmap(&ta, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, A, dims, strides, box));
    }
    {
        uint64_t dims[2] = {uint64_t(K), uint64_t(N)};
        uint64_t strides[1] = {uint64_t(ldb) * 2};
        uint32_t box[2] = {BK, uint32_t(PBN)};
        GB_TRY(encode_tmap(&tb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, B, dims, strides, box));
    }
    GB_TRY(prepare_persistent<PBN>());
    int *st = status ? status : device_status_word();
    if (!st) return GB_STATUS_CUDA_ERROR;
    const int sms = num_sms();
    if (sms <= 0) return GB_STATUS_CUDA_ERROR;
    const int64_t nM = (M + BM - 1) / BM, nN = (N + PBN - 1) / PBN;
    if (nM * nN > 0x7fffffffLL) return GB_STATUS_CUDA_ERROR;
    const int64_t grid = nM * nN < sms ? nM * nN : sms;
    const int nk = int(K / BK);
    const int nst = nk < PCfg<PBN>::STAGES ? nk : PCfg<PBN>::STAGES;
    LaunchScope ls(KK_GEMM_TC, s, 2.0 * M * N * K, 2.0 * (double(M) * K + double(K) * N) + 8.0 * M * N);
    return check(launch_pdl(tc_gemm_bf16_persistent_kernel<PBN>, dim3((unsigned)grid), dim3(320),
                            PCfg<PBN>::smem_for(nst), s, ta, tb, C, ldc, (int)M, (int)N, (int)K, alpha, (int)nM,
                            (int)nN, nst, st));
}

// C (M x N, FP32, column-major, ldc) = alpha*C - A*B with A (M x K, BF16
// row-major, lda) and B (K x N, BF16 column-major, ldb).  K % 64 == 0,
// lda % 8 == 0, ldb % 8 == 0, A and B 16-byte aligned; `status` is the
// device word that records wait timeouts (nullptr = the library's own word,
// allocated on first use).  The persistent kernel takes the widest N tile of
// 256 / 128 / 64 that still gives every CTA at least two tiles (so that an
// epilogue can overlap the next tile's MMAs); smaller updates run one CTA per
// 128 x 64 tile with the C tile read during the mainloop.
int launch_tc_gemm_bf16(int64_t M, int64_t N, int64_t K, const void *A, int64_t lda, const void *B,
                        int64_t ldb, float *C, int64_t ldc, float alpha, cudaStream_t s, int *status)
{
    if (M <= 0 || N <= 0) return 0;
    if (K <= 0 || K % BK || lda % 8 || ldb % 8 || (reinterpret_cast<uintptr_t>(A) & 15) ||
        (reinterpret_cast<uintptr_t>(B) & 15))
        return GB_STATUS_CUDA_ERROR;
    if (M > 0x7fffffffLL || N > 0x7fffffffLL || K > 0x7fffffffLL) return GB_STATUS_CUDA_ERROR;
    const int64_t mt = (M + BM - 1) / BM;
    const int64_t sms = num_sms() > 0 ? num_sms() : 152;
    // fraction of the last round of tiles that is filled, over all rounds
    auto wave_eff = [&](int64_t tiles) { return double(tiles) / double((tiles + sms - 1) / sms * sms); };
    const int64_t t256 = mt * ((N + 255) / 256), t128 = mt * ((N + 127) / 128);
    // the 256-wide tile unless the 128-wide one fills the rounds markedly better
    if (t256 >= 2 * sms && !(wave_eff(t128) > wave_eff(t256) + 0.1))
        return launch_persistent<256>(M, N, K, A, lda, B, ldb, C, ldc, alpha, s, status);
    if (mt * ((N + 127) / 128) >= 2 * sms)
        return launch_persistent<128>(M, N, K, A, lda, B, ldb, C, ldc, alpha, s, status);
    if (mt * ((N + 63) / 64) >= 2 * sms)
        return launch_persistent<64>(M, N, K, A, lda, B, ldb, C, ldc, alpha, s, status);
    return launch_bn<64>(M, N, K, A, lda, B, ldb, C, ldc, alpha, s, status);
}

}  // namespace gb

extern "C" int gb_bf16_gemm_update(int64_t M, int64_t N, int64_t K, const void *A, int64_t lda, const void *B,
                                   int64_t ldb, float *C, int64_t ldc, float alpha, void *stream)
{
    if (M < 0) return -1;
    if (N < 0) return -2;
    if (K < 0 || K % 64) return -3;
    if (A == nullptr && M * N * K > 0) return -4;
    if (lda < (K > 8 ? K : 8) || lda % 8) return -5;
    if (B == nullptr && M * N * K > 0) return -6;
    if (ldb < (K > 8 ? K : 8) || ldb % 8) return -7;
    if (C == nullptr && M * N > 0) return -8;
    if (ldc < (M > 1 ? M : 1)) return -9;
    if (M == 0 || N == 0) return 0;
    if (K == 0) return 0;
    return gb::launch_tc_gemm_bf16(M, N, K, A, lda, B, ldb, C, ldc, alpha, static_cast<cudaStream_t>(stream),
                                   nullptr);
}

extern "C" int gb_device_status(int clear)
{
    int *p = gb::device_status_word();
    if (!p) return GB_STATUS_CUDA_ERROR;
    int v = 0;
    if (cudaMemcpy(&v, p, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return GB_STATUS_CUDA_ERROR;
    if (clear && v) cudaMemset(p, 0, sizeof(int));
    return v;
}

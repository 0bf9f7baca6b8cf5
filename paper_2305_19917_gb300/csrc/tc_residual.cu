// Split-precision residual update on the tensor cores (mixed-precision path):
//
//     R(i,j) -= sum_k Mv(i,k) Z(k,j)         for the lower-triangular Mv
//
// where both factors are given as fixed-point digit slices (BF16 holding
// small integers), the strictly lower part of Mv as
//     Mv(i,k) = 2^e_i * sum_{p=1..6} a_p(i,k) 2^(-8p),   |a_p| <= 128
// (the diagonal part R -= Mv(i,i) Z(i,j) is applied in FP64 where the
// correction digits are formed, outside this kernel), and
//     Z(k,j)  = 2^f_j * sum_{q=1..2} z_q(k,j) 2^(-8q),   |z_q| <= 128,
// and only the pairs with 8p + 8q <= budget are formed: slices p = 1..P with
// z_1, and p = 1..P2 also with z_2.  Each digit product is at most 2^14 and
// the K range is accumulated in chunks of at most 1024, so every tensor-core
// sum S_pq = sum_k a_p z_q of a chunk is an exact integer of at most 2^24 in
// the FP32 accumulator.  The epilogue converts S_pq to integers and adds
// S_pq 2^(W - 8p - 8q) into int64 sums T (W = the largest weight exponent
// formed, so |S_pq 2^(W-8p-8q)| <= 2^(24+W-16) <= 2^56; with K <= 16384 per
// launch, i.e. at most 16 chunks, |T| < 16 * 1.01 * 2^56 < 2^61) and stores
// T; a separate elementwise pass applies R -= 2^(e_i + f_j - W) T in FP64
// (the one rounding of the whole product is that of T to FP64).  The FP64
// pipe of an SM retires two operations per clock: done here, that work
// would idle the tensor cores of the SM for tens of microseconds per tile.
//
// One CTA per 128 x 128 tile of R, with no cluster: each CTA loads its own
// A slice tile (128 x 64 per stage) and both correction slices of its 128
// columns (two 128 x 64 tiles), so no load is shared between CTAs (L2 reads
// per CTA and K step: 16 KB of A plus 32 or 16 KB of Z).  Pass p multiplies
// slice a_p with [z_1; z_2] (256 x 64, z_2 only in passes p < P2) into one of
// two 128 x 256 TMEM accumulators, so that draining pass p overlaps the MMAs
// of pass p+1.  A pass of one slice with z_1 alone needs 32 KB of operands
// per 256 tensor-core clocks, more than the L2 delivers to an SM; so when
// P2 = P - 1 <= 2 (the pairs (P-1, 2) and (P, 1) have the same weight) the
// last two slices share one pass: per K step a_(P-1) [z_1; z_2] and a_P z_1, the
// latter added into the z_2 half of the accumulator.  The K step takes two
// ring entries, slice P-1 with both z tiles, then slice P with its own copy
// of z_1 (80 KB per 768 clocks): each entry is released when its own MMAs
// are done, so the ring keeps its lookahead (with z_1 read from the first
// entry only, both stayed held until the second was done, and the pass ran
// slower than the separate passes).  Two products in one accumulator need
// its K range halved to 512 to keep every sum within 2^24, so such a pass
// runs as two half-chunk passes.
// Warp 0: TMA, warp 1: TMEM + MMA issue, warps 2-9: epilogue
// (warp w drains TMEM lanes 32*(w%4).., column half (w-2)/4).  Tiles are
// rasterised in groups of 8 row tiles, longest K ranges (lowest rows) first.
#include "common.cuh"
#include "tc_common.cuh"

namespace gb {

int *device_status_word();

namespace {

constexpr int BM = 128, BNO = 128, BK = 64, STAGES = 4;
constexpr int kASlices = 6;                        // digit slices of Mv (8 bits each)
constexpr uint32_t A_BYTES = BM * BK * 2;          // one A slice tile
constexpr uint32_t ZS_BYTES = BNO * BK * 2;        // one Z slice tile (128 columns)
constexpr uint32_t B_BYTES = 2 * ZS_BYTES;         // z_1 and z_2 tiles
constexpr uint32_t STAGE_BYTES = A_BYTES + B_BYTES;
constexpr size_t SMEM_BYTES = 1024 + STAGES * size_t(STAGE_BYTES) + 256;
constexpr int NTHREADS = 320;
constexpr int kRasterGroup = 8;
// exactness needs K <= 1024 per tensor-memory accumulation of one product
// (1024 x 2^14 = 2^24), K <= 512 where two products share an accumulator
constexpr int KC = 1024;

// One pass of a K chunk: A slice p (0-based) times z_1 (and z_2 if nsl = 2)
// over K in [kb, ke); a merged pass also multiplies slice p + 1 with z_1.
struct Pass {
    int p, nsl, kb, ke;
    bool merged;
};

// Passes of the chunk [kc0, kc1): slices 0..P-1 one pass each, or with
// merging, slices 0..P-3 and then the merged pair P-2, P-1 over the chunk's
// two halves (one if the chunk is at most 512 long).
__device__ __forceinline__ int chunk_passes(int kc0, int kc1, int P, bool merge)
{
    return merge ? P - 1 + (kc1 - kc0 > KC / 2 ? 1 : 0) : P;
}
__device__ __forceinline__ Pass chunk_pass(int j, int kc0, int kc1, int P, int P2, bool merge)
{
    if (!merge || j < P - 2) return Pass{j, j < P2 ? 2 : 1, kc0, kc1, false};
    const int mid = min(kc0 + KC / 2, kc1);
    return j == P - 2 ? Pass{P - 2, 2, kc0, mid, true} : Pass{P - 2, 2, mid, kc1, true};
}

__global__ void __launch_bounds__(NTHREADS, 1)
tc_residual_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmZ,
                   long long *__restrict__ Tg, int64_t ldr, int k_lo, int k_hi, int P, int P2, int W, int nMt,
                   int nNt, int *status)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *sA = base;
    uint8_t *sB = base + STAGES * A_BYTES;
    uint64_t *full = reinterpret_cast<uint64_t *>(sB + STAGES * B_BYTES);
    uint64_t *empty = full + STAGES;
    uint64_t *accf = empty + STAGES;  // [2]
    uint64_t *acce = accf + 2;        // [2]
    uint32_t *tslot = reinterpret_cast<uint32_t *>(acce + 2);
    __shared__ int abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int gm, n_blk;
    tc::raster_grouped(int(blockIdx.x), nMt, nNt, kRasterGroup, gm, n_blk);
    // longest K ranges first: the lowest row tiles are rasterised first
    const int m_blk = nMt - 1 - gm;
    const int i0 = m_blk * BM, j0 = n_blk * BNO;
    const int k_end = min(k_hi, i0 + BM);  // this tile's K range is [k_lo, k_end)
    if (k_end <= k_lo) return;             // the tile lies entirely above the diagonal
    // the K range is cut into chunks of at most 1024, each pass of each
    // chunk drained separately into the same int64 sums
    const int nchunks = (k_end - k_lo + KC - 1) / KC;
    // merged only up to P = 3: at P = 5 (the first residual, K = 16384) the
    // merged pass gained no time and read 1.8x the DRAM bytes of the
    // separate passes (35 against 19 GB), at P = 3 it was 4 % faster with
    // the same DRAM bytes
    const bool merge = P >= 2 && P <= 3 && P2 == P - 1;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; s++) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);  // one MMA commit
        }
        for (int b = 0; b < 2; b++) {
            tc::mbar_init(&accf[b], 1);
            tc::mbar_init(&acce[b], 8);  // one arrival per epilogue warp
        }
        abort_flag = 0;
        tc::fence_barrier_init();
    }
    if (warp == 1) tc::tmem_alloc(tslot, 512);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tslot;
    volatile int *ab = &abort_flag;

    if (warp == 0) {
        if (lane == 0) {
            tc::tma_prefetch_desc(&tmA);
            tc::tma_prefetch_desc(&tmZ);
            int g = 0;
            bool ok = true;
            // one ring entry: slice p's A tile and the first nsl z tiles
            auto load = [&](int kk, int p, int nsl) {
                const int s = g % STAGES;
                const uint32_t ph = (g / STAGES) & 1;
                if (!tc::mbar_wait(&empty[s], ph ^ 1, ab, status, tc::TC_TIMEOUT_PRODUCER)) return false;
                tc::mbar_arrive_expect_tx(&full[s], A_BYTES + uint32_t(nsl) * ZS_BYTES);
                tc::tma_load_3d(&tmA, &full[s], sA + s * A_BYTES, kk, i0, p);
                for (int q = 0; q < nsl; q++)
                    tc::tma_load_3d(&tmZ, &full[s], sB + s * B_BYTES + q * ZS_BYTES, kk, j0, q);
                g++;
                return true;
            };
            for (int c = 0; c < nchunks && ok; c++) {
                const int kc0 = k_lo + c * KC, kc1 = min(kc0 + KC, k_end);
                const int nj = chunk_passes(kc0, kc1, P, merge);
                for (int j = 0; j < nj && ok; j++) {
                    const Pass ps = chunk_pass(j, kc0, kc1, P, P2, merge);
                    for (int kk = ps.kb; kk < ps.ke && ok; kk += BK) {
                        ok = load(kk, ps.p, ps.nsl);
                        if (ok && ps.merged) ok = load(kk, ps.p + 1, 1);
                    }
                }
            }
            // tail: wait until the MMAs released every stage, so that no
            // commit is still on its way to this CTA's barriers when it exits
            for (int t = 0; t < STAGES && ok; t++, g++) {
                const int s = g % STAGES;
                const uint32_t ph = (g / STAGES) & 1;
                if (!tc::mbar_wait(&empty[s], ph ^ 1, ab, status, tc::TC_TIMEOUT_PRODUCER)) break;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint64_t dA0 = tc::desc_kmajor_sw128(tc::smem_u32(sA)), dB0 = tc::desc_kmajor_sw128(tc::smem_u32(sB));
            const uint32_t idesc256 = tc::idesc_bf16_f32(BM, 256), idesc128 = tc::idesc_bf16_f32(BM, 128);
            int g = 0, cp = 0;
            bool ok = true;
            // ring entry g: wait until its copies landed, return its stage
            auto take = [&](int &s) {
                s = g % STAGES;
                const uint32_t ph = (g / STAGES) & 1;
                g++;
                if (!tc::mbar_wait(&full[s], ph, ab, status, tc::TC_TIMEOUT_MMA)) return false;
                tc::tc_fence_after();
                return true;
            };
            for (int c = 0; c < nchunks && ok; c++) {
                const int kc0 = k_lo + c * KC, kc1 = min(kc0 + KC, k_end);
                const int nj = chunk_passes(kc0, kc1, P, merge);
                for (int j = 0; j < nj && ok; j++, cp++) {
                    const Pass ps = chunk_pass(j, kc0, kc1, P, P2, merge);
                    const int nk = (ps.ke - ps.kb) / BK;
                    const int buf = cp & 1;
                    const uint32_t use = cp >> 1;
                    if (!tc::mbar_wait(&acce[buf], (use & 1) ^ 1, ab, status, tc::TC_TIMEOUT_MMA)) {
                        ok = false;
                        break;
                    }
                    tc::tc_fence_after();
                    // pair (p+1, 2) formed: one N = 256 MMA over [z_1; z_2]
                    const uint32_t idesc = ps.nsl == 2 ? idesc256 : idesc128;
                    const uint32_t d = tmem + uint32_t(buf * 256);
                    for (int kt = 0; kt < nk; kt++) {
                        int s;
                        if (!(ok = take(s))) break;
                        // the stage's descriptors from the ring's base ones: the start
                        // address field counts 16-byte units, so a 32-byte step along
                        // K adds 2 (few instructions per MMA: an N = 128 MMA takes
                        // 64 tensor-core clocks)
                        const uint64_t da = dA0 + uint64_t(uint32_t(s) * (A_BYTES >> 4));
                        const uint64_t db = dB0 + uint64_t(uint32_t(s) * (B_BYTES >> 4));
                        tc::mma_f16(d, da, db, idesc, kt != 0);
#pragma unroll
                        for (int kk = 1; kk < BK / 16; kk++)
                            tc::mma_f16(d, da + uint64_t(2 * kk), db + uint64_t(2 * kk), idesc, 1);
                        tc::mma_commit(&empty[s]);
                        if (ps.merged) {
                            // slice p+2 (1-based) times its own copy of z_1, added
                            // into the z_2 half (the same pair weight)
                            int s2;
                            if (!(ok = take(s2))) break;
                            const uint64_t da2 = dA0 + uint64_t(uint32_t(s2) * (A_BYTES >> 4));
                            const uint64_t db2 = dB0 + uint64_t(uint32_t(s2) * (B_BYTES >> 4));
#pragma unroll
                            for (int kk = 0; kk < BK / 16; kk++)
                                tc::mma_f16(d + 128u, da2 + uint64_t(2 * kk), db2 + uint64_t(2 * kk), idesc128, 1);
                            tc::mma_commit(&empty[s2]);
                        }
                    }
                    tc::mma_commit(&accf[buf]);
                }
            }
        }
    } else {
        const int q = warp & 3;                 // TMEM lane group this warp may read
        const int half = (warp - 2) >> 2;       // output columns [half*64, half*64+64)
        const int row = q * 32 + lane;
        long long T[64];
#pragma unroll
        for (int c = 0; c < 64; c++) T[c] = 0;
        bool ok = true;
        int cp = 0;
        for (int c = 0; c < nchunks && ok; c++) {
          const int kc0 = k_lo + c * KC, kc1 = min(kc0 + KC, k_end);
          const int nj = chunk_passes(kc0, kc1, P, merge);
          for (int jp = 0; jp < nj; jp++, cp++) {
            const Pass ps = chunk_pass(jp, kc0, kc1, P, P2, merge);
            const int p = ps.p;
            const int buf = cp & 1;
            const uint32_t use = cp >> 1;
            if (!tc::mbar_wait(&accf[buf], use & 1, ab, status, tc::TC_TIMEOUT_EPILOGUE)) {
                ok = false;
                break;
            }
            tc::tc_fence_after();
            // the z_2 half holds pair (p+1, 2), and in a merged pass also
            // (p+2, 1): both of weight 2^-(8p+24)
            const bool two = ps.nsl == 2;
            const int s1 = W - (8 * (p + 1) + 8);
            const int s2 = W - (8 * (p + 1) + 16);
            const uint32_t tbase = tmem + (uint32_t(q * 32) << 16) + uint32_t(buf * 256 + half * 64);
#pragma unroll
            for (int c0 = 0; c0 < 64; c0 += 16) {
                uint32_t r1[16];
                tc::tmem_ld16(tbase + c0, r1);
                tc::tmem_ld_wait();
#pragma unroll
                for (int j = 0; j < 16; j++)
                    T[c0 + j] += static_cast<long long>(__float2int_rn(__uint_as_float(r1[j]))) << s1;
                if (two) {
                    uint32_t r2[16];
                    tc::tmem_ld16(tbase + 128 + c0, r2);
                    tc::tmem_ld_wait();
#pragma unroll
                    for (int j = 0; j < 16; j++)
                        T[c0 + j] += static_cast<long long>(__float2int_rn(__uint_as_float(r2[j]))) << s2;
                }
            }
            tc::tc_fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&acce[buf]);
          }
        }
        if (ok) {
            // the exact sums of this tile: lanes hold consecutive rows, so
            // each store instruction writes 256 contiguous bytes
            const int64_t o = i0 + row + int64_t(j0 + half * 64) * ldr;
#pragma unroll
            for (int c = 0; c < 64; c++) Tg[o + int64_t(c) * ldr] = T[c];
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, 512);
    }
}

}  // namespace

// Exponent of the largest pair weight formed (pair (p, q) has weight
// 2^-(8p + 8q)): the int64 sums T carry it as 2^W.
int residual_weight(int P, int P2) { return (P2 > 0 && 8 * P2 + 16 > 8 * P + 8) ? 8 * P2 + 16 : 8 * P + 8; }

// T (kp x np, int64 column-major, ldr) = the exact digit sums of
// (strictly lower Mv) * Z over k in [k_lo, k_hi) for the row tiles the range
// reaches (rows >= k_lo), scaled by 2^(W - e_i - f_j) with W from
// residual_weight(P, P2); A slices (6 x kp x kp BF16 row-major, contiguous) and Z slices
// (2 x np x kp BF16: slice q holds column j of z_q at Zs + q*np*kp + j*kp).
// kp, np multiples of 128; k_lo, k_hi multiples of 64; k_hi - k_lo <= 16384;
// P A slices with z_1, the first P2 of them also with z_2.
int launch_tc_residual(long long *Tg, int64_t ldr, const void *As, const void *Zs, int64_t kp, int64_t np,
                       int64_t k_lo, int64_t k_hi, int P, int P2, cudaStream_t s, int *status)
{
    if (kp <= 0 || np <= 0 || k_hi <= k_lo) return 0;
    if (kp % 128 || np % 128 || k_lo % 64 || k_hi % 64 || k_hi - k_lo > 16384 || P < 1 || P > kASlices || P2 < 0 ||
        P2 > P)
        return GB_STATUS_CUDA_ERROR;
    const int W = residual_weight(P, P2);
    // |T| <= 16 chunks x 1.01 x 2^(24 + W - 16) must stay below 2^63
    if (W > 50) return GB_STATUS_CUDA_ERROR;
    if (kp > 0x7fffffffLL || np > 0x7fffffffLL) return GB_STATUS_CUDA_ERROR;
    CUtensorMap ta, tz;
    {
        uint64_t dims[3] = {uint64_t(kp), uint64_t(kp), uint64_t(kASlices)};
        uint64_t strides[2] = {uint64_t(kp) * 2, uint64_t(kp) * uint64_t(kp) * 2};
        uint32_t box[3] = {BK, BM, 1};
        GB_TRY(encode_tmap(&ta, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, As, dims, strides, box));
    }
    {
        uint64_t dims[3] = {uint64_t(kp), uint64_t(np), 2};
        uint64_t strides[2] = {uint64_t(kp) * 2, uint64_t(np) * uint64_t(kp) * 2};
        uint32_t box[3] = {BK, BNO, 1};  // 128 columns of one slice
        GB_TRY(encode_tmap(&tz, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, Zs, dims, strides, box));
    }
    static PerDeviceOnce attr;
    GB_TRY(smem_attr_once(attr, tc_residual_kernel, SMEM_BYTES));
    int *st = status ? status : device_status_word();
    if (!st) return GB_STATUS_CUDA_ERROR;
    // 1-D grid over (row tiles) x (column tiles)
    const int64_t nM = kp / BM, nN = np / BNO;
    if (nM > 65535 || nN > 65535 || nM * nN > 0x7fffffffLL) return GB_STATUS_CUDA_ERROR;
    dim3 grid((unsigned)(nM * nN));
    // algorithmic work: P passes (P2 of them two slices wide) over the lower
    // triangle of the K range
    double tri = 0;
    for (int64_t i0 = 0; i0 < kp; i0 += BM) {
        int64_t ke = i0 + BM < k_hi ? i0 + BM : k_hi;
        if (ke > k_lo) tri += double(ke - k_lo);
    }
    double flops = 0;
    for (int p = 0; p < P; p++) flops += 2.0 * BM * tri * np * (p < P2 ? 2 : 1);
    LaunchScope ls(KK_RESIDUAL, s, flops, 8.0 * kp * np);
    tc_residual_kernel<<<grid, NTHREADS, SMEM_BYTES, s>>>(ta, tz, Tg, ldr, (int)k_lo, (int)k_hi, P, P2, W,
                                                          (int)nM, (int)nN, st);
    return check(cudaGetLastError());
}

}  // namespace gb

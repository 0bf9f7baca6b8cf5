// Batched uneven triangular solves in one persistent launch: "n instances of
// TS" (Section IV, many right-hand sides) generalised to many independent
// problems of different order and width.
//
// Work units are (instance, chunk of CW right-hand sides); a chunk of an
// order-k instance costs ~k^2 CW / 2 multiply-adds, so units are sorted by
// k (largest first) and handed out through a device-side work queue: each
// CTA of a persistent grid pops a ticket with one atomicAdd until the queue
// is empty (no CTA ever waits on another).  A unit is solved entirely in
// shared memory by its CTA with the blocked forward model of Section V-C in
// left-looking order: for each 32-row diagonal block, one register-tiled
// update with all solved blocks (the gemm tasks), then the 32 x 32 triangle
// by warp-shuffle substitution (the TS task).  Backward problems are index
// reversed and right-side problems transposed on the way in and out.
// Instances of order above KMAX are solved by the regular driver.
//
// Tile shapes (the autotuner's choice, gb_batched_autotune): in the gemm
// tasks each thread owns RR rows x one 16-byte vector of right-hand sides
// (PER = 2 FP64 / 4 FP32 columns), so a unit is CW = 8 PER RR right-hand
// sides wide: RR = 1 gives 16 (FP64) / 32 (FP32) columns and two CTAs per
// SM (109 KB of shared memory each); RR = 2 gives 32 / 64 columns, twice the
// multiply-adds per shared-memory load, one CTA per SM.  A tiles are stored
// k-major so that a thread's RR rows load as one vector.  A warp owns a few
// whole columns of the block (its lanes the rows), so a step's A rows load
// as whole wavefronts and its X vector as a broadcast, and the warps whose
// columns lie past the last right-hand side of a chunk skip their products
// (a chunk is often narrower than CW: the last one of every instance).
//
// FP32 solves the 32 x 32 diagonal blocks with their inverses: a first kernel
// of the plan's graph inverts every diagonal block of every instance once per
// run (one warp per block, one lane per column of the inverse, forward
// substitution in registers), and the TS task of a unit becomes a product
// with the inverse on the gemm tasks' register tiles -- the warp-shuffle
// substitution, about four times the instructions of a gemm tile, dominated
// the FP32 kernel's issue slots.  FP64 keeps the substitution: its DFMA rate,
// not instruction issue, bounds it.
#include <algorithm>
#include <cstring>
#include <vector>
#include "common.cuh"

namespace gb {

namespace {

constexpr int KMAX = 512;   // largest order solved in shared memory
constexpr int NBB = 32;     // diagonal block
constexpr int NT = 256;     // threads per CTA
constexpr int LT = NBB + 2; // k-major A tile: row stride of one k (keeps 8- and 16-byte alignment)

// Tile shape of the gemm tasks: RR rows x PER columns per thread.
template <typename T, int RR>
struct BCfg {
    static constexpr int PER = int(16 / sizeof(T));   // one 16-byte vector of right-hand sides
    static constexpr int ROWG = NBB / RR;             // row groups of a block row
    static constexpr int COLG = NT / ROWG;            // column groups
    static constexpr int CW = COLG * PER;             // right-hand sides per unit
    static constexpr int LX = CW + PER;               // row stride of X in shared memory
    static_assert(ROWG * COLG == NT, "thread split");
    static_assert(CW % 8 == 0, "warp split of the TS task");
};

template <typename T>
struct Unit {
    const T *A;   // A of the instance
    T *B;         // B of the instance, offset to the chunk's first right-hand side
    const T *Linv;  // inverses of the instance's 32 x 32 diagonal blocks (FP32), k-major 32 x 32 each
    int64_t lda, ldb;
    int k;        // order of the triangle
    int cw;       // right-hand sides in this chunk (<= CW)
    int flags;    // bit0 mt, bit1 rev (backward), bit2 unit diag, bit3 left
    T alpha;
};


// A tiles in the ring (NBUF - 1 in flight): the tiles stream from L2, whose
// latency a short ring leaves exposed; FP32 tiles are half the size, so it
// keeps twice as many.
template <typename T>
constexpr int nbuf() { return sizeof(T) == 4 ? 8 : 4; }

// Asynchronous copy of one element (4 or 8 bytes); `in` false writes zero.
template <typename T>
__device__ __forceinline__ void cp_async_elem(T *dst, const T *src, bool in)
{
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
    const int n = in ? int(sizeof(T)) : 0;
    if (sizeof(T) == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(n) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Address of Mv'(i, j) of the forward view of unit u (index reversal for a
// backward problem, transposition for mt).
template <typename T>
__device__ __forceinline__ const T *mv_addr(const Unit<T> &u, int i, int j)
{
    const bool mt = u.flags & 1, rev = u.flags & 2;
    const int io = rev ? u.k - 1 - i : i, jo = rev ? u.k - 1 - j : j;
    return mt ? u.A + jo + int64_t(io) * u.lda : u.A + io + int64_t(jo) * u.lda;
}

// A unit's tiles in sequence: block row jb, then tiles ib = 0..jb (ib < jb:
// gemm tasks, ib == jb: the TS task); the position steps along the sequence.
struct TilePos {
    int jb = 0, ib = 0;
    __device__ __forceinline__ void next()
    {
        if (ib == jb) {
            jb++;
            ib = 0;
        } else {
            ib++;
        }
    }
};

// Issue the asynchronous loads of tile (jb, ib) into buffer Tb (reading
// along A's contiguous dimension): the gemm tiles in full, the TS tile on
// and below its diagonal; everything else (and the ragged edge) reads as
// zero.  Tb is k-major: Tb[kk * LT + rr] = Mv'(j0 + rr, i0 + kk).
template <typename T>
__device__ __forceinline__ void load_tile(const Unit<T> &u, int jb, int ib, T *Tb)
{
    if (u.Linv && ib == jb) {
        // the TS task's tile: the block's precomputed inverse (k-major 32 x
        // 32 in global memory), in 8-byte pieces into the LT-strided layout
        const T *src = u.Linv + size_t(jb) * NBB * NBB;
        constexpr int PIECE = int(8 / sizeof(T));
        for (int idx = threadIdx.x; idx < NBB * NBB / PIECE; idx += NT) {
            const int kk = (idx * PIECE) / NBB, rr = (idx * PIECE) % NBB;
            const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(Tb + kk * LT + rr));
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src + kk * NBB + rr) : "memory");
        }
        return;
    }
    const int j0 = jb * NBB, i0 = ib * NBB, k = u.k;
    const bool mt = u.flags & 1;
    if (ib < jb && j0 + NBB <= k) {
        // a gemm tile inside the triangle: entry (fast, slow) of the copy
        // sits at base + s fast + s lda slow (s = -1 for a backward problem),
        // fast running along A's contiguous dimension
        const bool rev = u.flags & 2;
        const int x0 = mt ? i0 : j0, y0 = mt ? j0 : i0;  // origin along the contiguous / strided index
        const int64_t sg = rev ? -1 : 1;
        const T *base = u.A + (rev ? int64_t(k - 1 - x0) + int64_t(k - 1 - y0) * u.lda : int64_t(x0) + int64_t(y0) * u.lda);
        const int fast = threadIdx.x % NBB;
        const T *p = base + sg * (fast + int64_t(threadIdx.x / NBB) * u.lda);
        const int64_t step = sg * int64_t(NT / NBB) * u.lda;
#pragma unroll
        for (int q = 0; q < NBB * NBB / NT; q++) {
            const int slow = threadIdx.x / NBB + q * (NT / NBB);
            const int rr = mt ? slow : fast, kk = mt ? fast : slow;
            cp_async_elem(Tb + kk * LT + rr, p + q * step, true);
        }
        return;
    }
    for (int idx = threadIdx.x; idx < NBB * NBB; idx += NT) {
        const int fast = idx % NBB, slow = idx / NBB;
        const int rr = mt ? slow : fast, kk = mt ? fast : slow;
        const bool in = j0 + rr < k && i0 + kk < k && (ib < jb || kk <= rr);
        cp_async_elem(Tb + kk * LT + rr, in ? mv_addr(u, j0 + rr, i0 + kk) : u.A, in);
    }
}

// RR rows of a k-major A tile as one vector.
template <typename T, int RR>
struct RowVec {
    T v[RR];
};
template <typename T, int RR>
__device__ __forceinline__ void load_rows(const T *p, T (&a)[RR])
{
    if constexpr (RR * sizeof(T) == 16) {
        const uint4 q = *reinterpret_cast<const uint4 *>(p);
        const T *x = reinterpret_cast<const T *>(&q);
#pragma unroll
        for (int e = 0; e < RR; e++) a[e] = x[e];
    } else if constexpr (RR * sizeof(T) == 8) {
        const uint2 q = *reinterpret_cast<const uint2 *>(p);
        const T *x = reinterpret_cast<const T *>(&q);
#pragma unroll
        for (int e = 0; e < RR; e++) a[e] = x[e];
    } else {
#pragma unroll
        for (int e = 0; e < RR; e++) a[e] = p[e];
    }
}

// acc += (rows r .. r + RR - 1 of the k-major tile Tb) x (32 rows of X from
// xr, columns cq ..), software-pipelined: the operands of step kk + 2 are
// loaded while step kk multiplies (two warps per scheduler leave the
// shared-memory latency exposed otherwise).
template <typename T, int RR, int PER, int LX>
__device__ __forceinline__ void tile_fma(T (&acc)[RR][PER], const T *Tb, const T *xr, int r, int cq)
{
    constexpr int D = 3;  // operand sets in registers (2 steps ahead)
    T a[D][RR], x[D][PER];
    auto load = [&](int kk, int b) {
        load_rows<T, RR>(Tb + kk * LT + r, a[b]);
        const uint4 xv = *reinterpret_cast<const uint4 *>(xr + kk * LX + cq);
        const T *xp = reinterpret_cast<const T *>(&xv);
#pragma unroll
        for (int e = 0; e < PER; e++) x[b][e] = xp[e];
    };
    load(0, 0);
    load(1, 1);
#pragma unroll
    for (int kk = 0; kk < NBB; kk++) {
        if (kk + 2 < NBB) load(kk + 2, (kk + 2) % D);
        const int b = kk % D;
#pragma unroll
        for (int q = 0; q < RR; q++)
#pragma unroll
            for (int e = 0; e < PER; e++) acc[q][e] += a[b][q] * x[b][e];
    }
}

// smem: Xs[KMAX][LX], NBUF k-major tiles Ts[NBB][LT], inverse diagonal.
template <typename T, int RR>
__global__ void __launch_bounds__(NT)
batched_kernel(const Unit<T> *__restrict__ units, int nunits, unsigned *__restrict__ ticket)
{
    using C = BCfg<T, RR>;
    constexpr int CW = C::CW, LX = C::LX, PER = C::PER;
    constexpr int TS = NBB * LT;
    constexpr int CPW = CW / 8;  // columns per warp in the TS task
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *Xs = reinterpret_cast<T *>(smem_raw);
    T *Ts = Xs + KMAX * LX;
    constexpr int NBUF = nbuf<T>();
    T *inv = Ts + NBUF * TS;
    __shared__ int cur;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    for (;;) {
        if (tid == 0) cur = int(atomicAdd(ticket, 1u));
        __syncthreads();
        const int t = cur;
        __syncthreads();
        if (t >= nunits) return;
        const Unit<T> u = units[t];
        const int k = u.k, cw = u.cw;
        const bool rev = u.flags & 2, unitd = u.flags & 4, left = u.flags & 8;
        const int nblk = (k + NBB - 1) / NBB;
        const int ntile = nblk * (nblk + 1) / 2;

        // ---- Xs = Bv' (forward view of the chunk; alpha is applied on the
        // way out), issued together with the first A tiles --------------------
        // rows k .. 32*nblk-1 are zero: the ragged last block multiplies them
        // by zero tile entries, and stale shared memory could hold a NaN
        const int kr = nblk * NBB;
        if (left) {
            // contiguous along i: warp w takes columns w, w + 8, ..., its lanes the rows
            for (int c = warp; c < CW; c += NT / 32) {
                const T *bc = u.B + int64_t(c) * u.ldb;
                for (int i = lane; i < kr; i += 32) {
                    const bool in = c < cw && i < k;
                    cp_async_elem(Xs + i * LX + c, in ? bc + (rev ? k - 1 - i : i) : u.B, in);
                }
            }
        } else {
            for (int idx = tid; idx < kr * CW; idx += NT) {  // contiguous along c (CW is a power of two)
                const int c = idx % CW, i = idx / CW;
                const int io = rev ? k - 1 - i : i;
                const bool in = c < cw && i < k;
                cp_async_elem(Xs + i * LX + c, in ? u.B + c + int64_t(io) * u.ldb : u.B, in);
            }
        }
        cp_async_commit();
        TilePos pf;  // the next tile to load
#pragma unroll 1
        for (int q = 0; q < NBUF - 1; q++) {
            if (q < ntile) {
                load_tile(u, pf.jb, pf.ib, Ts + q * TS);
                pf.next();
            }
            cp_async_commit();
        }

        // a warp owns PER * 32 / ROWG columns of every row of the block, so
        // its A rows load as whole wavefronts and its X vector as a
        // broadcast, and a warp past the chunk's last right-hand side skips
        // its products (the columns of X there stay zero)
        const int r = (tid % C::ROWG) * RR, cq = (tid / C::ROWG) * PER;
        const bool live = cq < cw;
        T acc[RR][PER];
#pragma unroll
        for (int a = 0; a < RR; a++)
#pragma unroll
            for (int e = 0; e < PER; e++) acc[a][e] = T(0);
        TilePos cur;  // tile tt
        for (int tt = 0; tt < ntile; tt++, cur.next()) {
            // wait until tile tt (and the B chunk) has landed; the barrier
            // also means every thread is done with tile tt - 1, whose buffer
            // then takes tile tt + NBUF - 1 (NBUF - 1 tiles stay in flight)
            cp_async_wait<NBUF - 2>();
            __syncthreads();
            if (tt + NBUF - 1 < ntile) {
                load_tile(u, pf.jb, pf.ib, Ts + ((tt + NBUF - 1) % NBUF) * TS);
                pf.next();
            }
            cp_async_commit();
            const T *Tb = Ts + (tt % NBUF) * TS;
            const int jb = cur.jb, ib = cur.ib;
            const int j0 = jb * NBB, nr = min(NBB, k - j0);
            if (ib < jb) {
                // gemm task: acc += Mv'(j, i) X_i
                if (live) tile_fma<T, RR, PER, LX>(acc, Tb, Xs + ib * NBB * LX, r, cq);
            } else if (u.Linv) {
                // X_j -= sum of the gemm tasks, then the TS task as the
                // product X_j = L_jj^-1 X_j on the register tiles
#pragma unroll
                for (int q = 0; q < RR; q++) {
                    if (r + q < nr) {
#pragma unroll
                        for (int e = 0; e < PER; e++) Xs[(j0 + r + q) * LX + cq + e] -= acc[q][e];
                    }
#pragma unroll
                    for (int e = 0; e < PER; e++) acc[q][e] = T(0);
                }
                __syncthreads();
                if (live) tile_fma<T, RR, PER, LX>(acc, Tb, Xs + j0 * LX, r, cq);
                __syncthreads();  // every thread has read X_j
#pragma unroll
                for (int q = 0; q < RR; q++) {
                    if (r + q < nr) {
#pragma unroll
                        for (int e = 0; e < PER; e++) Xs[(j0 + r + q) * LX + cq + e] = acc[q][e];
                    }
#pragma unroll
                    for (int e = 0; e < PER; e++) acc[q][e] = T(0);
                }
            } else {
                // X_j -= sum of the gemm tasks, then the TS task: the nr x nr
                // triangle by warp-shuffle substitution
#pragma unroll
                for (int q = 0; q < RR; q++) {
                    if (r + q < nr) {
#pragma unroll
                        for (int e = 0; e < PER; e++) Xs[(j0 + r + q) * LX + cq + e] -= acc[q][e];
                    }
#pragma unroll
                    for (int e = 0; e < PER; e++) acc[q][e] = T(0);
                }
                if (tid < NBB) inv[tid] = (tid < nr && !unitd) ? T(1) / Tb[tid * LT + tid] : T(1);
                __syncthreads();
                // warp w solves columns w, w+8, ... (CPW columns, interleaved for ILP)
                T tv[CPW];
#pragma unroll
                for (int e = 0; e < CPW; e++) tv[e] = (lane < nr) ? Xs[(j0 + lane) * LX + warp + 8 * e] : T(0);
                // columns past the chunk's last right-hand side stay zero
                for (int kk = 0; kk < (warp < cw ? nr : 0); kk++) {
                    const T d = inv[kk];
                    const T lk = Tb[kk * LT + lane];
#pragma unroll
                    for (int e = 0; e < CPW; e++) {
                        const T x = __shfl_sync(0xffffffffu, tv[e], kk) * d;
                        if (lane == kk) tv[e] = x;
                        else if (lane > kk) tv[e] -= lk * x;
                    }
                }
                if (lane < nr) {
#pragma unroll
                    for (int e = 0; e < CPW; e++) Xs[(j0 + lane) * LX + warp + 8 * e] = tv[e];
                }
            }
        }
        cp_async_wait<0>();
        __syncthreads();  // the last block's X (written by every thread) is complete

        // ---- write back alpha * X (undo reversal / transposition) -----------
        if (left) {
            for (int c = warp; c < cw; c += NT / 32) {
                T *bc = u.B + int64_t(c) * u.ldb;
                for (int i = lane; i < k; i += 32) bc[rev ? k - 1 - i : i] = u.alpha * Xs[i * LX + c];
            }
        } else {
            for (int idx = tid; idx < k * CW; idx += NT) {
                const int c = idx % CW, i = idx / CW;
                if (c < cw) u.B[c + int64_t(rev ? k - 1 - i : i) * u.ldb] = u.alpha * Xs[i * LX + c];
            }
        }
        __syncthreads();
    }
}

// Diagonal-block inverses of one instance per CTA (FP32): warp w inverts the
// forward-view blocks w, w + 8, ...: the lower triangle (unit diagonal when
// flagged) goes to shared memory, lane c solves L x = e_c by forward
// substitution in registers (x_r = 0 above the diagonal; rows past the
// instance's order are the identity) and writes column c of the inverse,
// k-major (Linv[c * 32 + r] = inverse(r, c)).
struct InvJob {
    const float *A;
    float *Linv;
    int64_t lda;
    int k;
    int flags;  // as Unit::flags (bit0 mt, bit1 rev, bit2 unit diagonal)
};

__global__ void __launch_bounds__(NT) batched_inv_kernel(const InvJob *__restrict__ jobs, int njobs)
{
    __shared__ float Ls[NT / 32][NBB][NBB + 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int jj = blockIdx.x; jj < njobs; jj += gridDim.x) {
        const InvJob J = jobs[jj];
        Unit<float> u{};
        u.A = J.A;
        u.lda = J.lda;
        u.k = J.k;
        u.flags = J.flags;
        const bool unitd = J.flags & 4;
        const bool mt = J.flags & 1;
        const int nblk = (J.k + NBB - 1) / NBB;
        for (int b = warp; b < nblk; b += NT / 32) {
            const int j0 = b * NBB, nr = min(NBB, J.k - j0);
            // the block's lower triangle, read along A's contiguous dimension
            for (int idx = lane; idx < NBB * NBB; idx += 32) {
                const int fast = idx % NBB, slow = idx / NBB;
                const int rr = mt ? slow : fast, cc = mt ? fast : slow;
                float v = 0.f;
                if (rr < nr && cc < nr && cc <= rr) v = *mv_addr(u, j0 + rr, j0 + cc);
                if (rr == cc && (unitd || rr >= nr)) v = 1.f;
                Ls[warp][rr][cc] = v;
            }
            __syncwarp();
            float x[NBB];
#pragma unroll
            for (int r = 0; r < NBB; r++) {
                float sum = (r == lane) ? 1.f : 0.f;
#pragma unroll
                for (int t = 0; t < r; t++) sum -= Ls[warp][r][t] * x[t];
                x[r] = (r < lane) ? 0.f : sum / Ls[warp][r][r];
            }
            float *dst = J.Linv + size_t(b) * NBB * NBB + size_t(lane) * NBB;
#pragma unroll
            for (int r = 0; r < NBB; r++) dst[r] = x[r];
            __syncwarp();
        }
    }
}

template <typename T, int RR>
constexpr size_t batched_smem()
{
    return sizeof(T) * (size_t(KMAX) * BCfg<T, RR>::LX + nbuf<T>() * NBB * LT + NBB);
}

}  // namespace

// ---- plan object ------------------------------------------------------------

struct BatchedPlan {
    int dtype = 0;                 // 0 FP64, 1 FP32
    int tile = 1;                  // rows per thread in the gemm tasks (1 or 2)
    int64_t nunits = 0;
    void *units = nullptr;         // device array of Unit<T>
    unsigned *ticket = nullptr;    // device work-queue counter
    int grid = 0;
    // instances too large for shared memory, solved by the regular driver
    struct Big {
        int side, uplo, trans, diag;
        int64_t m, n, lda, ldb;
        double alpha;
        const void *A;
        void *B;
    };
    std::vector<Big> big;
    cudaGraphExec_t exec = nullptr;
    uint64_t graph_kernels = 0;
    double flops = 0, bytes = 0;
    // FP32: inverses of every instance's diagonal blocks, recomputed each run
    std::vector<InvJob> jobs_h;
    InvJob *jobs = nullptr;
    float *linv = nullptr;
    size_t linv_elems = 0;
};

namespace {

template <typename T>
void build_units(BatchedPlan &P, int64_t count, const int8_t *side, const int8_t *uplo, const int8_t *trans,
                 const int8_t *diag, const int64_t *m, const int64_t *n, const T *alpha, const void *const *A,
                 const int64_t *lda, void *const *B, const int64_t *ldb, std::vector<Unit<T>> &units)
{
    const int CW = P.tile == 2 ? BCfg<T, 2>::CW : BCfg<T, 1>::CW;
    for (int64_t i = 0; i < count; i++) {
        if (m[i] == 0 || n[i] == 0) continue;
        const bool left = side[i] == GB_LEFT;
        const int64_t k = left ? m[i] : n[i];
        const int64_t ncols = left ? n[i] : m[i];
        P.flops += double(k) * double(k) * double(ncols);
        P.bytes += sizeof(T) * (double(k) * double(k) / 2 + 2.0 * double(k) * double(ncols));
        if (k > KMAX || alpha[i] == T(0)) {
            P.big.push_back({side[i], uplo[i], trans[i], diag[i], m[i], n[i], lda[i], ldb[i], double(alpha[i]), A[i],
                             B[i]});
            continue;
        }
        const bool mt = left ? (trans[i] == GB_TRANS) : (trans[i] == GB_NOTRANS);
        const bool fwd = (uplo[i] == GB_LOWER) != mt;
        const int flags = (mt ? 1 : 0) | (fwd ? 0 : 2) | (diag[i] == GB_UNIT ? 4 : 0) | (left ? 8 : 0);
        // FP32: the instance's block inverses at this element offset of the
        // plan's inverse buffer (kept as offset + 1, 0 meaning none, until
        // the pointer is filled in on upload)
        size_t linv_off = 0;
        if (sizeof(T) == 4) {
            linv_off = P.linv_elems + 1;
            P.linv_elems += size_t((k + NBB - 1) / NBB) * NBB * NBB;
            InvJob j;
            j.A = reinterpret_cast<const float *>(A[i]);
            j.Linv = reinterpret_cast<float *>(linv_off);
            j.lda = lda[i];
            j.k = int(k);
            j.flags = flags;
            P.jobs_h.push_back(j);
        }
        for (int64_t c0 = 0; c0 < ncols; c0 += CW) {
            Unit<T> u;
            u.A = static_cast<const T *>(A[i]);
            T *b = static_cast<T *>(B[i]);
            u.B = left ? b + c0 * ldb[i] : b + c0;
            u.Linv = sizeof(T) == 4 ? reinterpret_cast<const T *>(linv_off) : nullptr;
            u.lda = lda[i];
            u.ldb = ldb[i];
            u.k = int(k);
            u.cw = int(std::min<int64_t>(CW, ncols - c0));
            u.flags = flags;
            u.alpha = alpha[i];
            units.push_back(u);
        }
    }
    // largest first (longest-processing-time order for the work queue)
    std::stable_sort(units.begin(), units.end(),
                     [](const Unit<T> &a, const Unit<T> &b) { return a.k * a.cw > b.k * b.cw; });
}

template <typename T, int RR>
int upload_and_capture(BatchedPlan &P, std::vector<Unit<T>> &units, cudaStream_t s)
{
    P.nunits = int64_t(units.size());
    const size_t ub = units.size() * sizeof(Unit<T>);
    GB_CUDA(cudaMalloc(&P.units, ub > 0 ? ub : sizeof(Unit<T>)));
    GB_CUDA(cudaMalloc(&P.ticket, sizeof(unsigned)));
    if (!P.jobs_h.empty()) {
        GB_CUDA(cudaMalloc(&P.linv, P.linv_elems * sizeof(float)));
        GB_CUDA(cudaMalloc(&P.jobs, P.jobs_h.size() * sizeof(InvJob)));
        for (auto &j : P.jobs_h) j.Linv = P.linv + (reinterpret_cast<size_t>(j.Linv) - 1);
        for (auto &u : units)
            if (u.Linv) u.Linv = reinterpret_cast<const T *>(P.linv) + (reinterpret_cast<size_t>(u.Linv) - 1);
        GB_CUDA(cudaMemcpyAsync(P.jobs, P.jobs_h.data(), P.jobs_h.size() * sizeof(InvJob), cudaMemcpyHostToDevice,
                                s));
    }
    if (ub) GB_CUDA(cudaMemcpyAsync(P.units, units.data(), ub, cudaMemcpyHostToDevice, s));
    GB_CUDA(cudaStreamSynchronize(s));
    static PerDeviceOnce attr;
    GB_TRY(smem_attr_once(attr, batched_kernel<T, RR>, batched_smem<T, RR>()));
    int dev = 0, sms = 0, per_sm = 0;
    GB_CUDA(cudaGetDevice(&dev));
    GB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    GB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_kernel<T, RR>, NT, batched_smem<T, RR>()));
    if (per_sm < 1) per_sm = 1;
    int64_t g = int64_t(sms) * per_sm;
    if (g > P.nunits) g = P.nunits;
    P.grid = int(g);
    if (P.nunits == 0) return 0;
    // CUDA graph: [reset the queue counter, persistent kernel]
    cudaStream_t cs;
    GB_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    const uint64_t before = capture_count();
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaMemsetAsync(P.ticket, 0, sizeof(unsigned), cs);
        if (!P.jobs_h.empty()) {
            const int64_t nj = int64_t(P.jobs_h.size());
            const int64_t gi = nj < int64_t(sms) * 8 ? nj : int64_t(sms) * 8;
            LaunchScope ls(KK_BATCHED, cs, 0.0, 4.0 * double(P.linv_elems));
            batched_inv_kernel<<<(unsigned)gi, NT, 0, cs>>>(P.jobs, int(nj));
        }
        {
            LaunchScope ls(KK_BATCHED, cs, P.flops, P.bytes);
            batched_kernel<T, RR><<<P.grid, NT, batched_smem<T, RR>(), cs>>>(
                static_cast<const Unit<T> *>(P.units), int(P.nunits), P.ticket);
        }
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(cs, &graph);
        if (e == cudaSuccess) {
            e = cudaGraphInstantiate(&P.exec, graph, 0);
            cudaGraphDestroy(graph);
        }
    }
    P.graph_kernels = capture_count() - before;
    cudaStreamDestroy(cs);
    return check(e);
}

}  // namespace

int batched_run(BatchedPlan &P, cudaStream_t s)
{
    if (P.nunits > 0) {
        LaunchScope ls(KK_BATCHED, s, P.flops, P.bytes, P.graph_kernels);
        GB_CUDA(cudaGraphLaunch(P.exec, s));
    }
    for (auto &b : P.big) {
        int st;
        if (P.dtype == 0)
            st = gb_dtrsm(b.side, b.uplo, b.trans, b.diag, b.m, b.n, b.alpha, static_cast<const double *>(b.A), b.lda,
                          static_cast<double *>(b.B), b.ldb, s);
        else
            st = gb_strsm(b.side, b.uplo, b.trans, b.diag, b.m, b.n, float(b.alpha), static_cast<const float *>(b.A),
                          b.lda, static_cast<float *>(b.B), b.ldb, s);
        if (st) return st;
    }
    return 0;
}

void batched_free(BatchedPlan *P)
{
    if (!P) return;
    if (P->exec) cudaGraphExecDestroy(P->exec);
    if (P->units) cudaFree(P->units);
    if (P->ticket) cudaFree(P->ticket);
    if (P->jobs) cudaFree(P->jobs);
    if (P->linv) cudaFree(P->linv);
    delete P;
}

int batched_create(int dtype, int64_t count, const int8_t *side, const int8_t *uplo, const int8_t *trans,
                   const int8_t *diag, const int64_t *m, const int64_t *n, const void *alpha, const void *const *A,
                   const int64_t *lda, void *const *B, const int64_t *ldb, cudaStream_t s, int tile, BatchedPlan **out)
{
    // argument checks (1-based argument numbers of gb_trsm_batched)
    if (dtype != 0 && dtype != 1) return -1;
    if (count < 0) return -2;
    if (count > 0) {
        const void *arrays[11] = {side, uplo, trans, diag, m, n, alpha, A, lda, B, ldb};
        for (int a = 0; a < 11; a++)
            if (!arrays[a]) return -(3 + a);
    }
    for (int64_t i = 0; i < count; i++) {
        if (side[i] != GB_LEFT && side[i] != GB_RIGHT) return -3;
        if (uplo[i] != GB_LOWER && uplo[i] != GB_UPPER) return -4;
        if (trans[i] != GB_NOTRANS && trans[i] != GB_TRANS) return -5;
        if (diag[i] != GB_NONUNIT && diag[i] != GB_UNIT) return -6;
        if (m[i] < 0) return -7;
        if (n[i] < 0) return -8;
        const int64_t k = side[i] == GB_LEFT ? m[i] : n[i];
        const bool empty = m[i] == 0 || n[i] == 0;
        const double a = dtype == 0 ? static_cast<const double *>(alpha)[i] : static_cast<const float *>(alpha)[i];
        if (!empty && A[i] == nullptr && a != 0.0) return -10;
        if (lda[i] < (k > 1 ? k : 1)) return -11;
        if (!empty && B[i] == nullptr) return -12;
        if (ldb[i] < (m[i] > 1 ? m[i] : 1)) return -13;
    }
    BatchedPlan *P = new BatchedPlan;
    P->dtype = dtype;
    P->tile = tile;
    int st;
    if (dtype == 0) {
        std::vector<Unit<double>> units;
        build_units<double>(*P, count, side, uplo, trans, diag, m, n, static_cast<const double *>(alpha), A, lda, B,
                            ldb, units);
        st = tile == 2 ? upload_and_capture<double, 2>(*P, units, s) : upload_and_capture<double, 1>(*P, units, s);
    } else {
        std::vector<Unit<float>> units;
        build_units<float>(*P, count, side, uplo, trans, diag, m, n, static_cast<const float *>(alpha), A, lda, B,
                           ldb, units);
        st = tile == 2 ? upload_and_capture<float, 2>(*P, units, s) : upload_and_capture<float, 1>(*P, units, s);
    }
    if (st) {
        batched_free(P);
        return st;
    }
    *out = P;
    return 0;
}

}  // namespace gb

extern "C" {

int gb_batched_plan_create_tiled(int dtype, int64_t count, const int8_t *side, const int8_t *uplo,
                                 const int8_t *trans, const int8_t *diag, const int64_t *m, const int64_t *n,
                                 const void *alpha, const void *const *A, const int64_t *lda, void *const *B,
                                 const int64_t *ldb, int tile, void *stream, void **plan_out)
{
    if (!plan_out) return -17;
    *plan_out = nullptr;
    if (tile == 0) tile = 1;
    if (tile != 1 && tile != 2) return -15;
    gb::BatchedPlan *P = nullptr;
    int st = gb::batched_create(dtype, count, side, uplo, trans, diag, m, n, alpha, A, lda, B, ldb,
                                static_cast<cudaStream_t>(stream), tile, &P);
    if (st) return st;
    *plan_out = P;
    return 0;
}

int gb_batched_plan_create(int dtype, int64_t count, const int8_t *side, const int8_t *uplo, const int8_t *trans,
                           const int8_t *diag, const int64_t *m, const int64_t *n, const void *alpha,
                           const void *const *A, const int64_t *lda, void *const *B, const int64_t *ldb,
                           void *stream, void **plan_out)
{
    if (!plan_out) return -15;
    const int st = gb_batched_plan_create_tiled(dtype, count, side, uplo, trans, diag, m, n, alpha, A, lda, B, ldb,
                                                1, stream, plan_out);
    return st == -17 ? -15 : st;
}

int gb_batched_autotune(int dtype, int64_t count, const int8_t *side, const int8_t *uplo, const int8_t *trans,
                        const int8_t *diag, const int64_t *m, const int64_t *n, const void *alpha,
                        const void *const *A, const int64_t *lda, void *const *B, const int64_t *ldb, int reps,
                        void *stream, int *tile_out, double *ms_out)
{
    if (!tile_out) return -16;
    if (reps < 1 || reps > 100) return -14;
    *tile_out = 1;
    if (ms_out) ms_out[0] = ms_out[1] = 0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the solves overwrite B: keep a device copy of every B and restore it
    // before each run and at the end
    const size_t esz = dtype == 0 ? 8 : 4;
    std::vector<size_t> off(count > 0 ? size_t(count) : 1, 0);
    size_t total = 0;
    for (int64_t i = 0; i < count; i++) {
        off[i] = total;
        if (m && n && m[i] > 0 && n[i] > 0) total += size_t(m[i]) * size_t(n[i]) * esz;
    }
    void *save = nullptr;
    if (total) GB_CUDA(cudaMallocAsync(&save, total, s));
    auto copy_all = [&](bool restore) {
        for (int64_t i = 0; i < count; i++) {
            if (m[i] <= 0 || n[i] <= 0) continue;
            char *sv = static_cast<char *>(save) + off[i];
            const cudaError_t e =
                restore ? cudaMemcpy2DAsync(B[i], esz * ldb[i], sv, esz * m[i], esz * m[i], n[i], cudaMemcpyDeviceToDevice, s)
                        : cudaMemcpy2DAsync(sv, esz * m[i], B[i], esz * ldb[i], esz * m[i], n[i], cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) return gb::check(e);
        }
        return 0;
    };
    int st = 0;
    double best = 1e300;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (!st) st = gb::check(cudaEventCreate(&e0));
    if (!st) st = gb::check(cudaEventCreate(&e1));
    if (!st && total) st = copy_all(false);
    for (int tile = 1; tile <= 2 && !st; tile++) {
        void *plan = nullptr;
        st = gb_batched_plan_create_tiled(dtype, count, side, uplo, trans, diag, m, n, alpha, A, lda, B, ldb, tile,
                                          stream, &plan);
        if (st) break;
        std::vector<float> t(reps);
        for (int r = 0; r <= reps && !st; r++) {  // run 0 is a warm-up
            if (total) st = copy_all(true);
            if (st) break;
            cudaEventRecord(e0, s);
            st = gb_batched_plan_run(plan, stream);
            cudaEventRecord(e1, s);
            if (!st) st = gb::check(cudaEventSynchronize(e1));
            if (!st && r > 0) st = gb::check(cudaEventElapsedTime(&t[r - 1], e0, e1));
        }
        gb_batched_plan_destroy(plan);
        if (st) break;
        std::sort(t.begin(), t.end());
        const double ms = t[reps / 2];
        if (ms_out) ms_out[tile - 1] = ms;
        if (ms < best) {
            best = ms;
            *tile_out = tile;
        }
    }
    if (total && save) {
        const int c = copy_all(true);
        if (!st) st = c;
        cudaFreeAsync(save, s);
    }
    const int c = gb::check(cudaStreamSynchronize(s));
    if (!st) st = c;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return st;
}

int gb_batched_plan_tile(const void *plan)
{
    if (!plan) return -1;
    return static_cast<const gb::BatchedPlan *>(plan)->tile;
}

int gb_batched_plan_run(void *plan, void *stream)
{
    if (!plan) return -1;
    return gb::batched_run(*static_cast<gb::BatchedPlan *>(plan), static_cast<cudaStream_t>(stream));
}

int gb_batched_plan_destroy(void *plan)
{
    gb::batched_free(static_cast<gb::BatchedPlan *>(plan));
    return 0;
}

int gb_batched_plan_info(const void *plan, int64_t *units, int *grid, int64_t *large_instances, double *flops)
{
    if (!plan) return -1;
    const gb::BatchedPlan *P = static_cast<const gb::BatchedPlan *>(plan);
    if (units) *units = P->nunits;
    if (grid) *grid = P->grid;
    if (large_instances) *large_instances = int64_t(P->big.size());
    if (flops) *flops = P->flops;
    return 0;
}

int gb_trsm_batched(int dtype, int64_t count, const int8_t *side, const int8_t *uplo, const int8_t *trans,
                    const int8_t *diag, const int64_t *m, const int64_t *n, const void *alpha, const void *const *A,
                    const int64_t *lda, void *const *B, const int64_t *ldb, void *stream)
{
    void *plan = nullptr;
    int st = gb_batched_plan_create(dtype, count, side, uplo, trans, diag, m, n, alpha, A, lda, B, ldb, stream, &plan);
    if (st) return st;
    st = gb_batched_plan_run(plan, stream);
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    gb_batched_plan_destroy(plan);
    if (st) return st;
    return gb::check(e);
}

}  // extern "C"

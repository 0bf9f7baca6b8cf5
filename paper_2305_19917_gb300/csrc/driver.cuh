// Decomposition drivers: the paper's three computation models (Section V),
// written once over an "executor" so that the same schedule either launches
// kernels or is counted on the host (gb_plan_counts).
//
// All drivers work on rows [r0, r1) of the canonical view Mv * Xv = alpha*Bv
// (see common.cuh).  Two task kinds are issued:
//   e.ts(b0, nr, a)              TS task: solve the diagonal block
//                                Mv[b0:b0+nr, b0:b0+nr] X = a * Bv[b0:b0+nr]
//   e.gemm(ci0, M, ak0, K, a)    gemm task: Bv[ci0:ci0+M] = a*Bv[ci0:ci0+M]
//                                - Mv[ci0:ci0+M, ak0:ak0+K] * Bv[ak0:ak0+K]
// alpha is applied at the first touch of each row of Bv.  Forward
// substitution (Mv lower) visits blocks top-down; backward (Mv upper) is the
// exact mirror image (blocks aligned at the bottom, visited bottom-up).
#pragma once
#include <stdint.h>

namespace gb {

// Split point of the recursive model.  The paper halves a power-of-two order
// (Section IV; Section V-A, r(i) = 2^i); for other orders the first part is
// rounded up to a multiple of nb: m1 = nb * ceil(ceil(n/2) / nb), clamped to
// [nb, n-1].
inline int64_t rec_split(int64_t n, int64_t nb)
{
    int64_t half = (n + 1) / 2;
    int64_t m1 = ((half + nb - 1) / nb) * nb;
    if (m1 < nb) m1 = nb;
    if (m1 > n - 1) m1 = n - 1;
    return m1;
}

// Blocked model (Section V-C): r = ceil(n/nb) diagonal blocks; after block j
// is solved, one GEMM updates every block below it (right-looking), i.e. the
// r(r-1)/2 off-diagonal blocks are issued as r-1 launches.
template <class E, typename T>
void drive_blocked(E &e, int64_t r0, int64_t r1, int64_t nb, T alpha, bool fwd)
{
    int64_t n = r1 - r0;
    if (n <= 0) return;
    int64_t r = (n + nb - 1) / nb;
    for (int64_t j = 0; j < r && e.ok(); j++) {
        T a = j == 0 ? alpha : T(1);
        if (fwd) {
            int64_t b0 = r0 + j * nb, b1 = b0 + nb < r1 ? b0 + nb : r1;
            e.ts(b0, b1 - b0, a);
            if (b1 < r1) e.gemm(b1, r1 - b1, b0, b1 - b0, a);
        } else {
            int64_t b1 = r1 - j * nb, b0 = b1 - nb > r0 ? b1 - nb : r0;
            e.ts(b0, b1 - b0, a);
            if (b0 > r0) e.gemm(r0, b0 - r0, b0, b1 - b0, a);
        }
    }
}

// Recursive model (Section V-A): split, solve the first part, one GEMM
// B2 = alpha*B2 - A21*X1, solve the second part; `depth` levels (refinement
// level 2^depth), leaves of order <= nb or at depth 0 are TS tasks.
template <class E, typename T>
void drive_recursive(E &e, int64_t r0, int64_t r1, int depth, int64_t nb, T alpha, bool fwd)
{
    int64_t n = r1 - r0;
    if (n <= 0 || !e.ok()) return;
    if (depth <= 0 || n <= nb) {
        e.ts(r0, n, alpha);
        return;
    }
    int64_t m1 = rec_split(n, nb);
    if (fwd) {
        int64_t s = r0 + m1;
        drive_recursive(e, r0, s, depth - 1, nb, alpha, fwd);
        e.gemm(s, r1 - s, r0, m1, alpha);
        drive_recursive(e, s, r1, depth - 1, nb, T(1), fwd);
    } else {
        int64_t s = r1 - m1;
        drive_recursive(e, s, r1, depth - 1, nb, alpha, fwd);
        e.gemm(r0, s - r0, s, m1, alpha);
        drive_recursive(e, r0, s, depth - 1, nb, T(1), fwd);
    }
}

// Iterative model (Section V-B): fixed TS granularity nb; before block row j
// is solved, one GEMM applies all solved blocks 0..j-1 to it (left-looking),
// i.e. gemm(i, j) for j = 0..r-2 plus r TS tasks.
template <class E, typename T>
void drive_iterative(E &e, int64_t r0, int64_t r1, int64_t nb, T alpha, bool fwd)
{
    int64_t n = r1 - r0;
    if (n <= 0) return;
    int64_t r = (n + nb - 1) / nb;
    for (int64_t j = 0; j < r && e.ok(); j++) {
        if (fwd) {
            int64_t b0 = r0 + j * nb, b1 = b0 + nb < r1 ? b0 + nb : r1;
            if (j > 0) e.gemm(b0, b1 - b0, r0, b0 - r0, alpha);
            e.ts(b0, b1 - b0, j == 0 ? alpha : T(1));
        } else {
            int64_t b1 = r1 - j * nb, b0 = b1 - nb > r0 ? b1 - nb : r0;
            if (j > 0) e.gemm(b0, b1 - b0, b1, r1 - b1, alpha);
            e.ts(b0, b1 - b0, j == 0 ? alpha : T(1));
        }
    }
}

template <class E, typename T>
void drive_plan(E &e, int driver, int64_t k, int64_t nb, int depth, T alpha, bool fwd)
{
    if (driver == GB_DRIVER_BLOCKED) drive_blocked(e, 0, k, nb, alpha, fwd);
    else if (driver == GB_DRIVER_RECURSIVE) drive_recursive(e, 0, k, depth, nb, alpha, fwd);
    else drive_iterative(e, 0, k, nb, alpha, fwd);
}

}  // namespace gb

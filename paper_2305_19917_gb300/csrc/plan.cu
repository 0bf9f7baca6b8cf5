// Planner: picks driver, nb and recursion depth for a shape.
#include "plan.cuh"

namespace gb {

// Built-in default: recursive halving down to leaves of about 512 rows
// (large-K GEMM updates), leaves blocked with nb = 64.
static gb_plan default_plan(int dtype, int64_t k)
{
    (void)dtype;
    gb_plan p;
    p.reserved = 0;
    p.nb = 64;
    if (k <= 512) {
        p.driver = GB_DRIVER_BLOCKED;
        p.depth = 0;
        return p;
    }
    int d = 0;
    while ((k >> (d + 1)) >= 512 && d < 8) d++;
    p.driver = GB_DRIVER_RECURSIVE;
    p.depth = d;
    return p;
}

gb_plan choose_plan(int dtype, int side, int uplo, int trans, int64_t m, int64_t n)
{
    (void)uplo;
    (void)trans;
    int64_t k = side == GB_LEFT ? m : n;
    return default_plan(dtype, k);
}

}  // namespace gb

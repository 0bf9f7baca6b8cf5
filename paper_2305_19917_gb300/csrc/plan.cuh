// Plan validation and choice (internal header).
#pragma once
#include "../../include/gbtrsm.h"

namespace gb {

enum { GB_DTYPE_F64 = 0, GB_DTYPE_F32 = 1, GB_DTYPE_BF16_MIXED = 2, GB_DTYPE_FP8_MIXED = 3 };

inline bool plan_valid(const gb_plan &p)
{
    if (p.reserved != 0) return false;
    if (p.driver == GB_DRIVER_AUTO) return true;
    if (p.driver != GB_DRIVER_BLOCKED && p.driver != GB_DRIVER_RECURSIVE &&
        p.driver != GB_DRIVER_ITERATIVE)
        return false;
    switch (p.nb) {
    case 16: case 32: case 64: case 128: case 256: case 512: break;
    default: return false;
    }
    if (p.depth < 0 || p.depth > 12) return false;
    return true;
}

// Planner: the loaded cost model's argmin if one is loaded, else the
// built-in default (defined in plan.cu).
gb_plan choose_plan(int dtype, int side, int uplo, int trans, int64_t m, int64_t n);
int plan_candidates(int dtype, gb_plan *out, int cap);
void plan_features(int dtype, int side, int uplo, int trans, int64_t m, int64_t n, const gb_plan &p, float *f);

}  // namespace gb

// Diagonal-block solve kernels instantiated for float (see diag_kernel.cuh).
#include "diag_kernel.cuh"

namespace gb {
template int launch_diag_solve<float>(const Canon<float> &, int64_t, int, float);
}  // namespace gb

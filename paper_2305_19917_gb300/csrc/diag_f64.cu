// Diagonal-block solve kernels instantiated for double (see diag_kernel.cuh).
#include "diag_kernel.cuh"

namespace gb {
template int launch_diag_solve<double>(const Canon<double> &, int64_t, int, double);
}  // namespace gb

// SpMV kernel variants with f64 values (see launch.cuh).
#include "launch.cuh"

namespace spmv {
SPMV_DEFINE_RUNNER(run_kernels_f64, SPMV_F64)
}  // namespace spmv

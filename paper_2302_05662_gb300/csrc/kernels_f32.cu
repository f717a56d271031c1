// SpMV kernel variants with f32 values (see launch.cuh).
#include "launch.cuh"

namespace spmv {
SPMV_DEFINE_RUNNER(run_kernels_f32, SPMV_F32)
}  // namespace spmv

// SpMV kernel variants with bf16 values (see launch.cuh).
#include "launch.cuh"

namespace spmv {
SPMV_DEFINE_RUNNER(run_kernels_bf16, SPMV_BF16)
}  // namespace spmv

/*
 * spmv_probe.h -- measurement kernels of the GB300 SpMV engine.
 *
 * These are not part of the product y <- alpha A x + beta y and the paper
 * (Auto-SpMV, arXiv 2302.05662) has no counterpart: they give the benchmark
 * two ceilings against which an SpMV kernel's time is judged besides the
 * HBM copy bandwidth.
 *
 *   - The gather floor: a kernel that moves the same bytes as the product
 *     (column indices, values, row pointers, x gathered at every column
 *     index, y written) with ideal streaming access and no floating-point
 *     instruction.  A kernel near this floor is held by the gathers of x
 *     (random 4- or 8-byte reads from an L2-resident vector), not by its own
 *     code.
 *   - The fp64 fused-multiply-add ceiling: GB300 issues fp64 arithmetic at
 *     a small fraction of its fp32 rate, so an fp64 SpMV (one fused
 *     multiply-add per nonzero) can be held by the fp64 pipe rather than by
 *     HBM.  This kernel runs independent fp64 FMA chains on every SM.
 *
 * Conventions as in spmv.h (status codes, spmv_last_error, stream as void*).
 */
#ifndef SPMV_GB300_SPMV_PROBE_H
#define SPMV_GB300_SPMV_PROBE_H

#include <stdint.h>

#include "spmv.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Gather floor of the handle's matrix: one launch on `stream` that streams
 * the handle's CSR column indices and values in order (16-byte vector loads,
 * consecutive nonzeros per thread), gathers d_x at every column index,
 * streams the m + 1 row pointers and writes m entries of d_y.  The bits of
 * every value and gathered x entry are combined with integer operations only,
 * and the bytes written to d_y are meaningless (the result is not a product).
 * d_x: device, n entries; d_y: device, m entries (double for SPMV_F64
 * handles, float otherwise); both caller-owned.
 * Errors: SPMV_ERR_INVALID (NULL handle or vector), SPMV_ERR_UNSUPPORTED (a
 * handle held in row panels), SPMV_ERR_CUDA.  Never synchronises.
 */
SPMV_API int spmv_probe_gather_floor(spmv_handle h, const void *d_x, void *d_y,
                                     void *stream);

/*
 * fp64 FMA ceiling: one launch on `stream` of a full wave of thread blocks
 * (every SM at its resident limit), each thread running 8 independent chains
 * of `iterations` fp64 fused multiply-adds.  *h_fma_count (host) receives
 * the number of fused multiply-adds performed (each is 2 flops).  d_sink:
 * device, one double, written only when the chains reach an impossible
 * value, so the arithmetic cannot be removed by the compiler.
 * Errors: SPMV_ERR_INVALID (iterations < 1, NULL pointers), SPMV_ERR_CUDA.
 * Never synchronises.
 */
SPMV_API int spmv_probe_fp64_fma(int64_t iterations, double *d_sink,
                                 int64_t *h_fma_count, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* SPMV_GB300_SPMV_PROBE_H */

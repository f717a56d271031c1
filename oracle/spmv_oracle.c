/*
 * CPU oracle for sparse matrix-vector multiplication (test infrastructure).
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * use this file; the CUDA library never includes, links or calls it.
 *
 * The operation is the SpMV of Section 2.2 of the paper, Y = A * X for a
 * sparse A and dense X, extended with the BLAS scalars:
 *     y_out[i] = alpha * sum_{k : rows[k] == i} vals[k] * x[cols[k]]
 *                + beta * y_in[i]
 * taken straight from COO triplets (the format the inputs arrive in,
 * Section 7.5), with no conversion to any storage format.
 *
 * Readings where the paper is silent:
 *   - duplicate (row, col) triplets are summed (each triplet contributes its
 *     own product);
 *   - beta == 0 means y_in is not read (NaN/Inf in y_in do not propagate);
 *   - the per-row sums use Kahan-compensated fp64 accumulation in triplet
 *     order, so the oracle is close to exactly rounded.
 *
 * Everything is fp64.  Build with -ffp-contract=off so the compensated sum
 * and every product round the same way on every host.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Returns 0 on success, -1 on an out-of-range triplet, -2 on allocation
 * failure.  y_in may be NULL when beta == 0.  y_out has m entries. */
int oracle_spmv_coo_f64(int64_t m, int64_t n, int64_t nnz,
                        const int32_t *rows, const int32_t *cols,
                        const double *vals, double alpha, const double *x,
                        double beta, const double *y_in, double *y_out)
{
    double *sum = NULL, *comp = NULL;
    int64_t i, k;
    if (m < 0 || n < 0 || nnz < 0) return -1;
    for (k = 0; k < nnz; ++k) {
        if (rows[k] < 0 || rows[k] >= m || cols[k] < 0 || cols[k] >= n)
            return -1;
    }
    sum = (double *)calloc((size_t)(m > 0 ? m : 1), sizeof(double));
    comp = (double *)calloc((size_t)(m > 0 ? m : 1), sizeof(double));
    if (!sum || !comp) {
        free(sum);
        free(comp);
        return -2;
    }
    for (k = 0; k < nnz; ++k) {
        int64_t r = rows[k];
        double term = vals[k] * x[cols[k]];
        double yk = term - comp[r];
        double t = sum[r] + yk;
        comp[r] = (t - sum[r]) - yk;
        sum[r] = t;
    }
    for (i = 0; i < m; ++i) {
        double acc = alpha * sum[i];
        y_out[i] = (beta == 0.0) ? acc : acc + beta * y_in[i];
    }
    free(sum);
    free(comp);
    return 0;
}

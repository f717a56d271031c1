// Checked products: with the environment variable SPMV_CHECKED=1, spmv_run
// first verifies every stored index of the active format against the
// matrix bounds -- the index arrays a product kernel dereferences: columns
// it gathers x at, rows (or permutation entries) it writes y at, and the
// row-pointer arrays that bound its loops.  A bad index sets STATUS_BOUNDS
// in the handle's status word and the product is not launched: spmv_run
// returns SPMV_ERR_BOUNDS, having accessed nothing through the bad index.
// The check costs one extra pass over the indices and a synchronisation per
// product; it is a debug mode for indices corrupted after spmv_create (which
// validates the triplets it converts), not the default.
#include <cstdlib>

#include "bulk.cuh"
#include "internal.cuh"

namespace spmv {
namespace {

// every a[i] in [lo, hi) or equal to `pad` (a padding marker)
__global__ void k_check_range(const int *a, int64_t count, int64_t lo, int64_t hi, int pad, unsigned *status) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
        const int v = a[i];
        if (v != pad && (v < lo || v >= hi)) bad = true;
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, STATUS_BOUNDS);
}

// ELL 16-bit column offsets: row r's entries r + d in [0, n), or the marker
__global__ void k_check_d16(const int16_t *a, int64_t width, int64_t pitch, int64_t m, int64_t n,
                            unsigned *status) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t count = width * pitch;
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
        const int d = a[i];
        const int64_t r = i % pitch, c = r + d;
        if (d != INT16_MIN && (r >= m || c < 0 || c >= n)) bad = true;
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, STATUS_BOUNDS);
}

// row pointers: p[0] == 0, nondecreasing, p[rows] == total
__global__ void k_check_ptr(const int *p, int64_t rows, int64_t total, unsigned *status) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= rows; i += stride) {
        const int v = p[i];
        if (v < 0 || v > total || (i == 0 && v != 0) || (i == rows && v != total) || (i < rows && p[i + 1] < v))
            bad = true;
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, STATUS_BOUNDS);
}

unsigned grid_for(int64_t n) {
    const int64_t g = (n + 255) / 256;
    return (unsigned)(g < 1 ? 1 : (g > 4096 ? 4096 : g));
}

}  // namespace

bool checked_mode() {
    const char *v = std::getenv("SPMV_CHECKED");
    return v && v[0] == '1';
}

// Verifies the handle's active-format indices (see the file comment); on a
// bad index returns SPMV_ERR_BOUNDS with STATUS_BOUNDS set.
int check_indices(const spmv_matrix *h, cudaStream_t s) {
    unsigned *st = h->d_status;
    const int64_t m = h->m, n = h->n;
    const int NOPAD = INT32_MIN;
    k_check_ptr<<<grid_for(m + 1), 256, 0, s>>>(h->rowptr, m, h->nnz, st);
    k_check_range<<<grid_for(h->nnz), 256, 0, s>>>(h->colidx, h->nnz, 0, n, NOPAD, st);
    switch (h->cfg.format) {
    case SPMV_FMT_ELL:
    case SPMV_FMT_HYB:
        if (h->ell_d16)
            k_check_d16<<<grid_for(h->ell_width * h->ell_pitch), 256, 0, s>>>(h->ell_d16, h->ell_width, h->ell_pitch,
                                                                             m, n, st);
        else if (h->ell_col)
            k_check_range<<<grid_for(h->ell_width * h->ell_pitch), 256, 0, s>>>(h->ell_col, h->ell_width * h->ell_pitch,
                                                                               0, n, -1, st);
        if (h->cfg.format == SPMV_FMT_HYB && h->hyb_nnz > 0) {
            k_check_range<<<grid_for(h->hyb_nnz), 256, 0, s>>>(h->hyb_rows, h->hyb_nnz, 0, m, NOPAD, st);
            k_check_range<<<grid_for(h->hyb_nnz), 256, 0, s>>>(h->hyb_cols, h->hyb_nnz, 0, n, NOPAD, st);
        }
        break;
    case SPMV_FMT_COO:
        k_check_range<<<grid_for(h->nnz), 256, 0, s>>>(h->coo_rows, h->nnz, 0, m, NOPAD, st);
        break;
    case SPMV_FMT_BSR:
        k_check_ptr<<<grid_for(h->bsr_mb + 1), 256, 0, s>>>(h->bsr_rowptr, h->bsr_mb, h->bsr_blocks, st);
        k_check_range<<<grid_for(h->bsr_blocks), 256, 0, s>>>(h->bsr_col, h->bsr_blocks, 0,
                                                             (n + h->bsr_r - 1) / h->bsr_r, NOPAD, st);
        break;
    case SPMV_FMT_SELL:
        k_check_ptr<<<grid_for(h->sell_nslices + 1), 256, 0, s>>>(h->sell_ptr, h->sell_nslices, h->sell_slots, st);
        k_check_range<<<grid_for(h->sell_slots), 256, 0, s>>>(h->sell_col, h->sell_slots, 0, n, -1, st);
        k_check_range<<<grid_for(m), 256, 0, s>>>(h->sell_perm, m, 0, m, NOPAD, st);
        break;
    default:
        break;
    }
    SPMV_CUDA_TRY(cudaGetLastError());
    unsigned w = 0;
    SPMV_CUDA_TRY(cudaMemcpyAsync(&w, st, sizeof w, cudaMemcpyDeviceToHost, s));
    SPMV_CUDA_TRY(cudaStreamSynchronize(s));
    if (w & STATUS_BOUNDS) {
        set_error("spmv_run: an index of the stored matrix is out of bounds; the product was not launched");
        return SPMV_ERR_BOUNDS;
    }
    return SPMV_OK;
}

}  // namespace spmv

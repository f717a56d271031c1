// Host-side launchers for every kernel family, templated on the value type.
// Each translation unit kernels_<type>.cu instantiates them for one type, so
// the ~150 kernel variants compile in parallel.
#pragma once

#include <algorithm>
#include <type_traits>

#include "kernels_rows.cuh"
#include "kernels_seg.cuh"

namespace spmv {

// occupancy-limited resident blocks per SM for (kernel, block size); cached
int resident_blocks(const void *kernel, int threads);

// grid of at most one full wave of resident blocks (grid-stride kernels)
inline int wave_grid(const void *kernel, int threads, int64_t needed_blocks, int sm_count) {
    const int64_t cap = (int64_t)resident_blocks(kernel, threads) * sm_count;
    int64_t g = needed_blocks < cap ? needed_blocks : cap;
    return (int)(g < 1 ? 1 : g);
}

#define SPMV_LAUNCH_CHECK()                                      \
    do {                                                         \
        cudaError_t _e = cudaGetLastError();                     \
        if (_e != cudaSuccess) return cuda_status(_e, "kernel launch"); \
    } while (0)

// ------------------------------- long rows ---------------------------------
template <typename V, typename T>
int launch_csr_long(const spmv_matrix *h, T alpha, const T *x, T beta, T *y, cudaStream_t s) {
    const LongRows &L = h->lng;
    if (L.nseg == 0) return SPMV_OK;
    auto kern = k_csr_long<V, T>;
    const int grid = wave_grid((const void *)kern, 256, L.nseg, h->sm_count);
    kern<<<grid, 256, 0, s>>>(L.nseg, L.seg_row, L.seg_begin, L.seg_end, L.seg_c0, L.seg_c1, h->colidx,
                              (const V *)h->vals, x, y, alpha, beta, PartialsT<T>::of(L.part));
    SPMV_LAUNCH_CHECK();
    return SPMV_OK;
}

template <typename V, typename T, int R>
int launch_bsr_long(const spmv_matrix *h, T alpha, const T *x, T beta, T *y, cudaStream_t s) {
    const LongRows &L = h->lng;
    if (L.nseg == 0) return SPMV_OK;
    auto kern = k_bsr_long<V, T, R>;
    const int grid = wave_grid((const void *)kern, 256, L.nseg, h->sm_count);
    kern<<<grid, 256, 0, s>>>(L.nseg, L.seg_row, L.seg_begin, L.seg_end, L.seg_c0, L.seg_c1, h->m, h->n, h->bsr_col,
                              (const V *)h->bsr_val, x, y, alpha, beta, PartialsT<T>::of(L.part));
    SPMV_LAUNCH_CHECK();
    return SPMV_OK;
}

// ------------------------------- CSR vector --------------------------------
template <typename V, typename T, int TPR, int U, int RC, int GW>
int launch_csr_vector(const spmv_matrix *h, T alpha, const T *x, T beta, T *y, cudaStream_t s) {
    auto kern = k_csr_vector<V, T, TPR, U, RC, GW>;
    const int tpb = h->cfg.threads_per_block;
    SPMV_TRY(apply_carveout((const void *)kern, h->cfg.carveout));
    const int64_t rows_per_block = tpb / TPR;
    const int grid = wave_grid((const void *)kern, tpb, (h->m + rows_per_block - 1) / rows_per_block, h->sm_count);
    const int thr = h->lng.nseg > 0 ? (int)h->lng.threshold : 0x7fffffff;
    kern<<<grid, tpb, 0, s>>>(h->m, h->rowptr, h->colidx, (const V *)h->vals, x, y, alpha, beta, thr);
    SPMV_LAUNCH_CHECK();
    return launch_csr_long<V, T>(h, alpha, x, beta, y, s);
}

// bsr_block selects the load group of one or two lanes per row: 8 entries
// (32-byte loads) or 4; more lanes per row read interleaved entries
template <typename V, typename T, int TPR, int U>
int csr_vector_rc(const spmv_matrix *h, T a, const T *x, T b, T *y, cudaStream_t s) {
    if constexpr (TPR <= 2) {
        if (h->cfg.bsr_block == 8)
            return h->cfg.regcap == 32 ? launch_csr_vector<V, T, TPR, U, 32, 8>(h, a, x, b, y, s)
                                       : launch_csr_vector<V, T, TPR, U, 64, 8>(h, a, x, b, y, s);
    }
    return h->cfg.regcap == 32 ? launch_csr_vector<V, T, TPR, U, 32, 4>(h, a, x, b, y, s)
                               : launch_csr_vector<V, T, TPR, U, 64, 4>(h, a, x, b, y, s);
}

template <typename V, typename T, int TPR>
int csr_vector_u(const spmv_matrix *h, T a, const T *x, T b, T *y, cudaStream_t s) {
    switch (h->cfg.unroll) {
    case 1: return csr_vector_rc<V, T, TPR, 1>(h, a, x, b, y, s);
    case 2: return csr_vector_rc<V, T, TPR, 2>(h, a, x, b, y, s);
    default: return csr_vector_rc<V, T, TPR, 4>(h, a, x, b, y, s);
    }
}

template <int VT>
int run_csr_vector_vt(const spmv_matrix *h, double alpha, const void *x, double beta, void *y, cudaStream_t s) {
    using V = typename VT_<VT>::V;
    using T = typename VT_<VT>::T;
    const T a = (T)alpha, b = (T)beta;
    const T *xx = (const T *)x;
    T *yy = (T *)y;
    switch (h->cfg.threads_per_row) {
    case 1: return csr_vector_u<V, T, 1>(h, a, xx, b, yy, s);
    case 2: return csr_vector_u<V, T, 2>(h, a, xx, b, yy, s);
    case 4: return csr_vector_u<V, T, 4>(h, a, xx, b, yy, s);
    case 8: return csr_vector_u<V, T, 8>(h, a, xx, b, yy, s);
    case 16: return csr_vector_u<V, T, 16>(h, a, xx, b, yy, s);
    default: return csr_vector_u<V, T, 32>(h, a, xx, b, yy, s);
    }
}

// ----------------------------------- ELL -----------------------------------
template <typename V, typename T, int U, int RC, typename CI>
int launch_ell_ci(const spmv_matrix *h, const CI *cols, int64_t width, T alpha, const T *x, T beta, T *y,
                  cudaStream_t s) {
    const int tpb = h->cfg.threads_per_block;
    if constexpr (!std::is_same<V, double>::value) {  // fp32/bf16: two rows per thread
        auto kern = k_ell2<V, T, U, RC, CI>;
        SPMV_TRY(apply_carveout((const void *)kern, h->cfg.carveout));
        const int64_t pairs = (h->m + 1) / 2;
        const int grid = wave_grid((const void *)kern, tpb, (pairs + tpb - 1) / tpb, h->sm_count);
        kern<<<grid, tpb, 0, s>>>(h->m, width, h->ell_pitch, cols, (const V *)h->ell_val, x, y, alpha, beta);
    } else {
        auto kern = k_ell<V, T, U, RC, CI>;
        SPMV_TRY(apply_carveout((const void *)kern, h->cfg.carveout));
        const int grid = wave_grid((const void *)kern, tpb, (h->m + tpb - 1) / tpb, h->sm_count);
        kern<<<grid, tpb, 0, s>>>(h->m, width, h->ell_pitch, cols, (const V *)h->ell_val, x, y, alpha, beta);
    }
    SPMV_LAUNCH_CHECK();
    return SPMV_OK;
}

template <typename V, typename T, int U, int RC>
int launch_ell_rc(const spmv_matrix *h, int64_t width, T alpha, const T *x, T beta, T *y, cudaStream_t s) {
    if (h->ell_d16) return launch_ell_ci<V, T, U, RC, int16_t>(h, h->ell_d16, width, alpha, x, beta, y, s);
    return launch_ell_ci<V, T, U, RC, int>(h, h->ell_col, width, alpha, x, beta, y, s);
}

template <typename V, typename T, int U>
int launch_ell(const spmv_matrix *h, int64_t width, T alpha, const T *x, T beta, T *y, cudaStream_t s) {
    switch (h->cfg.regcap) {
    case 32: return launch_ell_rc<V, T, U, 32>(h, width, alpha, x, beta, y, s);
    case 48: return launch_ell_rc<V, T, U, 48>(h, width, alpha, x, beta, y, s);
    default: return launch_ell_rc<V, T, U, 64>(h, width, alpha, x, beta, y, s);
    }
}

template <int VT>
int run_ell_vt(const spmv_matrix *h, double alpha, const void *x, double beta, void *y, cudaStream_t s) {
    using V = typename VT_<VT>::V;
    using T = typename VT_<VT>::T;
    const T a = (T)alpha, b = (T)beta;
    switch (h->cfg.unroll) {
    case 1: return launch_ell<V, T, 1>(h, h->ell_width, a, (const T *)x, b, (T *)y, s);
    case 2: return launch_ell<V, T, 2>(h, h->ell_width, a, (const T *)x, b, (T *)y, s);
    case 8: return launch_ell<V, T, 8>(h, h->ell_width, a, (const T *)x, b, (T *)y, s);
    default: return launch_ell<V, T, 4>(h, h->ell_width, a, (const T *)x, b, (T *)y, s);
    }
}

// ----------------------------------- BSR -----------------------------------
template <typename V, typename T, int R, int S>
int launch_bsr(const spmv_matrix *h, T alpha, const T *x, T beta, T *y, cudaStream_t s) {
    auto kern = k_bsr<V, T, R, S>;
    const int tpb = h->cfg.threads_per_block;
    SPMV_TRY(apply_carveout((const void *)kern, h->cfg.carveout));
    const int64_t brows_per_block = tpb / (R * S);
    const int grid =
        wave_grid((const void *)kern, tpb, (h->bsr_mb + brows_per_block - 1) / brows_per_block, h->sm_count);
    const int thr = h->lng.nseg > 0 ? (int)h->lng.threshold : 0x7fffffff;
    kern<<<grid, tpb, 0, s>>>(h->bsr_mb, h->m, h->n, h->bsr_rowptr, h->bsr_col, (const V *)h->bsr_val, x, y, alpha,
                              beta, thr);
    SPMV_LAUNCH_CHECK();
    return launch_bsr_long<V, T, R>(h, alpha, x, beta, y, s);
}

template <typename V, typename T, int R>
int bsr_s(const spmv_matrix *h, T a, const T *x, T b, T *y, cudaStream_t s) {
    switch (h->cfg.threads_per_row) {
    case 2: return launch_bsr<V, T, R, 2>(h, a, x, b, y, s);
    case 4: return launch_bsr<V, T, R, 4>(h, a, x, b, y, s);
    case 8: return launch_bsr<V, T, R, 8>(h, a, x, b, y, s);
    default: return launch_bsr<V, T, R, 1>(h, a, x, b, y, s);
    }
}

template <int VT>
int run_bsr_vt(const spmv_matrix *h, double alpha, const void *x, double beta, void *y, cudaStream_t s) {
    using V = typename VT_<VT>::V;
    using T = typename VT_<VT>::T;
    const T a = (T)alpha, b = (T)beta;
    if (h->bsr_r == 2) return bsr_s<V, T, 2>(h, a, (const T *)x, b, (T *)y, s);
    return bsr_s<V, T, 4>(h, a, (const T *)x, b, (T *)y, s);
}

// ----------------------------------- SELL ----------------------------------
template <typename V, typename T, int U, int RC, bool GROUPED>
int launch_sell_g(const spmv_matrix *h, T alpha, const T *x, T beta, T *y, cudaStream_t s) {
    auto kern = k_sell<V, T, U, RC, GROUPED>;
    const int tpb = h->cfg.threads_per_block;
    SPMV_TRY(apply_carveout((const void *)kern, h->cfg.carveout));
    const LongRows &L = h->lng;  // items; nrows = first slice of empty rows
    const int64_t wpb = tpb / 32;
    const int64_t empty_rows = h->m - 32 * L.nrows > 0 ? h->m - 32 * L.nrows : 0;
    const int64_t need = std::max((L.nseg + wpb - 1) / wpb, (empty_rows + tpb - 1) / tpb);
    const int grid = wave_grid((const void *)kern, tpb, need, h->sm_count);
    kern<<<grid, tpb, 0, s>>>(h->m, L.nseg, L.nrows, L.seg_row, L.seg_begin, L.seg_end, L.seg_c0, L.seg_c1, h->sell_col,
                              (const V *)h->sell_val, h->sell_perm, x, y, alpha, beta, PartialsT<T>::of(L.part));
    SPMV_LAUNCH_CHECK();
    return SPMV_OK;
}

template <typename V, typename T, int U, int RC>
int launch_sell_rc(const spmv_matrix *h, T alpha, const T *x, T beta, T *y, cudaStream_t s) {
    return h->sell_grouped ? launch_sell_g<V, T, U, RC, true>(h, alpha, x, beta, y, s)
                           : launch_sell_g<V, T, U, RC, false>(h, alpha, x, beta, y, s);
}

template <typename V, typename T, int U>
int launch_sell(const spmv_matrix *h, T alpha, const T *x, T beta, T *y, cudaStream_t s) {
    switch (h->cfg.regcap) {
    case 32: return launch_sell_rc<V, T, U, 32>(h, alpha, x, beta, y, s);
    case 48: return launch_sell_rc<V, T, U, 48>(h, alpha, x, beta, y, s);
    default: return launch_sell_rc<V, T, U, 64>(h, alpha, x, beta, y, s);
    }
}

template <int VT>
int run_sell_vt(const spmv_matrix *h, double alpha, const void *x, double beta, void *y, cudaStream_t s) {
    using V = typename VT_<VT>::V;
    using T = typename VT_<VT>::T;
    const T a = (T)alpha, b = (T)beta;
    switch (h->cfg.unroll) {
    case 1: return launch_sell<V, T, 1>(h, a, (const T *)x, b, (T *)y, s);
    case 2: return launch_sell<V, T, 2>(h, a, (const T *)x, b, (T *)y, s);
    case 8: return launch_sell<V, T, 8>(h, a, (const T *)x, b, (T *)y, s);
    default: return launch_sell<V, T, 4>(h, a, (const T *)x, b, (T *)y, s);
    }
}

// ---------------------------- COO / HYB / split ----------------------------
template <typename V, typename T, int ITEMS, bool ACCUM>
int launch_coo(const spmv_matrix *h, int64_t nnz, const int *rows, const int *cols, const V *vals, T alpha,
               const T *x, T beta, T *y, cudaStream_t s) {
    auto kern = k_coo_seg<V, T, ITEMS, ACCUM, true>;
    const int tpb = ITEMS >= 16 && h->cfg.threads_per_block > 512 ? 512 : h->cfg.threads_per_block;
    SPMV_TRY(apply_carveout((const void *)kern, h->cfg.carveout));
    const int64_t chunks = (nnz + 32 * ITEMS - 1) / (32 * ITEMS);
    const int64_t wpb = tpb / 32;
    const int grid = wave_grid((const void *)kern, tpb, (chunks + wpb - 1) / wpb, h->sm_count);
    kern<<<grid, tpb, 0, s>>>(nnz, h->m, rows, cols, vals, x, y, alpha, beta, h->seg.meta0, h->seg.meta1,
                              PartialsT<T>::of(h->seg.part));
    SPMV_LAUNCH_CHECK();
    return SPMV_OK;
}

template <typename V, typename T, bool ACCUM>
int coo_items(const spmv_matrix *h, int64_t nnz, const int *rows, const int *cols, const V *vals, T a,
              const T *x, T b, T *y, cudaStream_t s) {
    switch (h->seg.items) {
    case 4: return launch_coo<V, T, 4, ACCUM>(h, nnz, rows, cols, vals, a, x, b, y, s);
    case 8: return launch_coo<V, T, 8, ACCUM>(h, nnz, rows, cols, vals, a, x, b, y, s);
    default: return launch_coo<V, T, 16, ACCUM>(h, nnz, rows, cols, vals, a, x, b, y, s);
    }
}

template <int VT>
int run_coo_vt(const spmv_matrix *h, double alpha, const void *x, double beta, void *y, cudaStream_t s) {
    using V = typename VT_<VT>::V;
    using T = typename VT_<VT>::T;
    return coo_items<V, T, false>(h, h->nnz, h->coo_rows, h->colidx, (const V *)h->vals, (T)alpha, (const T *)x,
                                  (T)beta, (T *)y, s);
}

template <int VT>
int run_hyb_vt(const spmv_matrix *h, double alpha, const void *x, double beta, void *y, cudaStream_t s) {
    using V = typename VT_<VT>::V;
    using T = typename VT_<VT>::T;
    SPMV_TRY(run_ell_vt<VT>(h, alpha, x, beta, y, s));
    if (h->hyb_nnz == 0) return SPMV_OK;
    return coo_items<V, T, true>(h, h->hyb_nnz, h->hyb_rows, h->hyb_cols, (const V *)h->hyb_vals, (T)alpha,
                                 (const T *)x, (T)beta, (T *)y, s);
}

// occupancy-limited resident blocks per SM with dynamic shared memory (not cached)
inline int resident_blocks_smem(const void *kernel, int threads, size_t smem) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, smem) != cudaSuccess || nb < 1) {
        cudaGetLastError();
        nb = 1;
    }
    return nb;
}

// the staged nonzero-tile kernel: lanes per row from the mean row length (at
// most 8), gathers in flight per lane 4 (unroll <= 2) or 8 (unroll 4)
template <typename V, typename T, int TPR, int U>
int launch_tiles(const spmv_matrix *h, T alpha, const T *x, T beta, T *y, cudaStream_t s) {
    auto kern = k_csr_tiles<V, T, TPR, U>;
    const int tpb = h->cfg.threads_per_block < TPR ? TPR : h->cfg.threads_per_block;
    const int tile = 32 * h->seg.items;
    // a row segment longer than 8 gathers per lane of its group goes to a
    // whole warp, one longer than 8 gathers per lane of a warp to the block
    const int long_len = 8 * 32 * U;
    const int long_max = tile / (8 * TPR * U + 1) + 2;  // room for every segment the groups pass on
    const TileSmem L = tile_smem_layout<V>(tile, long_max);
    SPMV_CUDA_TRY(cudaFuncSetAttribute((const void *)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L.total));
    SPMV_TRY(apply_carveout((const void *)kern, h->cfg.carveout));
    const int64_t ntiles = h->seg.nchunks;
    const int64_t cap = (int64_t)resident_blocks_smem((const void *)kern, tpb, L.total) * h->sm_count;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, cap));
    kern<<<grid, tpb, L.total, s>>>(h->nnz, h->m, ntiles, tile, long_len, long_max, h->rowptr, h->colidx,
                                    (const V *)h->vals, x, y, alpha, beta, h->seg.meta0,
                                    PartialsT<T>::of(h->seg.part), h->d_status);
    SPMV_LAUNCH_CHECK();
    return SPMV_OK;
}

template <typename V, typename T, int U>
int tiles_tpr(const spmv_matrix *h, T a, const T *x, T b, T *y, cudaStream_t s) {
    const int tpr = std::min(8, default_tpr(h));
    switch (tpr) {
    case 1: return launch_tiles<V, T, 1, U>(h, a, x, b, y, s);
    case 2: return launch_tiles<V, T, 2, U>(h, a, x, b, y, s);
    case 4: return launch_tiles<V, T, 4, U>(h, a, x, b, y, s);
    default: return launch_tiles<V, T, 8, U>(h, a, x, b, y, s);
    }
}

// split CSR by warp chunks: one MergeSmem per warp in dynamic shared memory
template <typename V, typename T, int ITEMS>
int launch_merge(const spmv_matrix *h, T alpha, const T *x, T beta, T *y, cudaStream_t s) {
    auto kern = k_csr_merge<V, T, ITEMS>;
    const int tpb = ITEMS >= 16 && h->cfg.threads_per_block > 512 ? 512 : h->cfg.threads_per_block;
    const size_t smem = sizeof(MergeSmem<ITEMS>) * (size_t)(tpb / 32);
    if (smem > 48 * 1024)
        SPMV_CUDA_TRY(cudaFuncSetAttribute((const void *)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    SPMV_TRY(apply_carveout((const void *)kern, h->cfg.carveout));
    const int64_t chunks = h->seg.nchunks;
    const int64_t wpb = tpb / 32;
    const int64_t cap = (int64_t)resident_blocks_smem((const void *)kern, tpb, smem) * h->sm_count;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((chunks + wpb - 1) / wpb, cap));
    kern<<<grid, tpb, smem, s>>>(h->nnz, h->m, h->rowptr, h->colidx, (const V *)h->vals, x, y, alpha, beta,
                                 h->seg.meta0, PartialsT<T>::of(h->seg.part));
    SPMV_LAUNCH_CHECK();
    return SPMV_OK;
}

template <int VT>
int run_csr_split_vt(const spmv_matrix *h, double alpha, const void *x, double beta, void *y, cudaStream_t s) {
    using V = typename VT_<VT>::V;
    using T = typename VT_<VT>::T;
    const T a = (T)alpha, b = (T)beta;
    if (h->cfg.hyb_ell_width == 0) {
        switch (h->seg.items) {
        case 4: return launch_merge<V, T, 4>(h, a, (const T *)x, b, (T *)y, s);
        case 8: return launch_merge<V, T, 8>(h, a, (const T *)x, b, (T *)y, s);
        default: return launch_merge<V, T, 16>(h, a, (const T *)x, b, (T *)y, s);
        }
    }
    if (h->cfg.unroll >= 4) return tiles_tpr<V, T, 8>(h, a, (const T *)x, b, (T *)y, s);
    return tiles_tpr<V, T, 4>(h, a, (const T *)x, b, (T *)y, s);
}

template <int VT>
int run_scale_y_vt(int64_t m, double beta, void *y, cudaStream_t s) {
    using T = typename VT_<VT>::T;
    if (m == 0) return SPMV_OK;
    k_scale_y<T><<<(unsigned)((m + 255) / 256 < 4096 ? (m + 255) / 256 : 4096), 256, 0, s>>>(m, (T *)y, (T)beta);
    SPMV_LAUNCH_CHECK();
    return SPMV_OK;
}

#define SPMV_DEFINE_RUNNER(NAME, VT)                                                                 \
    int NAME(int kind, const spmv_matrix *h, double a, const void *x, double b, void *y, cudaStream_t s) { \
        switch (kind) {                                                                                  \
        case RUN_CSR_VECTOR: return run_csr_vector_vt<VT>(h, a, x, b, y, s);                             \
        case RUN_CSR_SPLIT: return run_csr_split_vt<VT>(h, a, x, b, y, s);                               \
        case RUN_ELL: return run_ell_vt<VT>(h, a, x, b, y, s);                                           \
        case RUN_COO: return run_coo_vt<VT>(h, a, x, b, y, s);                                           \
        case RUN_HYB: return run_hyb_vt<VT>(h, a, x, b, y, s);                                           \
        case RUN_BSR: return run_bsr_vt<VT>(h, a, x, b, y, s);                                           \
        case RUN_SCALE: return run_scale_y_vt<VT>(h->m, b, y, s);                                        \
        case RUN_SELL: return run_sell_vt<VT>(h, a, x, b, y, s);                                         \
        }                                                                                                \
        return SPMV_ERR_INVALID;                                                                         \
    }

}  // namespace spmv

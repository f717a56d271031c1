// Batched SpMV: hundreds of uneven matrices in one persistent launch.
//
// Each matrix contributes work items for one warp each, in the format its
// handle holds: ELL (groups of 32 rows, a row per lane), SELL (the handle's
// work items, plus groups of 32 of its empty rows), or otherwise CSR --
// chunks of 32*ITEMS nonzeros (split mode, for power-law or very short rows)
// or groups of 32 rows with a per-matrix number of lanes per row (vector
// mode).  A grid of
// resident thread blocks pulls items from one atomic counter, so small and
// large matrices share the GPU without a launch per matrix.  The counter
// reset and the kernel are captured once in a CUDA graph and replayed.  An
// autotuner times the per-matrix mode and the batch-wide chunk and block
// sizes (the paper's compile-time parameters of Section 4, chosen per
// matrix by measurement instead of by a model).
#include <algorithm>
#include <cmath>
#include <vector>

#include "launch.cuh"

struct spmv_batch {
    int count = 0, vt = SPMV_F64, items = 8, tpb = 256, sm_count = 0;
    int group = 4;  // work units (chunks, row groups, SELL items) per batch item
    std::vector<spmv_handle> hs;
    std::vector<double> alpha, beta;
    std::vector<const void *> x;
    std::vector<void *> y;
    std::vector<int> modes;  // 0 split, else threads per row
    // device state
    void *d_mats = nullptr;
    int64_t *d_item_off = nullptr;
    int64_t total_items = 0;
    std::vector<int32_t *> metas;
    spmv::Partials part;
    unsigned long long *d_counter = nullptr;
    cudaStream_t cs = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace spmv {
namespace {

struct BatchMat {
    const int *rowptr;
    const int *colidx;
    const void *vals;
    const void *x;
    void *y;
    double alpha, beta;
    int64_t m, nnz;
    int64_t part_off;  // first chunk of this matrix in the batch partials
    int64_t units;     // work units of this matrix (batch items take `group` of them)
    const int *meta0;  // split: first row starting at or after each chunk's first entry;
                       // COO: first chunk of each chunk's head row
    const int *meta1;  // COO: last chunk of each chunk's tail row
    const int *coo_rows;  // COO handles: the row index of each entry
    // BSR: block rows, r x r blocks; n bounds the last block column
    const int *bsr_rowptr, *bsr_col;
    const void *bsr_val;
    int64_t bsr_mb, n;
    int bsr_r, pad3;
    int mode;          // CSR: 0 split, -2 COO chunks, else lanes per row
    int fmt;           // the handle's format: SPMV_FMT_ELL, SPMV_FMT_SELL, or CSR (any other)
    // ELL: column-major arrays, int32 columns or 16-bit offsets
    const int *ell_col;
    const int16_t *ell_d16;
    const void *ell_val;
    int64_t ell_width, ell_pitch;
    // SELL: the handle's work items, arrays and partials; rows from slice
    // s_zero on are empty
    const int *it_slice, *it_base, *it_len, *it_c0, *it_c1;
    const int *sell_col, *sell_perm;
    const void *sell_val;
    int64_t nitems, s_zero;
    int sell_grouped;
    int wide;  // CSR vector mode: 8-entry load groups (32-byte loads)
    void *p_head, *p_tail;
    unsigned *p_count;
    unsigned long long *p_xslot;
};

// mode of a COO handle run as COO chunks (its own row indices), of a BSR
// handle run as BSR block rows (32 / r block rows per item, r lanes each)
constexpr int BATCH_COO = -SPMV_FMT_COO;
constexpr int BATCH_BSR = -SPMV_FMT_BSR;

// work items of one matrix: CSR split or COO chunks, or 32-row groups, ELL
// 32-row groups, SELL items plus 32-row groups of its empty rows
int64_t batch_items(const BatchMat &M, int C) {
    if (M.fmt == SPMV_FMT_ELL) return (M.m + 31) / 32;
    if (M.fmt == SPMV_FMT_SELL) return M.nitems + (std::max<int64_t>(0, M.m - 32 * M.s_zero) + 31) / 32;
    if (M.fmt == SPMV_FMT_BSR) return (M.bsr_mb + 32 / M.bsr_r - 1) / (32 / M.bsr_r);
    return M.mode == 0 || M.mode == BATCH_COO ? (M.nnz + C - 1) / C : (M.m + 31) / 32;
}

// chunk metadata of a split or COO matrix for chunks of C entries, in one
// allocation of 2 (nchunks + 1) ints (COO: meta0 then meta1)
int build_chunk_meta(const spmv_matrix *h, int mode, int C, int32_t **out, cudaStream_t s) {
    const int64_t nch = (h->nnz + C - 1) / C;
    *out = nullptr;
    SPMV_CUDA_TRY(dev_malloc((void **)out, sizeof(int32_t) * 2 * (nch + 1)));
    return mode == BATCH_COO ? build_coo_meta(h->coo_rows, h->rowptr, h->nnz, C, *out, *out + nch + 1, s)
                             : build_merge_meta(h->rowptr, h->m, h->nnz, C, *out, s);
}

void set_chunk_meta(BatchMat &M, const int32_t *meta, int C) {
    const int64_t nch = (M.nnz + C - 1) / C;
    M.meta0 = meta;
    M.meta1 = meta + nch + 1;
}

// the handle's active format as the batch runs it (ELL, SELL, else CSR modes)
void describe_format(const spmv_matrix *h, BatchMat &M) {
    M.fmt = SPMV_FMT_CSR;
    M.coo_rows = h->cfg.format == SPMV_FMT_COO ? h->coo_rows : nullptr;
    if (h->cfg.format == SPMV_FMT_BSR && h->bsr_rowptr) {
        M.bsr_rowptr = h->bsr_rowptr;
        M.bsr_col = h->bsr_col;
        M.bsr_val = h->bsr_val;
        M.bsr_mb = h->bsr_mb;
        M.bsr_r = h->bsr_r;
    }
    M.n = h->n;
    if (h->cfg.format == SPMV_FMT_ELL && (h->ell_col || h->ell_d16)) {
        M.fmt = SPMV_FMT_ELL;
        M.ell_col = h->ell_col;
        M.ell_d16 = h->ell_d16;
        M.ell_val = h->ell_val;
        M.ell_width = h->ell_width;
        M.ell_pitch = h->ell_pitch;
    } else if (h->cfg.format == SPMV_FMT_SELL && h->sell_col) {
        const LongRows &L = h->lng;
        M.fmt = SPMV_FMT_SELL;
        M.it_slice = L.seg_row;
        M.it_base = L.seg_begin;
        M.it_len = L.seg_end;
        M.it_c0 = L.seg_c0;
        M.it_c1 = L.seg_c1;
        M.sell_col = h->sell_col;
        M.sell_perm = h->sell_perm;
        M.sell_val = h->sell_val;
        M.nitems = L.nseg;
        M.s_zero = L.nrows;
        M.sell_grouped = h->sell_grouped ? 1 : 0;
        M.p_head = L.part.head;
        M.p_tail = L.part.tail;
        M.p_count = L.part.count;
        M.p_xslot = L.part.xslot;
    }
}

// register budget: 16 items per lane, or fp64 sums, need more than 64
// vector mode with one or two lanes per row takes 8-entry load groups once
// a lane's part of a mean row holds 16 or more entries (the single-matrix
// default rule)
int wide_groups(const spmv_matrix *h, int mode) {
    const double mean = h->m > 0 ? (double)h->nnz / (double)h->m : 0.0;
    return mode >= 1 && mode <= 2 && mean / mode >= 16.0 ? 1 : 0;
}

template <typename V, typename T, int ITEMS>
__global__ void __launch_bounds__(512) __maxnreg__(ITEMS >= 16 ? 128 : (sizeof(T) == 8 ? 96 : 64))
k_batch(const BatchMat *__restrict__ mats, int count, const int64_t *__restrict__ item_off, int64_t total,
        int group, unsigned long long *counter, const PartialsT<T> P) {
    __shared__ MergeSmem<ITEMS> s_merge[16];  // split chunks: one per warp
    const int lane = threadIdx.x & 31;
    for (;;) {
        unsigned long long item = 0;
        if (lane == 0) item = atomicAdd(counter, 1ull);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= (unsigned long long)total) break;
        int lo = 0, hi = count - 1;  // matrix owning the item
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if ((unsigned long long)__ldg(item_off + mid) <= item) lo = mid; else hi = mid - 1;
        }
        const BatchMat &M = mats[lo];  // fields read where a branch needs them
        const int64_t u0 = ((int64_t)item - __ldg(item_off + lo)) * group;
        const int64_t u1 = u0 + group < M.units ? u0 + group : M.units;
        const Epi<T> ep((T)M.alpha, (T)M.beta);
        const V *vals = (const V *)M.vals;
        const T *x = (const T *)M.x;
        T *y = (T *)M.y;
        for (int64_t local = u0; local < u1; ++local) {
        if (M.fmt == SPMV_FMT_ELL) {  // 32 rows, one per lane
            const int64_t r = local * 32 + lane;
            if (r < M.m) {
                if (M.ell_d16)
                    ell_row<V, T, 4, int16_t>(r, M.ell_width, M.ell_pitch, M.ell_d16, (const V *)M.ell_val, x, y, ep);
                else
                    ell_row<V, T, 4, int>(r, M.ell_width, M.ell_pitch, M.ell_col, (const V *)M.ell_val, x, y, ep);
            }
        } else if (M.fmt == SPMV_FMT_SELL) {
            if (local < M.nitems) {
                const PartialsT<T> Ps{(T *)M.p_head, (T *)M.p_tail, M.p_count, M.p_xslot, 32};
                if (M.sell_grouped)  // two groups of four in flight, one with 4 items per lane (register budget)
                    sell_item<V, T, (ITEMS >= 8 ? 8 : 4), true>(local, M.m, M.it_slice, M.it_base, M.it_len, M.it_c0, M.it_c1,
                                             M.sell_col, (const V *)M.sell_val, M.sell_perm, x, y, ep, Ps);
                else
                    sell_item<V, T, 4, false>(local, M.m, M.it_slice, M.it_base, M.it_len, M.it_c0, M.it_c1,
                                              M.sell_col, (const V *)M.sell_val, M.sell_perm, x, y, ep, Ps);
            } else {  // 32 of the empty rows
                const int64_t p = M.s_zero * 32 + (local - M.nitems) * 32 + lane;
                if (p < M.m) ep.store(y, __ldg(M.sell_perm + p), T(0));
            }
        } else if (M.fmt == SPMV_FMT_BSR) {  // 32 / r block rows, r lanes per block row
            const int big = 0x7fffffff;
            if (M.bsr_r == 4)
                bsr_rows<V, T, 4, 1>(local * 8, M.bsr_mb, M.m, M.n, M.bsr_rowptr, M.bsr_col, (const V *)M.bsr_val, x,
                                     y, ep, big);
            else
                bsr_rows<V, T, 2, 1>(local * 16, M.bsr_mb, M.m, M.n, M.bsr_rowptr, M.bsr_col, (const V *)M.bsr_val,
                                     x, y, ep, big);
        } else if (M.mode == 0 || M.mode == BATCH_COO) {
            PartialsT<T> Pm = P;
            Pm.head += M.part_off;
            Pm.tail += M.part_off;
            Pm.count += M.part_off;
            Pm.xslot += M.part_off;
            if (M.mode == BATCH_COO)
                coo_chunk<V, T, ITEMS, false, true>(local, M.nnz, M.m, M.coo_rows, M.colidx, vals, x, y, ep, M.meta0,
                                                    M.meta1, Pm);
            else
                csr_merge_chunk<V, T, ITEMS>(local, M.nnz, M.m, M.rowptr, M.colidx, vals, x, y, ep,
                                             __ldg(M.meta0 + local), __ldg(M.meta0 + local + 1), Pm,
                                             s_merge[threadIdx.x >> 5]);
        } else {
            const int64_t base = local * 32;
            const int big = 0x7fffffff;
            switch (M.mode) {
            case 1:
                if (M.wide) csr_vector_rows<V, T, 1, 2, 8>(base, M.m, M.rowptr, M.colidx, vals, x, y, ep, big);
                else csr_vector_rows<V, T, 1, 2>(base, M.m, M.rowptr, M.colidx, vals, x, y, ep, big);
                break;
            case 2:
                if (M.wide) csr_vector_rows<V, T, 2, 2, 8>(base, M.m, M.rowptr, M.colidx, vals, x, y, ep, big);
                else csr_vector_rows<V, T, 2, 2>(base, M.m, M.rowptr, M.colidx, vals, x, y, ep, big);
                break;
            case 4: csr_vector_rows<V, T, 4, 2>(base, M.m, M.rowptr, M.colidx, vals, x, y, ep, big); break;
            case 8: csr_vector_rows<V, T, 8, 2>(base, M.m, M.rowptr, M.colidx, vals, x, y, ep, big); break;
            case 16: csr_vector_rows<V, T, 16, 2>(base, M.m, M.rowptr, M.colidx, vals, x, y, ep, big); break;
            default: csr_vector_rows<V, T, 32, 2>(base, M.m, M.rowptr, M.colidx, vals, x, y, ep, big); break;
            }
        }
        }
    }
}

template <typename V, typename T, int ITEMS>
int launch_batch_t(const spmv_batch *b, const BatchMat *mats, int count, const int64_t *item_off, int64_t total,
                   cudaStream_t s) {
    auto kern = k_batch<V, T, ITEMS>;
    const int per_sm = resident_blocks((const void *)kern, b->tpb);
    const int64_t need = (total + b->tpb / 32 - 1) / (b->tpb / 32);
    const int64_t cap = (int64_t)per_sm * b->sm_count;
    const int grid = (int)std::max<int64_t>(1, std::min(need, cap));
    kern<<<grid, b->tpb, 0, s>>>(mats, count, item_off, total, b->group, b->d_counter, PartialsT<T>::of(b->part));
    SPMV_CUDA_TRY(cudaGetLastError());
    return SPMV_OK;
}

template <int VT>
int launch_batch_vt(const spmv_batch *b, const BatchMat *mats, int count, const int64_t *item_off, int64_t total,
                    cudaStream_t s) {
    using V = typename VT_<VT>::V;
    using T = typename VT_<VT>::T;
    switch (b->items) {
    case 4: return launch_batch_t<V, T, 4>(b, mats, count, item_off, total, s);
    case 16: return launch_batch_t<V, T, 16>(b, mats, count, item_off, total, s);
    default: return launch_batch_t<V, T, 8>(b, mats, count, item_off, total, s);
    }
}

// counter reset + one persistent kernel over `count` descriptors
int launch_batch(const spmv_batch *b, const BatchMat *mats, int count, const int64_t *item_off, int64_t total,
                 cudaStream_t s) {
    SPMV_CUDA_TRY(cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned long long), s));
    if (total == 0) return SPMV_OK;
    switch (b->vt) {
    case SPMV_F64: return launch_batch_vt<SPMV_F64>(b, mats, count, item_off, total, s);
    case SPMV_F32: return launch_batch_vt<SPMV_F32>(b, mats, count, item_off, total, s);
    default: return launch_batch_vt<SPMV_BF16>(b, mats, count, item_off, total, s);
    }
}

int default_mode(const spmv_matrix *h) {
    if (h->nnz == 0 || h->m == 0) return 1;  // vector mode writes y = beta*y for every row
    const double mean = (double)h->nnz / (double)h->m;
    if ((double)h->max_row > 8.0 * mean + 64.0 || mean < 2.0) return 0;
    int t = 1;
    while (t < 32 && 2.0 * t <= mean / 8.0) t *= 2;
    return t;
}

void free_device(spmv_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    if (b->d_mats) cudaFree(b->d_mats);
    if (b->d_item_off) cudaFree(b->d_item_off);
    b->d_mats = nullptr;
    b->d_item_off = nullptr;
    for (int32_t *p : b->metas)
        if (p) cudaFree(p);
    b->metas.clear();
    free_partials(&b->part);
}

// Builds descriptors, item offsets, split metadata and partials for the
// current modes / items, then captures the graph.
int build(spmv_batch *b, cudaStream_t s) {
    free_device(b);
    const int C = 32 * b->items;
    std::vector<BatchMat> mats(b->count);
    std::vector<int64_t> off(b->count + 1, 0);
    b->metas.assign(b->count, nullptr);
    int64_t chunks_total = 0;
    for (int i = 0; i < b->count; ++i) {
        const spmv_matrix *h = b->hs[i];
        BatchMat &M = mats[i];
        M.rowptr = h->rowptr;
        M.colidx = h->colidx;
        M.vals = h->vals;
        M.x = b->x[i];
        M.y = b->y[i];
        M.alpha = b->alpha[i];
        M.beta = b->beta[i];
        M.m = h->m;
        M.nnz = h->nnz;
        M.mode = b->modes[i];
        M.wide = wide_groups(h, M.mode);
        M.part_off = 0;
        M.meta0 = M.meta1 = nullptr;
        describe_format(h, M);
        if (M.mode == BATCH_COO && !M.coo_rows) M.mode = b->modes[i] = 0;  // COO chunks need COO rows
        if (M.mode == BATCH_BSR) {
            if (M.bsr_rowptr) M.fmt = SPMV_FMT_BSR;
            else M.mode = b->modes[i] = default_mode(h);
        }
        if (M.fmt == SPMV_FMT_CSR && (M.mode == 0 || M.mode == BATCH_COO)) {
            const int64_t nch = (h->nnz + C - 1) / C;
            SPMV_TRY(build_chunk_meta(h, M.mode, C, &b->metas[i], s));
            set_chunk_meta(M, b->metas[i], C);
            M.part_off = chunks_total;
            chunks_total += nch;
        }
        M.units = batch_items(M, C);
        off[i + 1] = off[i] + (M.units + b->group - 1) / b->group;
    }
    b->total_items = off[b->count];
    SPMV_TRY(alloc_partials(&b->part, chunks_total, 1, b->vt, s));
    SPMV_CUDA_TRY(dev_malloc(&b->d_mats, sizeof(BatchMat) * std::max(1, b->count)));
    SPMV_CUDA_TRY(dev_malloc((void **)&b->d_item_off, sizeof(int64_t) * (b->count + 1)));
    SPMV_CUDA_TRY(cudaMemcpyAsync(b->d_mats, mats.data(), sizeof(BatchMat) * b->count, cudaMemcpyHostToDevice, s));
    SPMV_CUDA_TRY(cudaMemcpyAsync(b->d_item_off, off.data(), sizeof(int64_t) * (b->count + 1),
                                  cudaMemcpyHostToDevice, s));
    SPMV_CUDA_TRY(cudaStreamSynchronize(s));
    // capture: counter reset + kernel, replayed by spmv_batch_launch
    SPMV_CUDA_TRY(cudaStreamBeginCapture(b->cs, cudaStreamCaptureModeThreadLocal));
    int st = launch_batch(b, (const BatchMat *)b->d_mats, b->count, b->d_item_off, b->total_items, b->cs);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->cs, &g);
    if (st != SPMV_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return cuda_status(e, "cudaStreamEndCapture");
    b->graph = g;
    SPMV_CUDA_TRY(cudaGraphInstantiate(&b->exec, g, 0));
    return SPMV_OK;
}

// median time (us) of `reps` launches of a sub-batch on stream s
float time_launch(const spmv_batch *b, const BatchMat *mats, int count, const int64_t *off, int64_t total,
                  cudaStream_t s, int reps, int *status) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    std::vector<float> ts;
    *status = launch_batch(b, mats, count, off, total, s);  // warm-up
    for (int r = 0; r < reps && *status == SPMV_OK; ++r) {
        cudaEventRecord(e0, s);
        *status = launch_batch(b, mats, count, off, total, s);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ts.push_back(ms * 1e3f);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (ts.empty()) return 1e30f;
    std::sort(ts.begin(), ts.end());
    return ts[ts.size() / 2];
}

}  // namespace
}  // namespace spmv

using namespace spmv;

extern "C" {

int spmv_batch_create(spmv_batch_handle *out, const spmv_handle *hs, int32_t count, const double *alpha,
                      const void *const *d_x, const double *beta, void *const *d_y, void *stream) {
    entry_reset();
    if (!out || count < 0 || (count > 0 && (!hs || !alpha || !d_x || !beta || !d_y))) {
        set_error("spmv_batch_create: bad arguments");
        return SPMV_ERR_INVALID;
    }
    *out = nullptr;
    int vt = -1;
    for (int i = 0; i < count; ++i) {
        if (!hs[i]) {
            set_error("spmv_batch_create: NULL handle %d", i);
            return SPMV_ERR_INVALID;
        }
        if (vt >= 0 && hs[i]->vt != vt) {
            set_error("spmv_batch_create: handles mix value types");
            return SPMV_ERR_INVALID;
        }
        vt = hs[i]->vt;
        if (hs[i]->npanels > 0) {
            set_error("spmv_batch_create: matrix %d is held in row panels (too many nonzeros for a batch)", i);
            return SPMV_ERR_UNSUPPORTED;
        }
        if ((hs[i]->m > 0 && !d_y[i]) || (hs[i]->nnz > 0 && !d_x[i])) {
            set_error("spmv_batch_create: NULL vector for matrix %d", i);
            return SPMV_ERR_INVALID;
        }
    }
    spmv_batch *b = new (std::nothrow) spmv_batch();
    if (!b) {
        set_error("spmv_batch_create: host allocation failed");
        return SPMV_ERR_OOM;
    }
    b->count = count;
    b->vt = vt < 0 ? SPMV_F64 : vt;
    b->hs.assign(hs, hs + count);
    b->alpha.assign(alpha, alpha + count);
    b->beta.assign(beta, beta + count);
    b->x.assign(d_x, d_x + count);
    b->y.assign(d_y, d_y + count);
    b->modes.resize(count);
    for (int i = 0; i < count; ++i) {
        BatchMat probe{};
        describe_format(hs[i], probe);
        // ELL and SELL matrices run in their own format (mode -format), COO
        // matrices as COO chunks (mode -2, which the tuner may trade for a
        // CSR mode); the others in a CSR mode
        b->modes[i] = probe.fmt != SPMV_FMT_CSR                 ? -probe.fmt
                      : probe.coo_rows && hs[i]->nnz > 0   ? BATCH_COO
                      : probe.bsr_rowptr && hs[i]->nnz > 0 ? BATCH_BSR
                                                           : default_mode(hs[i]);
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = dev_malloc((void **)&b->d_counter, sizeof(unsigned long long));
    int st = e == cudaSuccess ? SPMV_OK : cuda_status(e, "spmv_batch_create");
    if (st == SPMV_OK) st = build(b, (cudaStream_t)stream);
    if (st != SPMV_OK) {
        free_device(b);
        if (b->d_counter) cudaFree(b->d_counter);
        if (b->cs) cudaStreamDestroy(b->cs);
        delete b;
        return st;
    }
    *out = b;
    return SPMV_OK;
}

int spmv_batch_launch(spmv_batch_handle b, void *stream) {
    entry_reset();
    if (!b) {
        set_error("spmv_batch_launch: NULL batch");
        return SPMV_ERR_INVALID;
    }
    SPMV_CUDA_TRY(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
    return SPMV_OK;
}

int spmv_batch_tune(spmv_batch_handle b, void *stream) {
    entry_reset();
    if (!b) {
        set_error("spmv_batch_tune: NULL batch");
        return SPMV_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int cand[9] = {BATCH_COO, BATCH_BSR, 0, 1, 2, 4, 8, 16, 32};
    // 1) per matrix: time each mode on a one-matrix sub-batch
    for (int i = 0; i < b->count; ++i) {
        const spmv_matrix *h = b->hs[i];
        if (h->m == 0) continue;
        {
            BatchMat probe{};
            describe_format(h, probe);
            if (probe.fmt != SPMV_FMT_CSR) continue;  // ELL and SELL matrices keep their own kernel bodies
        }
        int best_mode = b->modes[i];
        float best_t = 1e30f;
        BatchMat probe{};
        describe_format(h, probe);
        for (int mode : cand) {
            if ((mode == 0 || mode == BATCH_COO) && h->nnz == 0) continue;
            if (mode == BATCH_COO && !probe.coo_rows) continue;
            if (mode == BATCH_BSR && (!probe.bsr_rowptr || h->nnz == 0)) continue;
            b->modes[i] = mode;
            spmv_batch one;  // a view of matrix i only (shares the counter, no graph)
            one.count = 1;
            one.vt = b->vt;
            one.items = b->items;
            one.tpb = b->tpb;
            one.group = 1;
            one.sm_count = b->sm_count;
            one.hs = {b->hs[i]};
            one.alpha = {b->alpha[i]};
            one.beta = {b->beta[i]};
            one.x = {b->x[i]};
            one.y = {b->y[i]};
            one.modes = {mode};
            one.d_counter = b->d_counter;
            one.cs = b->cs;
            // build descriptors without capturing a graph
            const int C = 32 * one.items;
            BatchMat M{};
            M.rowptr = h->rowptr;
            M.colidx = h->colidx;
            M.vals = h->vals;
            M.x = b->x[i];
            M.y = b->y[i];
            M.alpha = b->alpha[i];
            M.beta = b->beta[i];
            M.m = h->m;
            M.nnz = h->nnz;
            M.mode = mode;
            M.wide = wide_groups(h, mode);
            M.fmt = mode == BATCH_BSR ? SPMV_FMT_BSR : SPMV_FMT_CSR;
            M.coo_rows = probe.coo_rows;
            M.bsr_rowptr = probe.bsr_rowptr;
            M.bsr_col = probe.bsr_col;
            M.bsr_val = probe.bsr_val;
            M.bsr_mb = probe.bsr_mb;
            M.bsr_r = probe.bsr_r;
            M.n = h->n;
            // the mode is timed on k copies of the matrix in one launch (about
            // 4M entries in all), so that a small matrix is timed at the
            // throughput the full batch sees rather than at one launch's
            // latency; the copies write the same y (timing only)
            const int64_t per = batch_items(M, C);
            const int64_t k = std::max<int64_t>(1, std::min<int64_t>(256, (int64_t(4) << 20) /
                                                                              std::max<int64_t>(1, h->nnz + h->m)));
            int32_t *meta = nullptr;
            BatchMat *d_m = nullptr;
            int64_t *d_off = nullptr;
            int st = SPMV_OK;
            if (mode == 0 || mode == BATCH_COO) {
                st = build_chunk_meta(h, mode, C, &meta, s);
                if (st == SPMV_OK) set_chunk_meta(M, meta, C);
                if (st == SPMV_OK) st = alloc_partials(&one.part, k * per, 1, one.vt, s);
            }
            M.units = per;
            std::vector<BatchMat> copies((size_t)k, M);
            std::vector<int64_t> offs((size_t)k + 1);
            for (int64_t r = 0; r <= k; ++r) offs[r] = r * per;
            for (int64_t r = 0; r < k; ++r) copies[r].part_off = mode == 0 || mode == BATCH_COO ? r * per : 0;
            one.count = (int)k;
            if (st == SPMV_OK && (dev_malloc((void **)&d_m, sizeof(BatchMat) * k) != cudaSuccess ||
                                  dev_malloc((void **)&d_off, sizeof(int64_t) * (k + 1)) != cudaSuccess))
                st = SPMV_ERR_OOM;
            if (st == SPMV_OK) {
                cudaMemcpyAsync(d_m, copies.data(), sizeof(BatchMat) * k, cudaMemcpyHostToDevice, s);
                cudaMemcpyAsync(d_off, offs.data(), sizeof(int64_t) * (k + 1), cudaMemcpyHostToDevice, s);
                const float t = time_launch(&one, d_m, (int)k, d_off, k * per, s, 3, &st);
                if (st == SPMV_OK && t < best_t) {
                    best_t = t;
                    best_mode = mode;
                }
            }
            free_partials(&one.part);
            if (meta) cudaFree(meta);
            if (d_m) cudaFree(d_m);
            if (d_off) cudaFree(d_off);
            one.d_counter = nullptr;
            one.cs = nullptr;
            if (st != SPMV_OK) return st;
        }
        b->modes[i] = best_mode;
    }
    // 2) batch-wide: chunk size and block size on the whole batch
    int best_items = b->items, best_tpb = b->tpb, best_group = b->group;
    float best_t = 1e30f;
    for (int group : {1, 4}) {
        for (int items : {4, 8, 16}) {
            for (int tpb : {128, 256, 512}) {
                b->items = items;
                b->tpb = tpb;
                b->group = group;
                SPMV_TRY(build(b, s));
                int st = SPMV_OK;
                const float t = time_launch(b, (const BatchMat *)b->d_mats, b->count, b->d_item_off,
                                            b->total_items, s, 5, &st);
                SPMV_TRY(st);
                if (t < best_t) {
                    best_t = t;
                    best_items = items;
                    best_tpb = tpb;
                    best_group = group;
                }
            }
        }
    }
    b->items = best_items;
    b->tpb = best_tpb;
    b->group = best_group;
    return build(b, s);
}

int spmv_batch_get_plan(spmv_batch_handle b, int32_t *h_modes, int32_t *items, int32_t *threads_per_block) {
    if (!b) {
        set_error("spmv_batch_get_plan: NULL batch");
        return SPMV_ERR_INVALID;
    }
    if (h_modes)
        for (int i = 0; i < b->count; ++i) h_modes[i] = b->modes[i];
    if (items) *items = b->items;
    if (threads_per_block) *threads_per_block = b->tpb;
    return SPMV_OK;
}

int spmv_batch_destroy(spmv_batch_handle b) {
    if (!b) return SPMV_OK;
    if (b->cs) cudaStreamSynchronize(b->cs);
    free_device(b);
    if (b->d_counter) cudaFree(b->d_counter);
    if (b->cs) cudaStreamDestroy(b->cs);
    delete b;
    return SPMV_OK;
}

int spmv_batch_run(const spmv_handle *hs, int32_t count, const double *alpha, const void *const *d_x,
                   const double *beta, void *const *d_y, void *stream) {
    spmv_batch_handle b = nullptr;
    SPMV_TRY(spmv_batch_create(&b, hs, count, alpha, d_x, beta, d_y, stream));
    int st = spmv_batch_launch(b, stream);
    if (st == SPMV_OK) {
        cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
        if (e != cudaSuccess) st = cuda_status(e, "spmv_batch_run");
    }
    spmv_batch_destroy(b);
    return st;
}

}  // extern "C"

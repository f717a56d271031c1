// C ABI of the SpMV engine (include/spmv.h): handle life cycle, format
// selection, and dispatch of y = alpha*A*x + beta*y to the kernel families.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>

#include "bulk.cuh"
#include "internal.cuh"

namespace spmv {

namespace {
thread_local char g_err[512] = "";
thread_local long long g_alloc_count = 0;

// SPMV_FAULT_ALLOC=k (k >= 1): the k-th allocation of each entry-point call
// fails; read on every allocation so a test can set and clear it at will
bool fault_injected() {
    const char *v = std::getenv("SPMV_FAULT_ALLOC");
    ++g_alloc_count;
    if (!v || !*v) return false;
    const long long k = std::atoll(v);
    return k > 0 && g_alloc_count == k;
}
}  // namespace

void entry_reset() {
    g_err[0] = 0;
    g_alloc_count = 0;
}

cudaError_t dev_malloc(void **p, size_t bytes) {
    if (fault_injected()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

cudaError_t dev_malloc_async(void **p, size_t bytes, cudaStream_t s) {
    if (fault_injected()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMallocAsync(p, bytes, s);
}

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}

int cuda_status(cudaError_t e, const char *what) {
    set_error("%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();  // clear the sticky-free allocation error
        return SPMV_ERR_OOM;
    }
    return SPMV_ERR_CUDA;
}

namespace {
std::mutex g_attr_mu;
std::map<std::pair<const void *, int>, int> g_occ;
std::map<std::pair<const void *, int>, int> g_carve;  // (kernel, device): function attributes are per device
}  // namespace

int resident_blocks(const void *kernel, int threads) {
    std::lock_guard<std::mutex> lk(g_attr_mu);
    int dev = 0;
    cudaGetDevice(&dev);
    auto key = std::make_pair(kernel, threads * 64 + dev);
    auto it = g_occ.find(key);
    if (it != g_occ.end()) return it->second;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, 0) != cudaSuccess || nb < 1) {
        cudaGetLastError();
        nb = 1;
    }
    g_occ[key] = nb;
    return nb;
}

int apply_carveout(const void *kernel, int carveout) {
    std::lock_guard<std::mutex> lk(g_attr_mu);
    int dev = 0;
    cudaGetDevice(&dev);
    const auto key = std::make_pair(kernel, dev);
    auto it = g_carve.find(key);
    const int current = it == g_carve.end() ? -1 : it->second;
    if (current == carveout) return SPMV_OK;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         carveout < 0 ? (int)cudaSharedmemCarveoutDefault : carveout);
    if (e != cudaSuccess) return cuda_status(e, "cudaFuncSetAttribute(carveout)");
    g_carve[key] = carveout;
    // resident block counts of this kernel on this device may change with the carveout
    for (auto i = g_occ.begin(); i != g_occ.end();) {
        if (i->first.first == kernel && i->first.second % 64 == dev) i = g_occ.erase(i);
        else ++i;
    }
    return SPMV_OK;
}

// default threads per row: the largest power of two (1..32) that leaves each
// lane at least eight entries of a mean-length row, so lanes accumulate
// sequentially and the cross-lane adds (costly in fp64 on this GPU) are few
int default_tpr(const spmv_matrix *h) {
    const double q = h->m ? (double)h->nnz / (double)h->m / 8.0 : 1.0;
    int t = 1;
    while (t < 32 && 2.0 * t <= q) t *= 2;
    return t;
}

namespace {

bool pow2_in(int v, int lo, int hi) { return v >= lo && v <= hi && (v & (v - 1)) == 0; }

// Loads in flight per lane when the configuration leaves unroll at 0.  ELL
// and HYB with fp64 values keep two (a group of four fp64 loads needs more
// registers than the 32-register variant has, and the loads then wait on
// each other); fp32/bf16 keep four; SELL keeps eight with 64 registers, one
// for fp64 values in the column-major layout (measured with the L2 flushed by
// reading, fp64: R-MAT scale 20 74.8 against 76.8 us at 512 threads per
// block, Poisson(16) rows 78.5 against 80.2).  Chunked kernels (COO, HYB
// tail, split CSR) take 4 x unroll entries a lane.
int default_unroll(int format, int vt, int sell_groups) {
    if (format == SPMV_FMT_SELL) return vt == SPMV_F64 && sell_groups == 1 ? 1 : 8;
    if (format == SPMV_FMT_ELL || format == SPMV_FMT_HYB) return vt == SPMV_F64 ? 2 : 4;
    return 2;
}

// Register cap when the configuration leaves regcap at 0: fp64 ELL and HYB
// run the 32-register variant (two 1024-thread blocks per SM); fp32/bf16 ELL
// and HYB (two rows per thread, twice the loads in flight) and the other
// formats 64.
int default_regcap(int format, int vt) {
    return (format == SPMV_FMT_ELL || format == SPMV_FMT_HYB) && vt == SPMV_F64 ? 32 : 64;
}

// Fills defaults and validates; returns SPMV_ERR_INVALID on a bad field.
int resolve_config(const spmv_matrix *h, const spmv_config *in, spmv_config *out) {
    spmv_config c;
    spmv_config_default(&c, SPMV_FMT_CSR);
    if (in) c = *in;
    if (c.threads_per_block == 0) c.threads_per_block = 256;
    if (c.regcap == 0) c.regcap = default_regcap(c.format, h->vt);
    if (c.bsr_block == 0) {
        // SELL: groups of four columns unless the rows follow a power law
        // (a longest row beyond 32 mean rows: there most slices are a few
        // columns wide and column-major runs faster) or, with fp64 values,
        // their columns are scattered (under a quarter of consecutive
        // entries with consecutive columns: column-major was 1-5.6% faster
        // on every fp64 Poisson-row matrix over 30 us of the held-out set,
        // grouped faster on stencils and bands); BSR: 4 x 4 blocks
        const double mean = h->m > 0 ? (double)h->nnz / (double)h->m : 0.0;
        const bool colmajor = (double)h->max_row > 32.0 * mean + 32.0 || (h->vt == SPMV_F64 && h->contig < 0.25);
        c.bsr_block = c.format == SPMV_FMT_SELL && colmajor ? 1 : 4;
        // CSR vector with one or two lanes per row: 8-entry groups (32-byte
        // loads) once a lane's part of a mean row holds 16 or more entries,
        // else 4 (fewer masked slots: shorter rows); set below with the
        // lanes per row
        if (c.format == SPMV_FMT_CSR) c.bsr_block = 0;
    }
    if (c.format < SPMV_FMT_CSR || c.format > SPMV_FMT_SELL) {
        set_error("config: unknown format %d", c.format);
        return SPMV_ERR_INVALID;
    }
    if (c.unroll == 0) c.unroll = default_unroll(c.format, h->vt, c.bsr_block);
    if (!pow2_in(c.threads_per_block, 32, 1024)) {
        set_error("config: threads_per_block %d is not a power of two in [32, 1024]", c.threads_per_block);
        return SPMV_ERR_INVALID;
    }
    const bool ell_family = c.format == SPMV_FMT_ELL || c.format == SPMV_FMT_HYB || c.format == SPMV_FMT_SELL;
    if (c.unroll != 1 && c.unroll != 2 && c.unroll != 4 && !(c.unroll == 8 && ell_family)) {
        set_error("config: unroll %d not in {1, 2, 4} (8 also for ELL, HYB, SELL)", c.unroll);
        return SPMV_ERR_INVALID;
    }
    if (c.regcap != 32 && c.regcap != 64 && !(c.regcap == 48 && ell_family)) {
        set_error("config: regcap %d not in {32, 64} (48 also for ELL, HYB, SELL)", c.regcap);
        return SPMV_ERR_INVALID;
    }
    if (c.carveout < -1 || c.carveout > 100) {
        set_error("config: carveout %d not in [-1, 100]", c.carveout);
        return SPMV_ERR_INVALID;
    }
    if (c.format == SPMV_FMT_SELL   ? (c.bsr_block != 1 && c.bsr_block != 4)
        : c.format == SPMV_FMT_CSR  ? (c.bsr_block != 0 && c.bsr_block != 4 && c.bsr_block != 8)
                                    : (c.bsr_block != 2 && c.bsr_block != 4)) {
        set_error("config: bsr_block %d not in {2, 4} ({1, 4} for SELL column groups, {4, 8} for CSR load groups)",
                  c.bsr_block);
        return SPMV_ERR_INVALID;
    }
    if (c.hyb_ell_width < 0) {
        set_error("config: negative hyb_ell_width");
        return SPMV_ERR_INVALID;
    }
    if (c.format == SPMV_FMT_SELL) {  // SELL: columns of a slice per work item
        // 128 balances warps best on power-law rows (R-MAT scale 20, fp64:
        // 80.6 us at 128, 86.7 at 256, 95.9 at 64, 197 at 1024)
        if (c.hyb_ell_width == 0) c.hyb_ell_width = 128;
        if (c.hyb_ell_width < 8 || c.hyb_ell_width > 65536 || c.hyb_ell_width % 4 != 0) {
            set_error("config: SELL columns per work item %d not a multiple of 4 in [8, 65536]", c.hyb_ell_width);
            return SPMV_ERR_INVALID;
        }
    }
    switch (c.format) {
    case SPMV_FMT_CSR:
        if (c.threads_per_row == 0) c.threads_per_row = default_tpr(h);
        if (c.bsr_block == 0) {
            const double mean = h->m > 0 ? (double)h->nnz / (double)h->m : 0.0;
            c.bsr_block = c.threads_per_row >= 1 && mean / c.threads_per_row >= 16.0 ? 8 : 4;
        }
        if (c.threads_per_row != SPMV_TPR_SPLIT && !pow2_in(c.threads_per_row, 1, 32)) {
            set_error("config: CSR threads_per_row %d not in {1..32 powers of two, -1}", c.threads_per_row);
            return SPMV_ERR_INVALID;
        }
        if (c.threads_per_row == SPMV_TPR_SPLIT) {  // 0: warp chunks; else nonzeros per staged tile
            if (c.hyb_ell_width != 0 &&
                (c.hyb_ell_width < 256 || c.hyb_ell_width > 8192 || c.hyb_ell_width % 256 != 0)) {
                set_error("config: CSR tile size %d not 0 or a multiple of 256 in [256, 8192]", c.hyb_ell_width);
                return SPMV_ERR_INVALID;
            }
        }
        break;
    case SPMV_FMT_BSR:
        if (c.threads_per_row == 0) c.threads_per_row = 1;
        if (!pow2_in(c.threads_per_row, 1, 8)) {
            set_error("config: BSR blocks per row group %d not in {1, 2, 4, 8}", c.threads_per_row);
            return SPMV_ERR_INVALID;
        }
        break;
    default:
        if (c.threads_per_row != 0 && c.threads_per_row != 1) {
            set_error("config: threads_per_row must be 0 or 1 for ELL, COO, HYB and SELL");
            return SPMV_ERR_INVALID;
        }
        c.threads_per_row = 1;
        break;
    }
    *out = c;
    return SPMV_OK;
}

int runner(const spmv_matrix *h, int kind, double alpha, const void *x, double beta, void *y, cudaStream_t s) {
    switch (h->vt) {
    case SPMV_F64: return run_kernels_f64(kind, h, alpha, x, beta, y, s);
    case SPMV_F32: return run_kernels_f32(kind, h, alpha, x, beta, y, s);
    default: return run_kernels_bf16(kind, h, alpha, x, beta, y, s);
    }
}

void destroy_all(spmv_matrix *h) {
    free_cg(h);
    for (int p = 0; p < h->npanels; ++p)
        if (h->panels[p]) {
            destroy_all(h->panels[p]);
            delete h->panels[p];
        }
    delete[] h->panels;
    delete[] h->panel_row0;
    h->panels = nullptr;
    h->panel_row0 = nullptr;
    h->npanels = 0;
    free_packed(h);
    if (h->d_status) cudaFree(h->d_status);
    h->d_status = nullptr;
    if (h->rowptr) cudaFree(h->rowptr);
    if (h->colidx) cudaFree(h->colidx);
    if (h->vals) cudaFree(h->vals);
    h->rowptr = h->colidx = nullptr;
    h->vals = nullptr;
}

}  // namespace

int run_product(const spmv_matrix *h, double alpha, const void *x, double beta, void *y, cudaStream_t s) {
    if (h->npanels > 0) {  // each panel writes its own rows of y
        for (int p = 0; p < h->npanels; ++p)
            SPMV_TRY(run_product(h->panels[p], alpha, x, beta,
                                 static_cast<char *>(y) + vec_size(h->vt) * (size_t)h->panel_row0[p], s));
        return SPMV_OK;
    }
    if (h->nnz == 0) return runner(h, RUN_SCALE, alpha, x, beta, y, s);
    switch (h->cfg.format) {
    case SPMV_FMT_CSR:
        return runner(h, h->cfg.threads_per_row == SPMV_TPR_SPLIT ? RUN_CSR_SPLIT : RUN_CSR_VECTOR, alpha, x, beta, y,
                      s);
    case SPMV_FMT_ELL: return runner(h, RUN_ELL, alpha, x, beta, y, s);
    case SPMV_FMT_COO: return runner(h, RUN_COO, alpha, x, beta, y, s);
    case SPMV_FMT_HYB: return runner(h, RUN_HYB, alpha, x, beta, y, s);
    case SPMV_FMT_BSR: return runner(h, RUN_BSR, alpha, x, beta, y, s);
    case SPMV_FMT_SELL: return runner(h, RUN_SELL, alpha, x, beta, y, s);
    }
    set_error("spmv_run: bad format");
    return SPMV_ERR_INVALID;
}

namespace {
std::atomic<int64_t> g_panel_limit{SPMV_PANEL_LIMIT_MAX};

// a handle over row panels: sub-handles built from the stably gathered
// triplets of each panel's rows, so duplicates still sum in triplet order
int create_panelled(spmv_handle *out, int64_t m, int64_t n, int64_t nnz, const int32_t *d_rows,
                    const int32_t *d_cols, const void *d_vals, int32_t vt, const spmv_config *cfg,
                    cudaStream_t s, int64_t limit) {
    SPMV_TRY(check_triplet_bounds(d_rows, d_cols, nnz, m, n, s));
    std::vector<int64_t> bounds;
    SPMV_TRY(plan_panels(d_rows, nnz, m, limit, s, &bounds));
    spmv_matrix *h = new (std::nothrow) spmv_matrix();
    if (!h) {
        set_error("spmv_create: host allocation failed");
        return SPMV_ERR_OOM;
    }
    const int np = (int)bounds.size() - 1;
    h->m = m;
    h->n = n;
    h->vt = vt;
    h->panels = new (std::nothrow) spmv_matrix *[np]();
    h->panel_row0 = new (std::nothrow) int64_t[np + 1];
    if (!h->panels || !h->panel_row0) {
        delete[] h->panels;
        delete[] h->panel_row0;
        delete h;
        set_error("spmv_create: host allocation failed");
        return SPMV_ERR_OOM;
    }
    h->npanels = np;
    for (int p = 0; p <= np; ++p) h->panel_row0[p] = bounds[p];
    int st = SPMV_OK;
    for (int p = 0; p < np && st == SPMV_OK; ++p) {
        int32_t *pr = nullptr, *pc = nullptr;
        void *pv = nullptr;
        int64_t cnt = 0;
        st = gather_panel(d_rows, d_cols, d_vals, value_size(vt), nnz, bounds[p], bounds[p + 1], &pr, &pc, &pv,
                          &cnt, s);
        if (st == SPMV_OK)
            st = spmv_create(&h->panels[p], bounds[p + 1] - bounds[p], n, cnt, pr, pc, pv, vt, cfg, (void *)s);
        cudaFree(pr);
        cudaFree(pc);
        cudaFree(pv);
        if (st == SPMV_OK) {
            h->nnz += h->panels[p]->nnz;
            h->max_row = std::max(h->max_row, h->panels[p]->max_row);
            h->sm_count = h->panels[p]->sm_count;
        }
    }
    if (st != SPMV_OK) {
        destroy_all(h);
        delete h;
        return st;
    }
    h->cfg = h->panels[0]->cfg;
    h->packed = true;
    *out = h;
    return SPMV_OK;
}
}  // namespace

}  // namespace spmv

using namespace spmv;

extern "C" {

void spmv_config_default(spmv_config *cfg, int32_t format) {
    if (!cfg) return;
    cfg->format = format;
    cfg->threads_per_block = 256;
    cfg->threads_per_row = 0;
    cfg->unroll = 0;  // per format and value type, resolved when applied
    cfg->regcap = 0;
    cfg->carveout = -1;
    // SELL column groups and CSR load groups chosen per matrix
    cfg->bsr_block = format == SPMV_FMT_SELL || format == SPMV_FMT_CSR ? 0 : 4;
    cfg->hyb_ell_width = 0;
}

const char *spmv_last_error(void) { return g_err; }

int spmv_set_panel_limit(int64_t max_triplets) {
    if (max_triplets < 1 || max_triplets > SPMV_PANEL_LIMIT_MAX) {
        set_error("spmv_set_panel_limit: %lld not in [1, 2^31 - 2^20]", (long long)max_triplets);
        return SPMV_ERR_INVALID;
    }
    g_panel_limit.store(max_triplets);
    return SPMV_OK;
}

int64_t spmv_get_panel_limit(void) { return g_panel_limit.load(); }

int spmv_create(spmv_handle *out, int64_t m, int64_t n, int64_t nnz, const int32_t *d_rows, const int32_t *d_cols,
                const void *d_vals, int32_t value_type, const spmv_config *cfg, void *stream) {
    entry_reset();
    if (!out) {
        set_error("spmv_create: NULL output handle");
        return SPMV_ERR_INVALID;
    }
    *out = nullptr;
    if (m < 0 || n < 0 || nnz < 0) {
        set_error("spmv_create: negative size");
        return SPMV_ERR_INVALID;
    }
    if (value_type != SPMV_F64 && value_type != SPMV_F32 && value_type != SPMV_BF16) {
        set_error("spmv_create: unknown value type %d", value_type);
        return SPMV_ERR_INVALID;
    }
    if (nnz > 0 && (!d_rows || !d_cols || !d_vals)) {
        set_error("spmv_create: NULL triplet array with nnz > 0");
        return SPMV_ERR_INVALID;
    }
    if (m >= (int64_t(1) << 31) || n >= (int64_t(1) << 31)) {
        set_error("spmv_create: m and n must be below 2^31");
        return SPMV_ERR_UNSUPPORTED;
    }
    if (nnz > 0 && (m == 0 || n == 0)) {
        set_error("spmv_create: nonzeros in an empty matrix");
        return SPMV_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t limit = g_panel_limit.load();
    if (nnz > limit) return create_panelled(out, m, n, nnz, d_rows, d_cols, d_vals, value_type, cfg, s, limit);
    spmv_matrix *h = new (std::nothrow) spmv_matrix();
    if (!h) {
        set_error("spmv_create: host allocation failed");
        return SPMV_ERR_OOM;
    }
    h->m = m;
    h->n = n;
    h->nnz = nnz;
    h->vt = value_type;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = dev_malloc(reinterpret_cast<void **>(&h->d_status), sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_status, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) {
        int st = cuda_status(e, "device query");
        if (h->d_status) cudaFree(h->d_status);
        delete h;
        return st;
    }
    int st = build_csr(h, d_rows, d_cols, d_vals, s);
    spmv_config rc;
    if (st == SPMV_OK) st = resolve_config(h, cfg, &rc);
    if (st == SPMV_OK) st = pack_format(h, rc, s);
    if (st != SPMV_OK) {
        destroy_all(h);
        delete h;
        return st;
    }
    *out = h;
    return SPMV_OK;
}

int spmv_set_config(spmv_handle h, const spmv_config *cfg, void *stream) {
    entry_reset();
    if (!h) {
        set_error("spmv_set_config: NULL handle");
        return SPMV_ERR_INVALID;
    }
    spmv_config rc;
    SPMV_TRY(resolve_config(h, cfg, &rc));
    if (h->npanels > 0) {
        // every panel takes the configuration, or every panel falls back to CSR
        free_cg(h);
        int st = SPMV_OK;
        for (int p = 0; p < h->npanels && st == SPMV_OK; ++p) st = spmv_set_config(h->panels[p], cfg, stream);
        if (st != SPMV_OK) {
            char saved[512];
            std::strncpy(saved, g_err, sizeof saved);
            saved[sizeof saved - 1] = 0;
            spmv_config csr;
            spmv_config_default(&csr, SPMV_FMT_CSR);
            for (int p = 0; p < h->npanels; ++p) spmv_set_config(h->panels[p], &csr, stream);
            std::strncpy(g_err, saved, sizeof g_err);
        }
        h->cfg = h->panels[0]->cfg;
        return st;
    }
    int st = pack_format(h, rc, (cudaStream_t)stream);
    if (st != SPMV_OK) {
        // leave a usable handle: fall back to plain CSR
        spmv_config csr;
        spmv_config_default(&csr, SPMV_FMT_CSR);
        spmv_config rcsr;
        if (resolve_config(h, &csr, &rcsr) == SPMV_OK) {
            char saved[512];
            std::strncpy(saved, g_err, sizeof saved);
            saved[sizeof saved - 1] = 0;
            pack_format(h, rcsr, (cudaStream_t)stream);
            std::strncpy(g_err, saved, sizeof g_err);
        }
    }
    return st;
}

int spmv_get_config(spmv_handle h, spmv_config *out) {
    if (!h || !out) {
        set_error("spmv_get_config: NULL argument");
        return SPMV_ERR_INVALID;
    }
    *out = h->cfg;
    return SPMV_OK;
}

int spmv_get_info(spmv_handle h, spmv_info *out) {
    if (!h || !out) {
        set_error("spmv_get_info: NULL argument");
        return SPMV_ERR_INVALID;
    }
    std::memset(out, 0, sizeof *out);
    if (h->npanels > 0) {  // sums over the panels (widths: the largest)
        for (int p = 0; p < h->npanels; ++p) {
            spmv_info pi;
            SPMV_TRY(spmv_get_info(h->panels[p], &pi));
            out->ell_width = std::max(out->ell_width, pi.ell_width);
            out->hyb_coo_nnz += pi.hyb_coo_nnz;
            out->bsr_blocks += pi.bsr_blocks;
            out->sell_slots += pi.sell_slots;
            out->format_bytes += pi.format_bytes;
        }
        out->m = h->m;
        out->n = h->n;
        out->nnz = h->nnz;
        out->max_row = h->max_row;
        out->value_type = h->vt;
        out->format = h->cfg.format;
        out->panels = h->npanels;
        return SPMV_OK;
    }
    out->m = h->m;
    out->n = h->n;
    out->nnz = h->nnz;
    out->max_row = h->max_row;
    out->value_type = h->vt;
    out->format = h->cfg.format;
    out->panels = 1;
    const int64_t vs = (int64_t)value_size(h->vt);
    switch (h->cfg.format) {
    case SPMV_FMT_CSR:
        out->format_bytes = h->nnz * (vs + 4) + 4 * (h->m + 1);
        break;
    case SPMV_FMT_ELL:
        out->ell_width = h->ell_width;
        out->format_bytes = h->ell_width * h->ell_pitch * (vs + (h->ell_d16 ? 2 : 4));
        break;
    case SPMV_FMT_COO:
        out->format_bytes = h->nnz * (vs + 8);
        break;
    case SPMV_FMT_HYB:
        out->ell_width = h->ell_width;
        out->hyb_coo_nnz = h->hyb_nnz;
        out->format_bytes = h->ell_width * h->ell_pitch * (vs + (h->ell_d16 ? 2 : 4)) + h->hyb_nnz * (vs + 8);
        break;
    case SPMV_FMT_BSR:
        out->bsr_blocks = h->bsr_blocks;
        out->format_bytes = h->bsr_blocks * (vs * h->bsr_r * h->bsr_r + 4) + 4 * (h->bsr_mb + 1);
        break;
    case SPMV_FMT_SELL:
        out->sell_slots = h->sell_slots;
        out->format_bytes = h->sell_slots * (vs + 4) + 4 * (h->sell_nslices + 1) + 4 * h->m;
        break;
    }
    return SPMV_OK;
}

int spmv_run(spmv_handle h, double alpha, const void *d_x, double beta, void *d_y, void *stream) {
    if (!h) {
        set_error("spmv_run: NULL handle");
        return SPMV_ERR_INVALID;
    }
    if ((h->m > 0 && !d_y) || (h->n > 0 && h->nnz > 0 && !d_x)) {
        set_error("spmv_run: NULL vector");
        return SPMV_ERR_INVALID;
    }
    if (h->m == 0) return SPMV_OK;
    if (checked_mode()) {  // debug mode: verify the stored indices first (checked.cu)
        const int parts = h->npanels > 0 ? h->npanels : 1;
        for (int p = 0; p < parts; ++p)
            SPMV_TRY(check_indices(h->npanels > 0 ? h->panels[p] : h, (cudaStream_t)stream));
    }
    return run_product(h, alpha, d_x, beta, d_y, (cudaStream_t)stream);
}

namespace {
int array_of(spmv_handle h, int32_t id, const void **ptr, int64_t *bytes) {
    if (h->npanels > 0) {
        set_error("spmv_export: the matrix is held in %d row panels; arrays are per panel", h->npanels);
        return SPMV_ERR_UNSUPPORTED;
    }
    const int64_t vs = (int64_t)value_size(h->vt);
    const bool hyb = h->cfg.format == SPMV_FMT_HYB;
    *ptr = nullptr;
    *bytes = 0;
    switch (id) {
    case SPMV_ARR_CSR_ROWPTR: *ptr = h->rowptr; *bytes = 4 * (h->m + 1); break;
    case SPMV_ARR_CSR_COLIDX: *ptr = h->colidx; *bytes = 4 * h->nnz; break;
    case SPMV_ARR_CSR_VALS: *ptr = h->vals; *bytes = vs * h->nnz; break;
    case SPMV_ARR_ELL_COLIDX:
        if (h->ell_col || h->ell_d16) { *ptr = h->ell_col; *bytes = 4 * h->ell_width * h->ell_pitch; }
        break;
    case SPMV_ARR_ELL_VALS:
        if (h->ell_val) { *ptr = h->ell_val; *bytes = vs * h->ell_width * h->ell_pitch; }
        break;
    case SPMV_ARR_COO_ROWS:
        if (hyb) { *ptr = h->hyb_rows; *bytes = 4 * h->hyb_nnz; }
        else if (h->coo_rows) { *ptr = h->coo_rows; *bytes = 4 * h->nnz; }
        break;
    case SPMV_ARR_COO_COLS:
        if (hyb) { *ptr = h->hyb_cols; *bytes = 4 * h->hyb_nnz; }
        else if (h->coo_rows) { *ptr = h->colidx; *bytes = 4 * h->nnz; }
        break;
    case SPMV_ARR_COO_VALS:
        if (hyb) { *ptr = h->hyb_vals; *bytes = vs * h->hyb_nnz; }
        else if (h->coo_rows) { *ptr = h->vals; *bytes = vs * h->nnz; }
        break;
    case SPMV_ARR_BSR_ROWPTR:
        if (h->bsr_rowptr) { *ptr = h->bsr_rowptr; *bytes = 4 * (h->bsr_mb + 1); }
        break;
    case SPMV_ARR_BSR_COLIDX:
        if (h->bsr_col) { *ptr = h->bsr_col; *bytes = 4 * h->bsr_blocks; }
        break;
    case SPMV_ARR_BSR_VALS:
        if (h->bsr_val) { *ptr = h->bsr_val; *bytes = vs * h->bsr_blocks * h->bsr_r * h->bsr_r; }
        break;
    case SPMV_ARR_ELL_PITCH: *bytes = h->ell_pitch; break;
    case SPMV_ARR_SELL_PTR:
        if (h->sell_ptr) { *ptr = h->sell_ptr; *bytes = 4 * (h->sell_nslices + 1); }
        break;
    case SPMV_ARR_SELL_COLIDX:
        if (h->sell_col) { *ptr = h->sell_col; *bytes = 4 * h->sell_slots; }
        break;
    case SPMV_ARR_SELL_VALS:
        if (h->sell_val) { *ptr = h->sell_val; *bytes = vs * h->sell_slots; }
        break;
    case SPMV_ARR_SELL_PERM:
        if (h->sell_perm) { *ptr = h->sell_perm; *bytes = 4 * h->m; }
        break;
    default:
        set_error("spmv_export: unknown array id %d", id);
        return SPMV_ERR_INVALID;
    }
    return SPMV_OK;
}
}  // namespace

int spmv_export_bytes(spmv_handle h, int32_t array_id, int64_t *bytes) {
    if (!h || !bytes) {
        set_error("spmv_export_bytes: NULL argument");
        return SPMV_ERR_INVALID;
    }
    const void *p;
    return array_of(h, array_id, &p, bytes);
}

int spmv_export(spmv_handle h, int32_t array_id, void *d_dst, int64_t bytes, void *stream) {
    if (!h) {
        set_error("spmv_export: NULL handle");
        return SPMV_ERR_INVALID;
    }
    if (array_id == SPMV_ARR_ELL_PITCH) {
        set_error("spmv_export: the pitch is a size query only");
        return SPMV_ERR_INVALID;
    }
    const void *p;
    int64_t have;
    SPMV_TRY(array_of(h, array_id, &p, &have));
    if (bytes != have) {
        set_error("spmv_export: %lld bytes requested, array holds %lld", (long long)bytes, (long long)have);
        return SPMV_ERR_INVALID;
    }
    if (have == 0) return SPMV_OK;
    if (!d_dst) {
        set_error("spmv_export: NULL destination");
        return SPMV_ERR_INVALID;
    }
    if (array_id == SPMV_ARR_ELL_COLIDX && h->ell_d16)  // 16-bit row offsets: export int32 columns
        return decode_ell_columns(h, static_cast<int32_t *>(d_dst), (cudaStream_t)stream);
    SPMV_CUDA_TRY(cudaMemcpyAsync(d_dst, p, (size_t)have, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return SPMV_OK;
}

int spmv_check(spmv_handle h, void *stream) {
    entry_reset();
    if (!h) {
        set_error("spmv_check: NULL handle");
        return SPMV_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    unsigned bits = 0;
    const int parts = h->npanels > 0 ? h->npanels : 1;
    for (int p = 0; p < parts; ++p) {
        spmv_matrix *q = h->npanels > 0 ? h->panels[p] : h;
        if (!q->d_status) continue;
        unsigned w = 0;
        SPMV_CUDA_TRY(cudaMemcpyAsync(&w, q->d_status, sizeof w, cudaMemcpyDeviceToHost, s));
        SPMV_CUDA_TRY(cudaStreamSynchronize(s));
        if (w) SPMV_CUDA_TRY(cudaMemsetAsync(q->d_status, 0, sizeof w, s));
        bits |= w;
    }
    SPMV_CUDA_TRY(cudaStreamSynchronize(s));
    if (bits & STATUS_BOUNDS) {
        set_error("spmv_check: a kernel found an index out of bounds and skipped the access");
        return SPMV_ERR_BOUNDS;
    }
    if (bits & STATUS_TIMEOUT) {
        set_error("spmv_check: a kernel gave up waiting for a copy; its product is incomplete");
        return SPMV_ERR_TIMEOUT;
    }
    return SPMV_OK;
}

int spmv_destroy(spmv_handle h) {
    if (!h) return SPMV_OK;
    destroy_all(h);  // cudaFree waits for work still using the arrays
    delete h;
    return SPMV_OK;
}

}  // extern "C"

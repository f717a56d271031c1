// COO SpMV that allocates no device memory.
//
// Some callers cannot allocate: code running inside another library's
// memory pool or callback, real-time or embedded code that must not call
// cudaMalloc after start-up, or a process whose allocator is already
// exhausted or fenced off.  spmv_coo_run_noalloc serves them: it runs the
// segmented-reduction COO kernel directly on the caller's sorted triplets,
// and keeps the kernel's per-chunk bookkeeping (chunk metadata, partial row
// sums, arrival counters and exchange slots) in one fixed device array
// compiled into the library instead of in allocated memory.
#include <mutex>

#include "launch.cuh"

namespace spmv {
namespace {

constexpr int NA_ITEMS = 8;                                // entries per lane
constexpr int64_t NA_CHUNK = 32 * NA_ITEMS;                // entries per chunk
constexpr int64_t NA_MAX_CHUNKS = SPMV_NOALLOC_MAX_NNZ / NA_CHUNK;
// per chunk: two int32 metadata words, two partial sums and an exchange
// slot (8 bytes each), one arrival counter; plus one validation word
constexpr size_t NA_BYTES = (size_t)NA_MAX_CHUNKS * (4 + 4 + 8 + 8 + 8 + 4) + 256;

// The scratch every GPU that loads this library holds until the process
// exits.  In host code this name is only a stand-in for the device object:
// its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

struct NaLayout {
    int32_t *meta0, *meta1;
    void *head, *tail;
    unsigned long long *xslot;
    uint32_t *count;
    unsigned *flag;
};

NaLayout layout_of(unsigned char *base) {
    NaLayout L;
    const size_t C = (size_t)NA_MAX_CHUNKS;
    L.meta0 = reinterpret_cast<int32_t *>(base);
    L.meta1 = reinterpret_cast<int32_t *>(base + 4 * C);
    L.head = base + 8 * C;
    L.tail = base + 16 * C;
    L.xslot = reinterpret_cast<unsigned long long *>(base + 24 * C);
    L.count = reinterpret_cast<uint32_t *>(base + 32 * C);
    L.flag = reinterpret_cast<unsigned *>(base + 36 * C);
    return L;
}

std::mutex g_na_mu;
void *g_na_addr[256] = {};

// Device address of the scratch on the current device, looked up once per
// device (the first call on a device does this set-up).  The address is kept
// for the life of the process: cudaDeviceReset on a device destroys the
// context that holds the array, so the entry point must not be used on a
// device after it has been reset.
int scratch_address(unsigned char **out) {
    int dev = 0;
    SPMV_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) {
        set_error("spmv_coo_run_noalloc: device ordinal %d out of range", dev);
        return SPMV_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress(noalloc scratch)");
        g_na_addr[dev] = p;
    }
    *out = static_cast<unsigned char *>(g_na_addr[dev]);
    return SPMV_OK;
}

// Checks the triplets (indices in range, rows nondecreasing), derives each
// chunk's metadata by binary search over the sorted rows (first chunk of
// the chunk's head row, last chunk of its tail row) and clears the arrival
// counters and exchange slots the kernel expects in their initial state.
__global__ void k_noalloc_prep(int64_t nnz, int64_t m, int64_t n, const int *rows, const int *cols,
                               int64_t nchunks, unsigned long long empty, NaLayout L) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned bad = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nnz; i += stride) {
        const int r = rows[i], c = cols[i];
        if (r < 0 || r >= m || c < 0 || c >= n) bad = 1;
        if (i + 1 < nnz && rows[i + 1] < r) bad = 1;
    }
    if (bad) atomicOr(L.flag, 1u);
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nchunks; c += stride) {
        const int64_t e0 = c * NA_CHUNK, e1 = e0 + NA_CHUNK < nnz ? e0 + NA_CHUNK : nnz;
        const int hrow = rows[e0], trow = rows[e1 - 1];
        int64_t lo = 0, hi = nnz;  // first entry with row >= hrow
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (rows[mid] < hrow) lo = mid + 1; else hi = mid;
        }
        L.meta0[c] = (int32_t)(lo / NA_CHUNK);
        lo = 0;
        hi = nnz;  // first entry with row > trow
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (rows[mid] <= trow) lo = mid + 1; else hi = mid;
        }
        L.meta1[c] = (int32_t)((lo - 1) / NA_CHUNK);
        L.count[c] = 0u;
        L.xslot[c] = empty;
    }
}

template <int VT>
int run_noalloc(int64_t m, int64_t n, int64_t nnz, const int32_t *rows, const int32_t *cols, const void *vals,
                double alpha, const void *x, double beta, void *y, cudaStream_t s) {
    using V = typename VT_<VT>::V;
    using T = typename VT_<VT>::T;
    int dev = 0, sms = 0;
    SPMV_CUDA_TRY(cudaGetDevice(&dev));
    SPMV_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (nnz == 0) {
        const int64_t blocks = (m + 255) / 256;
        k_scale_y<T><<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(m, (T *)y, (T)beta);
        SPMV_CUDA_TRY(cudaGetLastError());
        return SPMV_OK;
    }
    unsigned char *base = nullptr;
    SPMV_TRY(scratch_address(&base));
    const NaLayout L = layout_of(base);
    const int64_t nchunks = (nnz + NA_CHUNK - 1) / NA_CHUNK;
    SPMV_CUDA_TRY(cudaMemsetAsync(L.flag, 0, sizeof(unsigned), s));
    const unsigned long long empty = VT == SPMV_F64 ? XEnc<double>::EMPTY : XEnc<float>::EMPTY;
    const int64_t work = nnz > nchunks ? nnz : nchunks;
    const int64_t pblocks = (work + 255) / 256;
    k_noalloc_prep<<<(unsigned)(pblocks < 4096 ? pblocks : 4096), 256, 0, s>>>(nnz, m, n, rows, cols, nchunks,
                                                                               empty, L);
    SPMV_CUDA_TRY(cudaGetLastError());
    unsigned hflag = 0;
    SPMV_CUDA_TRY(cudaMemcpyAsync(&hflag, L.flag, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    SPMV_CUDA_TRY(cudaStreamSynchronize(s));
    if (hflag) {
        set_error("spmv_coo_run_noalloc: triplets must have rows in [0, m), columns in [0, n) and rows "
                  "in nondecreasing order");
        return SPMV_ERR_INVALID;
    }
    auto kern = k_coo_seg<V, T, NA_ITEMS, false>;
    const int tpb = 256;
    int per_sm = 0;  // queried directly each call: no host-side cache to grow
    SPMV_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, tpb, 0));
    const int64_t need = (nchunks + tpb / 32 - 1) / (tpb / 32);
    const int64_t cap = (int64_t)(per_sm > 0 ? per_sm : 1) * sms;
    const int grid = (int)(need < cap ? need : cap);
    PartialsT<T> P{(T *)L.head, (T *)L.tail, L.count, L.xslot, 1};
    kern<<<grid, tpb, 0, s>>>(nnz, m, rows, cols, (const V *)vals, (const T *)x, (T *)y, (T)alpha, (T)beta,
                              L.meta0, L.meta1, P);
    SPMV_CUDA_TRY(cudaGetLastError());
    return SPMV_OK;
}

}  // namespace
}  // namespace spmv

using namespace spmv;

extern "C" int spmv_coo_run_noalloc(int64_t m, int64_t n, int64_t nnz, const int32_t *d_rows, const int32_t *d_cols,
                                    const void *d_vals, int32_t value_type, double alpha, const void *d_x,
                                    double beta, void *d_y, void *stream) {
    if (m < 0 || n < 0 || nnz < 0) {
        set_error("spmv_coo_run_noalloc: negative size");
        return SPMV_ERR_INVALID;
    }
    if (value_type != SPMV_F64 && value_type != SPMV_F32 && value_type != SPMV_BF16) {
        set_error("spmv_coo_run_noalloc: unknown value type %d", value_type);
        return SPMV_ERR_INVALID;
    }
    if (nnz > SPMV_NOALLOC_MAX_NNZ) {
        set_error("spmv_coo_run_noalloc: nnz = %lld exceeds the fixed scratch limit of %lld entries",
                  (long long)nnz, (long long)SPMV_NOALLOC_MAX_NNZ);
        return SPMV_ERR_UNSUPPORTED;
    }
    if (m >= (int64_t(1) << 31) || n >= (int64_t(1) << 31)) {
        set_error("spmv_coo_run_noalloc: m and n must be below 2^31");
        return SPMV_ERR_UNSUPPORTED;
    }
    if (nnz > 0 && (!d_rows || !d_cols || !d_vals || !d_x)) {
        set_error("spmv_coo_run_noalloc: NULL triplet array or x with nnz > 0");
        return SPMV_ERR_INVALID;
    }
    if (nnz > 0 && (m == 0 || n == 0)) {
        set_error("spmv_coo_run_noalloc: nonzeros in an empty matrix");
        return SPMV_ERR_INVALID;
    }
    // the kernel reads whole chunks with 16-byte vector loads from the
    // caller's arrays, so their base addresses must be 16-byte aligned (a
    // view starting mid-array is refused here, before anything is launched)
    if (nnz > 0 && (((uintptr_t)d_rows | (uintptr_t)d_cols | (uintptr_t)d_vals) & 15u) != 0) {
        set_error("spmv_coo_run_noalloc: d_rows, d_cols and d_vals must be 16-byte aligned");
        return SPMV_ERR_INVALID;
    }
    if (m == 0) return SPMV_OK;
    if (!d_y) {
        set_error("spmv_coo_run_noalloc: NULL y");
        return SPMV_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    // every call with nonzeros waits on the stream to read its triplet
    // check, which a stream being captured into a graph does not allow
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    SPMV_CUDA_TRY(cudaStreamIsCapturing(s, &cap));
    if (cap != cudaStreamCaptureStatusNone) {
        set_error("spmv_coo_run_noalloc: the stream is being captured; this call synchronises it");
        return SPMV_ERR_UNSUPPORTED;
    }
    switch (value_type) {
    case SPMV_F64: return run_noalloc<SPMV_F64>(m, n, nnz, d_rows, d_cols, d_vals, alpha, d_x, beta, d_y, s);
    case SPMV_F32: return run_noalloc<SPMV_F32>(m, n, nnz, d_rows, d_cols, d_vals, alpha, d_x, beta, d_y, s);
    default: return run_noalloc<SPMV_BF16>(m, n, nnz, d_rows, d_cols, d_vals, alpha, d_x, beta, d_y, s);
    }
}

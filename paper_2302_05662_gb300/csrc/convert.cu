// Device-side format conversion: COO triplets -> CSR -> ELL / COO / HYB / BSR.
//
// The paper converts the input COO matrix to the chosen format on the CPU
// (Section 5.3 step 4; overhead in Section 7.5).  Here every step runs on
// the GPU: validation, a stable LSD radix sort on the (row, col) key,
// merging of duplicate pairs, the row-pointer array, and the packs of the
// other formats from CSR (Section 2.3 layouts).
#include <algorithm>
#include <vector>

#include "combine.cuh"

namespace spmv {

namespace {

constexpr unsigned FULL = 0xffffffffu;

// ---------------------------------------------------------------------------
// temporary device buffer, freed (stream-ordered) when it goes out of scope
// ---------------------------------------------------------------------------
template <typename T>
struct Tmp {
    T *p = nullptr;
    cudaStream_t s = nullptr;
    Tmp() = default;
    Tmp(const Tmp &) = delete;
    Tmp &operator=(const Tmp &) = delete;
    ~Tmp() { if (p) cudaFreeAsync(p, s); }
    int alloc(size_t count, cudaStream_t stream) {
        s = stream;
        cudaError_t e = dev_malloc_async(reinterpret_cast<void **>(&p),
                                        std::max<size_t>(count, 1) * sizeof(T), stream);
        if (e != cudaSuccess) { p = nullptr; return cuda_status(e, "dev_malloc_async(temp)"); }
        return SPMV_OK;
    }
};

template <typename T>
int dalloc(T **p, size_t count) {
    cudaError_t e = dev_malloc(reinterpret_cast<void **>(p), std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) { *p = nullptr; return cuda_status(e, "cudaMalloc"); }
    return SPMV_OK;
}
int dalloc_bytes(void **p, size_t bytes) {
    cudaError_t e = dev_malloc(p, std::max<size_t>(bytes, 1));
    if (e != cudaSuccess) { *p = nullptr; return cuda_status(e, "cudaMalloc"); }
    return SPMV_OK;
}

inline int bits_for(int64_t count) {  // bits to hold 0 .. count-1
    int b = 0;
    while ((int64_t(1) << b) < count) ++b;
    return b;
}
inline unsigned grid1d(int64_t work, int threads, int cap = 152 * 32) {
    int64_t g = (work + threads - 1) / threads;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, cap));
}

// ---------------------------------------------------------------------------
// validation: bit 0 = index out of range, bit 1 = not sorted by (row, col),
// bit 2 = a repeated (row, col) pair
// ---------------------------------------------------------------------------
__global__ void k_check_triplets(const int *rows, const int *cols, int64_t nnz, int64_t m,
                                 int64_t n, unsigned *flags) {
    unsigned f = 0;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nnz; i += stride) {
        int r = rows[i], c = cols[i];
        if (r < 0 || r >= m || c < 0 || c >= n) f |= 1u;
        if (i + 1 < nnz) {
            int r2 = rows[i + 1], c2 = cols[i + 1];
            if (r2 < r || (r2 == r && c2 < c)) f |= 2u;
            else if (r2 == r && c2 == c) f |= 4u;
        }
    }
    f = __reduce_or_sync(FULL, f);
    if ((threadIdx.x & 31) == 0 && f) atomicOr(flags, f);
}

// rowptr[r] = first position whose row is >= r, over rows sorted ascending
__global__ void k_rowptr_from_sorted(const int *rows, int64_t nnz, int64_t m, int *rowptr) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r <= m; r += stride) {
        int64_t lo = 0, hi = nnz;
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            if (rows[mid] < r) lo = mid + 1; else hi = mid;
        }
        rowptr[r] = (int)lo;
    }
}

// row of entry k: the r with rowptr[r] <= k < rowptr[r+1]
__device__ __forceinline__ int row_of(const int *rowptr, int64_t m, int64_t k) {
    int64_t lo = 0, hi = m;  // answer in [0, m-1]
    while (lo < hi) {
        int64_t mid = (lo + hi + 1) >> 1;
        if (rowptr[mid] <= k) lo = mid; else hi = mid - 1;
    }
    return (int)lo;
}

__global__ void k_expand_rows(const int *rowptr, int64_t m, int64_t nnz, int *rows) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += stride)
        rows[k] = row_of(rowptr, m, k);
}

__global__ void k_max_row(const int *rowptr, int64_t m, int *out) {
    int best = 0;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < m; r += stride)
        best = max(best, rowptr[r + 1] - rowptr[r]);
    best = __reduce_max_sync(FULL, best);
    if ((threadIdx.x & 31) == 0) atomicMax(out, best);
}

// consecutive stored entries whose columns are consecutive (col[k] ==
// col[k-1] + 1): the column contiguity of the rows (a pair across a row
// boundary can count too; the statistic only steers a layout default)
__global__ void k_contiguous_pairs(const int *colidx, int64_t nnz, unsigned long long *out) {
    unsigned long long cnt = 0;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x + 1; k < nnz; k += stride)
        cnt += colidx[k] == colidx[k - 1] + 1;
    cnt = __reduce_add_sync(FULL, (unsigned)cnt);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(out, cnt);
}

// ---------------------------------------------------------------------------
// exclusive scan of int32 (three passes: tile sums, scan of sums, tiles)
// ---------------------------------------------------------------------------
constexpr int SC_THREADS = 256, SC_ITEMS = 8, SC_TILE = SC_THREADS * SC_ITEMS;

__device__ __forceinline__ int block_exclusive_scan(int v, int *total) {
    __shared__ int warp_sums[SC_THREADS / 32];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        int t = __shfl_up_sync(FULL, incl, d);
        if (lane >= d) incl += t;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int w = lane < SC_THREADS / 32 ? warp_sums[lane] : 0;
        int wi = w;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            int t = __shfl_up_sync(FULL, wi, d);
            if (lane >= d) wi += t;
        }
        if (lane < SC_THREADS / 32) warp_sums[lane] = wi - w;
        if (lane == SC_THREADS / 32 - 1) *total = wi;
    }
    __syncthreads();
    int r = incl - v + warp_sums[warp];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(SC_THREADS) k_scan_reduce(const int *in, int64_t n, int *sums) {
    int64_t base = (int64_t)blockIdx.x * SC_TILE;
    int s = 0;
    for (int k = threadIdx.x; k < SC_TILE; k += SC_THREADS) {
        int64_t i = base + k;
        if (i < n) s += in[i];
    }
    s = __reduce_add_sync(FULL, s);
    __shared__ int ws[SC_THREADS / 32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < SC_THREADS / 32; ++w) t += ws[w];
        sums[blockIdx.x] = t;
    }
}

// single block: exclusive scan of nb tile sums in place
__global__ void __launch_bounds__(SC_THREADS) k_scan_sums(int *sums, int64_t nb) {
    __shared__ int carry_s;
    __shared__ int total_s;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    for (int64_t base = 0; base < nb; base += SC_THREADS) {
        int64_t i = base + threadIdx.x;
        int v = i < nb ? sums[i] : 0;
        int ex = block_exclusive_scan(v, &total_s);
        int carry = carry_s;
        if (i < nb) sums[i] = ex + carry;
        __syncthreads();
        if (threadIdx.x == 0) carry_s = carry + total_s;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(SC_THREADS) k_scan_down(const int *in, int *out, int64_t n,
                                                          const int *sums) {
    __shared__ int total_s;
    int64_t base = (int64_t)blockIdx.x * SC_TILE + (int64_t)threadIdx.x * SC_ITEMS;
    int v[SC_ITEMS];
    int t = 0;
#pragma unroll
    for (int j = 0; j < SC_ITEMS; ++j) {
        int64_t i = base + j;
        v[j] = i < n ? in[i] : 0;
        t += v[j];
    }
    int ex = block_exclusive_scan(t, &total_s) + sums[blockIdx.x];
#pragma unroll
    for (int j = 0; j < SC_ITEMS; ++j) {
        int64_t i = base + j;
        if (i < n) out[i] = ex;
        ex += v[j];
    }
}

// exclusive scan in -> out (may alias); returns the total through *total_host
// when non-null (synchronises the stream in that case)
int exclusive_scan(const int *in, int *out, int64_t n, cudaStream_t s, int64_t *total_host) {
    if (n <= 0) {
        if (total_host) *total_host = 0;
        return SPMV_OK;
    }
    int64_t nb = (n + SC_TILE - 1) / SC_TILE;
    Tmp<int> sums;
    SPMV_TRY(sums.alloc(nb + 1, s));
    k_scan_reduce<<<(unsigned)nb, SC_THREADS, 0, s>>>(in, n, sums.p);
    int last_in = 0;
    if (total_host) {
        SPMV_CUDA_TRY(cudaMemcpyAsync(&last_in, in + n - 1, sizeof(int), cudaMemcpyDeviceToHost, s));
    }
    k_scan_sums<<<1, SC_THREADS, 0, s>>>(sums.p, nb);
    k_scan_down<<<(unsigned)nb, SC_THREADS, 0, s>>>(in, out, n, sums.p);
    SPMV_CUDA_TRY(cudaGetLastError());
    if (total_host) {
        int last_out = 0;
        SPMV_CUDA_TRY(cudaMemcpyAsync(&last_out, out + n - 1, sizeof(int), cudaMemcpyDeviceToHost, s));
        SPMV_CUDA_TRY(cudaStreamSynchronize(s));
        *total_host = (int64_t)last_out + last_in;
    }
    return SPMV_OK;
}

// ---------------------------------------------------------------------------
// stable LSD radix sort of (uint64 key, uint32 value) pairs, 8 bits a pass
// ---------------------------------------------------------------------------
constexpr int RS_THREADS = 256, RS_WARPS = RS_THREADS / 32, RS_ITEMS = 16;
constexpr int RS_WARP_TILE = 32 * RS_ITEMS, RS_TILE = RS_THREADS * RS_ITEMS;

__global__ void __launch_bounds__(RS_THREADS) k_radix_hist(const uint64_t *keys, int64_t n,
                                                           int shift, unsigned *hist, int nblocks) {
    __shared__ unsigned h[256];
    for (int i = threadIdx.x; i < 256; i += RS_THREADS) h[i] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    unsigned lane = threadIdx.x & 31;
    for (int k = threadIdx.x; k < RS_TILE; k += RS_THREADS) {
        int64_t i = base + k;
        bool valid = i < n;
        unsigned d = valid ? (unsigned)((keys[i] >> shift) & 255u) : 256u;
        unsigned peers = __match_any_sync(FULL, d);
        if (valid && lane == (unsigned)(31 - __clz(peers))) atomicAdd(&h[d], (unsigned)__popc(peers));
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += RS_THREADS) hist[(int64_t)d * nblocks + blockIdx.x] = h[d];
}

__global__ void __launch_bounds__(RS_THREADS) k_radix_scatter(const uint64_t *kin, const uint32_t *vin,
                                                              uint64_t *kout, uint32_t *vout, int64_t n,
                                                              int shift, const int *offsets, int nblocks) {
    __shared__ unsigned wh[RS_WARPS][256];
    __shared__ unsigned boff[256];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < RS_WARPS * 256; i += RS_THREADS) (&wh[0][0])[i] = 0;
    for (int d = threadIdx.x; d < 256; d += RS_THREADS)
        boff[d] = (unsigned)offsets[(int64_t)d * nblocks + blockIdx.x];
    __syncthreads();
    const int64_t wbase = (int64_t)blockIdx.x * RS_TILE + (int64_t)warp * RS_WARP_TILE;
    const unsigned lt = (1u << lane) - 1u;
    unsigned loc[RS_ITEMS];
#pragma unroll
    for (int r = 0; r < RS_ITEMS; ++r) {
        int64_t i = wbase + r * 32 + lane;
        bool valid = i < n;
        unsigned d = valid ? (unsigned)((kin[i] >> shift) & 255u) : 256u;
        unsigned peers = __match_any_sync(FULL, d);
        unsigned cnt = valid ? wh[warp][d] : 0u;
        __syncwarp();
        if (valid && lane == 31 - __clz(peers)) wh[warp][d] = cnt + __popc(peers);
        __syncwarp();
        loc[r] = cnt + __popc(peers & lt);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += RS_THREADS) {
        unsigned run = 0;
        for (int w = 0; w < RS_WARPS; ++w) {
            unsigned c = wh[w][d];
            wh[w][d] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RS_ITEMS; ++r) {
        int64_t i = wbase + r * 32 + lane;
        if (i < n) {
            uint64_t k = kin[i];
            unsigned d = (unsigned)((k >> shift) & 255u);
            unsigned pos = boff[d] + wh[warp][d] + loc[r];
            kout[pos] = k;
            vout[pos] = vin[i];
        }
    }
}

// Sorts keys[0..n) with their values; the result is left in (*kres, *vres),
// which point either at the inputs or at the scratch pair (kalt, valt).
int radix_sort_pairs(uint64_t *keys, uint32_t *vals, uint64_t *kalt, uint32_t *valt, int64_t n,
                     int total_bits, cudaStream_t s, uint64_t **kres, uint32_t **vres) {
    int nblocks = (int)((n + RS_TILE - 1) / RS_TILE);
    Tmp<int> hist;
    SPMV_TRY(hist.alloc((size_t)256 * nblocks, s));
    uint64_t *ka = keys, *kb = kalt;
    uint32_t *va = vals, *vb = valt;
    for (int shift = 0; shift < total_bits; shift += 8) {
        k_radix_hist<<<nblocks, RS_THREADS, 0, s>>>(ka, n, shift, reinterpret_cast<unsigned *>(hist.p),
                                                    nblocks);
        SPMV_TRY(exclusive_scan(hist.p, hist.p, (int64_t)256 * nblocks, s, nullptr));
        k_radix_scatter<<<nblocks, RS_THREADS, 0, s>>>(ka, va, kb, vb, n, shift, hist.p, nblocks);
        SPMV_CUDA_TRY(cudaGetLastError());
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    *kres = ka;
    *vres = va;
    return SPMV_OK;
}

// ---------------------------------------------------------------------------
// unsorted / duplicated triplets: sort by (row, col), merge duplicates
// ---------------------------------------------------------------------------
__global__ void k_make_keys(const int *rows, const int *cols, int64_t nnz, int colbits,
                            uint64_t *keys, uint32_t *idx) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nnz; i += stride) {
        keys[i] = ((uint64_t)(uint32_t)rows[i] << colbits) | (uint32_t)cols[i];
        idx[i] = (uint32_t)i;
    }
}

__global__ void k_heads(const uint64_t *keys, int64_t n, int *head) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        head[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1 : 0;
}

__device__ __forceinline__ double to_acc(double v) { return v; }
__device__ __forceinline__ float to_acc(float v) { return v; }
__device__ __forceinline__ float to_acc(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ void from_acc(double a, double *o) { *o = a; }
__device__ __forceinline__ void from_acc(float a, float *o) { *o = a; }
__device__ __forceinline__ void from_acc(float a, __nv_bfloat16 *o) { *o = __float2bfloat16_rn(a); }

// each run of equal keys becomes one entry; its value is the sum of the
// run's values in original triplet order (the sort is stable)
template <typename V, typename T>
__global__ void k_merge_runs(const uint64_t *keys, const uint32_t *perm, const V *vin,
                             const int *head, const int *pos, int64_t n, int colbits,
                             int *urows, int *ucols, V *uvals) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const uint64_t mask = (uint64_t(1) << colbits) - 1;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        if (!head[i]) continue;
        uint64_t k = keys[i];
        T acc = to_acc(vin[perm[i]]);
        for (int64_t j = i + 1; j < n && !head[j]; ++j) acc += to_acc(vin[perm[j]]);
        int u = pos[i];
        urows[u] = (int)(k >> colbits);
        ucols[u] = (int)(k & mask);
        from_acc(acc, &uvals[u]);
    }
}

template <typename V>
int merge_dispatch(const uint64_t *keys, const uint32_t *perm, const void *vin, const int *head,
                   const int *pos, int64_t n, int colbits, int *urows, int *ucols, void *uvals,
                   cudaStream_t s) {
    using T = typename std::conditional<std::is_same<V, double>::value, double, float>::type;
    k_merge_runs<V, T><<<grid1d(n, 256), 256, 0, s>>>(keys, perm, (const V *)vin, head, pos, n, colbits,
                                                       urows, ucols, (V *)uvals);
    return SPMV_OK;
}

// ---------------------------------------------------------------------------
// format packs from CSR
// ---------------------------------------------------------------------------
// ELL columns as stored: int32 column (padding -1), or the 16-bit offset
// column - row (padding INT16_MIN) when every offset fits
__device__ __forceinline__ void ell_code(int *p, int c, int64_t r) { *p = c; }
__device__ __forceinline__ void ell_code(int16_t *p, int c, int64_t r) {
    *p = c < 0 ? (int16_t)INT16_MIN : (int16_t)(c - r);
}

template <typename V, typename CI>
__global__ void k_ell_pack(const int *rowptr, const int *colidx, const V *vals, int64_t m,
                           int64_t width, int64_t pitch, CI *ell_col, V *ell_val) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < pitch; r += stride) {
        int64_t s = 0, len = 0;
        if (r < m) {
            s = rowptr[r];
            len = rowptr[r + 1] - s;
        }
        for (int64_t k = 0; k < width; ++k) {
            bool have = k < len;
            ell_code(ell_col + k * pitch + r, have ? colidx[s + k] : -1, r);
            ell_val[k * pitch + r] = have ? vals[s + k] : V(0.0f);
        }
    }
}

// largest |column - row| of the matrix (columns ascend within a row, so a
// row's first and last entries bound it)
__global__ void k_max_offset(const int *rowptr, const int *colidx, int64_t m, int *out) {
    int best = 0;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < m; r += stride) {
        const int b = rowptr[r], e = rowptr[r + 1];
        if (b < e) {
            const int64_t lo = colidx[b] - r, hi = colidx[e - 1] - r;
            const int64_t d = max(lo < 0 ? -lo : lo, hi < 0 ? -hi : hi);
            best = max(best, (int)min(d, (int64_t)0x7fffffff));
        }
    }
    best = __reduce_max_sync(FULL, best);
    if ((threadIdx.x & 31) == 0) atomicMax(out, best);
}

// int32 columns of a 16-bit-offset ELL (for export)
__global__ void k_ell_decode(const int16_t *d16, int64_t width, int64_t pitch, int *out) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < width * pitch; i += stride) {
        const int v = d16[i];
        out[i] = v == INT16_MIN ? -1 : (int)(i % pitch) + v;
    }
}

// histogram of min(row length, cap)
__global__ void k_len_hist(const int *rowptr, int64_t m, int cap, unsigned *hist) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned lane = threadIdx.x & 31;
    int64_t mr = (m + 31) / 32 * 32;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < mr; r += stride) {
        bool valid = r < m;
        int len = valid ? min(rowptr[r + 1] - rowptr[r], cap) : -1;
        unsigned peers = __match_any_sync(__activemask(), len);
        if (valid && lane == (unsigned)(31 - __clz(peers))) atomicAdd(&hist[len], (unsigned)__popc(peers));
    }
}

__global__ void k_tail_counts(const int *rowptr, int64_t m, int width, int *cnt) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < m; r += stride)
        cnt[r] = max(0, rowptr[r + 1] - rowptr[r] - width);
}

// tail entry o belongs to the row r with tptr[r] <= o < tptr[r+1]; entries
// are spread over the threads (long rows do not serialise on one thread)
template <typename V>
__global__ void k_hyb_tail(const int *rowptr, const int *colidx, const V *vals, int64_t m, int width,
                           const int *tptr, int64_t tail, int *trows, int *tcols, V *tvals) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < tail; o += stride) {
        const int r = row_of(tptr, m, o);
        const int64_t k = (int64_t)rowptr[r] + width + (o - tptr[r]);
        trows[o] = r;
        tcols[o] = colidx[k];
        tvals[o] = vals[k];
    }
}

__global__ void k_block_keys(const int *rows, const int *cols, int64_t nnz, int r, int bcbits,
                             uint64_t *keys, uint32_t *idx) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nnz; i += stride) {
        keys[i] = ((uint64_t)(rows[i] / r) << bcbits) | (uint64_t)(cols[i] / r);
        idx[i] = (uint32_t)i;
    }
}

template <typename V>
__global__ void k_bsr_fill(const uint64_t *keys, const uint32_t *perm, const int *head, const int *pos,
                           int64_t n, const int *rows, const int *cols, const V *vals, int r, int bcbits,
                           int *bcol, int *brow_of_block, V *bval) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const uint64_t mask = (uint64_t(1) << bcbits) - 1;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        int b = pos[i] + head[i] - 1;
        if (head[i]) {
            bcol[b] = (int)(keys[i] & mask);
            brow_of_block[b] = (int)(keys[i] >> bcbits);
        }
        uint32_t e = perm[i];
        int rr = rows[e] % r, cc = cols[e] % r;
        bval[(int64_t)b * r * r + rr * r + cc] = vals[e];
    }
}

// segmented-kernel chunk metadata (COO and HYB tail): first chunk of the
// chunk's head row and last chunk of its tail row
__global__ void k_seg_meta_coo(const int *rows, const int *rowptr, int64_t nnz, int C,
                               int64_t nchunks, int *meta0, int *meta1) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nchunks; c += stride) {
        int64_t e0 = c * C, e1 = min(e0 + C, nnz);
        int hrow = rows[e0], trow = rows[e1 - 1];
        meta0[c] = rowptr[hrow] / C;
        meta1[c] = (rowptr[trow + 1] - 1) / C;
    }
}

// split CSR: row holding each chunk's first entry; entry nchunks = m - 1
__global__ void k_seg_meta_split(const int *rowptr, int64_t m, int64_t nnz, int C, int64_t nchunks,
                                 int *meta0) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c <= nchunks; c += stride) {
        if (c == nchunks) { meta0[c] = (int)(m - 1); continue; }
        meta0[c] = row_of(rowptr, m, c * C);
    }
}

// split CSR by warp chunks: first row starting at or after each chunk's
// first entry (lower bound of c*C in rowptr[0..m)); entry nchunks = m
__global__ void k_seg_meta_merge(const int *rowptr, int64_t m, int C, int64_t nchunks, int *meta) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c <= nchunks; c += stride) {
        if (c == nchunks) { meta[c] = (int)m; continue; }
        const int64_t k = c * (int64_t)C;
        int64_t lo = 0, hi = m;  // first r in [0, m] with r == m or rowptr[r] >= k
        while (lo < hi) {
            const int64_t mid = lo + ((hi - lo) >> 1);
            if (rowptr[mid] >= k) hi = mid; else lo = mid + 1;
        }
        meta[c] = (int)lo;
    }
}

__global__ void k_fill_u64(unsigned long long *p, int64_t n, unsigned long long v) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) p[i] = v;
}

// segments per long row: ceil(len / seg) if len > threshold, else 0
__global__ void k_long_count(const int *rowptr, int64_t nrows, int64_t threshold, int64_t seg, int *cnt) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nrows; r += stride) {
        const int64_t len = rowptr[r + 1] - rowptr[r];
        cnt[r] = len > threshold ? (int)((len + seg - 1) / seg) : 0;
    }
}

__global__ void k_long_fill(const int *rowptr, int64_t nrows, int64_t threshold, int64_t seg, const int *off,
                            int *seg_row, int *seg_begin, int *seg_end, int *seg_c0, int *seg_c1) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nrows; r += stride) {
        const int64_t b = rowptr[r], e = rowptr[r + 1];
        if (e - b <= threshold) continue;
        const int64_t ns = (e - b + seg - 1) / seg;
        const int o = off[r];
        for (int64_t j = 0; j < ns; ++j) {
            seg_row[o + j] = (int)r;
            seg_begin[o + j] = (int)(b + j * seg);
            seg_end[o + j] = (int)min(b + (j + 1) * seg, e);
            seg_c0[o + j] = o;
            seg_c1[o + j] = (int)(o + ns - 1);
        }
    }
}

// SELL: sort key per row = descending length (the sort is stable, so rows of
// equal length keep their order)
__global__ void k_sell_keys(const int *rowptr, int64_t m, uint64_t *keys, uint32_t *idx) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < m; r += stride) {
        const int len = rowptr[r + 1] - rowptr[r];
        keys[r] = (uint64_t)(uint32_t)(0x7fffffff - len);
        idx[r] = (uint32_t)r;
    }
}

// slice width = length of its first (longest) sorted row; slots = 32 * width
__global__ void k_sell_widths(const int *rowptr, const uint32_t *perm, int64_t m, int64_t nslices, int *slots) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t sl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; sl < nslices; sl += stride) {
        const uint32_t r = perm[sl * 32];
        slots[sl] = 32 * (rowptr[r + 1] - rowptr[r]);
    }
}

// Slot of entry k of lane l in a slice of width w starting at slot base:
// the first w & ~3 columns in groups of four, each group 32 lanes x 4
// consecutive entries (a lane's four entries of a group contiguous), then
// the remaining w & 3 columns column-major (32 lanes each).
// (grouped = false: every column column-major, entry k at base + 32 k + l)
__host__ __device__ __forceinline__ int64_t sell_slot(int64_t base, int64_t w, int64_t k, int l, bool grouped) {
    const int64_t w4 = grouped ? (w & ~int64_t(3)) : 0;
    return k < w4 ? base + 128 * (k >> 2) + 4 * l + (k & 3) : base + 32 * w4 + 32 * (k - w4) + l;
}

// one warp per entry index k of a slice (slices hold 32 slots per column,
// so the warp finds (sl, k) from its 32-slot index with one binary search,
// the same address in every lane) and lane l fills sorted row 32 sl + l
template <typename V>
__global__ void k_sell_fill(const int *rowptr, const int *colidx, const V *vals, const uint32_t *perm, int64_t m,
                            int64_t nslices, const int *sptr, int64_t total, int *scol, V *sval, int *sperm,
                            bool grouped) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w = warp; w < total / 32; w += nwarps) {
        const int64_t p0 = 32 * w;
        const int sl = row_of(sptr, nslices, p0);
        const int64_t k = (p0 - sptr[sl]) / 32;
        const int64_t q = (int64_t)sl * 32 + lane;
        int c = -1;
        V v = V(0.0f);
        if (q < m) {
            const uint32_t r = perm[q];
            const int64_t rs = rowptr[r];
            if (k < rowptr[r + 1] - rs) {
                c = colidx[rs + k];
                v = vals[rs + k];
            }
        }
        const int64_t at = sell_slot(sptr[sl], (sptr[sl + 1] - sptr[sl]) / 32, k, lane, grouped);
        scol[at] = c;
        sval[at] = v;
    }
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < m; q += stride) sperm[q] = (int)perm[q];
}

// work items per slice: ceil(width / kmax), at least one
__global__ void k_sell_item_count(const int *sptr, int64_t nslices, int kmax, int *cnt) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t sl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; sl < nslices; sl += stride) {
        const int width = (sptr[sl + 1] - sptr[sl]) / 32;
        cnt[sl] = (width + kmax - 1) / kmax;  // zero-width slices (empty rows) get no item
    }
}

// first zero-width slice: the first s with ptr[s] == ptr[nslices] (rows are
// sorted by descending length, so every later slice is empty too)
__global__ void k_sell_first_empty(const int *sptr, int64_t nslices, int *out) {
    const int total = sptr[nslices];
    int64_t lo = 0, hi = nslices;
    while (lo < hi) {
        const int64_t mid = lo + ((hi - lo) >> 1);
        if (sptr[mid] >= total) hi = mid; else lo = mid + 1;
    }
    *out = (int)lo;
}

// item j of a slice: its slice, the slot offset of its first column
// (ptr[slice] + 32 j kmax), its column count, and the slice's item range
__global__ void k_sell_item_fill(const int *sptr, int64_t nslices, int kmax, const int *off, int *it_slice,
                                 int *it_base, int *it_len, int *it_c0, int *it_c1) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t sl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; sl < nslices; sl += stride) {
        const int width = (sptr[sl + 1] - sptr[sl]) / 32;
        const int n = (width + kmax - 1) / kmax;
        const int o = off[sl];
        for (int j = 0; j < n; ++j) {
            it_slice[o + j] = (int)sl;
            it_base[o + j] = sptr[sl] + 32 * j * kmax;
            it_len[o + j] = min((j + 1) * kmax, width) - j * kmax;
            it_c0[o + j] = o;
            it_c1[o + j] = o + n - 1;
        }
    }
}

// ---------------------------------------------------------------------------
// row panels: more triplets than one handle indexes with int32 offsets
// ---------------------------------------------------------------------------
constexpr int PANEL_CHUNK_SHIFT = 18;  // 2^18-row chunks, a multiple of 4 rows
constexpr int PC_THREADS = SC_THREADS, PC_ITEMS = 16, PC_TILE = PC_THREADS * PC_ITEMS;

// triplets per 2^18-row chunk; lanes of a warp on the same chunk add once
__global__ void k_chunk_hist(const int *rows, int64_t nnz, int nchunks, unsigned long long *counts) {
    extern __shared__ unsigned sh_chunks[];
    for (int c = threadIdx.x; c < nchunks; c += blockDim.x) sh_chunks[c] = 0;
    __syncthreads();
    const unsigned lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t nr = (nnz + 31) / 32 * 32;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nr; i += stride) {
        const int c = i < nnz ? rows[i] >> PANEL_CHUNK_SHIFT : -1;
        const unsigned peers = __match_any_sync(FULL, c);
        if (c >= 0 && lane == (unsigned)(__ffs(peers) - 1)) atomicAdd(&sh_chunks[c], (unsigned)__popc(peers));
    }
    __syncthreads();
    for (int c = threadIdx.x; c < nchunks; c += blockDim.x)
        if (sh_chunks[c]) atomicAdd(&counts[c], (unsigned long long)sh_chunks[c]);
}

// triplets per 4-row group of rows [lo, hi)
__global__ void k_group_hist(const int *rows, int64_t nnz, int lo, int hi, unsigned long long *counts) {
    const unsigned lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t nr = (nnz + 31) / 32 * 32;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nr; i += stride) {
        const int r = i < nnz ? rows[i] : -1;
        const int g = r >= lo && r < hi ? (r - lo) >> 2 : -1;
        const unsigned peers = __match_any_sync(FULL, g);
        if (g >= 0 && lane == (unsigned)(__ffs(peers) - 1)) atomicAdd(&counts[g], (unsigned long long)__popc(peers));
    }
}

// per 4096-triplet tile: triplets with row in [r0, r1)
__global__ void __launch_bounds__(PC_THREADS) k_panel_tile_count(const int *rows, int64_t nnz, int r0, int r1,
                                                                 int *cnt) {
    const int64_t base = (int64_t)blockIdx.x * PC_TILE;
    int c = 0;
    for (int k = threadIdx.x; k < PC_TILE; k += PC_THREADS) {
        const int64_t i = base + k;
        if (i < nnz) {
            const int r = rows[i];
            c += r >= r0 && r < r1;
        }
    }
    c = __reduce_add_sync(FULL, c);
    __shared__ int ws[PC_THREADS / 32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < PC_THREADS / 32; ++w) t += ws[w];
        cnt[blockIdx.x] = t;
    }
}

// stable scatter of the tile's in-panel triplets to off[tile] + rank
template <typename W>
__global__ void __launch_bounds__(PC_THREADS) k_panel_scatter(const int *rows, const int *cols, const W *vals,
                                                              int64_t nnz, int r0, int r1, const int *off,
                                                              int *orow, int *ocol, W *oval) {
    __shared__ int total_s;
    const int64_t base = (int64_t)blockIdx.x * PC_TILE + (int64_t)threadIdx.x * PC_ITEMS;
    int c = 0;
#pragma unroll
    for (int j = 0; j < PC_ITEMS; ++j) {
        const int64_t i = base + j;
        if (i < nnz) {
            const int r = rows[i];
            c += r >= r0 && r < r1;
        }
    }
    int pos = block_exclusive_scan(c, &total_s) + off[blockIdx.x];
#pragma unroll
    for (int j = 0; j < PC_ITEMS; ++j) {
        const int64_t i = base + j;
        if (i < nnz) {
            const int r = rows[i];
            if (r >= r0 && r < r1) {
                orow[pos] = r - r0;
                ocol[pos] = cols[i];
                oval[pos] = vals[i];
                ++pos;
            }
        }
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// public (library-internal) entry points
// ---------------------------------------------------------------------------

int decode_ell_columns(const spmv_matrix *h, int32_t *d_out, cudaStream_t s) {
    const int64_t n = h->ell_width * h->ell_pitch;
    if (n == 0) return SPMV_OK;
    k_ell_decode<<<grid1d(n, 256), 256, 0, s>>>(h->ell_d16, h->ell_width, h->ell_pitch, d_out);
    SPMV_CUDA_TRY(cudaGetLastError());
    return SPMV_OK;
}

int expand_rows(const int32_t *rowptr, int64_t m, int64_t nnz, int32_t *rows_out, cudaStream_t s) {
    if (nnz == 0) return SPMV_OK;
    k_expand_rows<<<grid1d(nnz, 256), 256, 0, s>>>(rowptr, m, nnz, rows_out);
    SPMV_CUDA_TRY(cudaGetLastError());
    return SPMV_OK;
}

int check_triplet_bounds(const int32_t *d_rows, const int32_t *d_cols, int64_t nnz, int64_t m, int64_t n,
                         cudaStream_t s) {
    if (nnz == 0) return SPMV_OK;
    Tmp<unsigned> flags;
    SPMV_TRY(flags.alloc(1, s));
    SPMV_CUDA_TRY(cudaMemsetAsync(flags.p, 0, sizeof(unsigned), s));
    k_check_triplets<<<grid1d(nnz, 256), 256, 0, s>>>(d_rows, d_cols, nnz, m, n, flags.p);
    SPMV_CUDA_TRY(cudaGetLastError());
    unsigned hflags = 0;
    SPMV_CUDA_TRY(cudaMemcpyAsync(&hflags, flags.p, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    SPMV_CUDA_TRY(cudaStreamSynchronize(s));
    if (hflags & 1u) {
        set_error("spmv_create: a triplet lies outside the %lld x %lld matrix", (long long)m, (long long)n);
        return SPMV_ERR_INVALID;
    }
    return SPMV_OK;
}

int plan_panels(const int32_t *d_rows, int64_t nnz, int64_t m, int64_t limit, cudaStream_t s,
                std::vector<int64_t> *bounds) {
    const int64_t chunk = int64_t(1) << PANEL_CHUNK_SHIFT;
    const int nchunks = (int)((m + chunk - 1) / chunk);
    Tmp<unsigned long long> counts;
    SPMV_TRY(counts.alloc(nchunks, s));
    SPMV_CUDA_TRY(cudaMemsetAsync(counts.p, 0, sizeof(unsigned long long) * nchunks, s));
    k_chunk_hist<<<grid1d(nnz, 256, 152 * 8), 256, sizeof(unsigned) * nchunks, s>>>(d_rows, nnz, nchunks, counts.p);
    SPMV_CUDA_TRY(cudaGetLastError());
    std::vector<unsigned long long> hc(nchunks);
    SPMV_CUDA_TRY(cudaMemcpyAsync(hc.data(), counts.p, sizeof(unsigned long long) * nchunks,
                                  cudaMemcpyDeviceToHost, s));
    SPMV_CUDA_TRY(cudaStreamSynchronize(s));
    bounds->assign(1, 0);
    int64_t cur = 0;  // triplets in the open panel
    for (int c = 0; c < nchunks; ++c) {
        const int64_t lo = (int64_t)c * chunk, hi = std::min<int64_t>(m, lo + chunk);
        if ((int64_t)hc[c] <= limit) {
            if (cur > 0 && cur + (int64_t)hc[c] > limit) {
                bounds->push_back(lo);
                cur = 0;
            }
            cur += (int64_t)hc[c];
            continue;
        }
        // a chunk over the limit: split it at 4-row groups
        const int64_t ng = (hi - lo + 3) / 4;
        Tmp<unsigned long long> g;
        SPMV_TRY(g.alloc(ng, s));
        SPMV_CUDA_TRY(cudaMemsetAsync(g.p, 0, sizeof(unsigned long long) * ng, s));
        k_group_hist<<<grid1d(nnz, 256, 152 * 8), 256, 0, s>>>(d_rows, nnz, (int)lo, (int)hi, g.p);
        SPMV_CUDA_TRY(cudaGetLastError());
        std::vector<unsigned long long> hg(ng);
        SPMV_CUDA_TRY(cudaMemcpyAsync(hg.data(), g.p, sizeof(unsigned long long) * ng, cudaMemcpyDeviceToHost, s));
        SPMV_CUDA_TRY(cudaStreamSynchronize(s));
        for (int64_t k = 0; k < ng; ++k) {
            if ((int64_t)hg[k] > limit) {
                set_error("spmv_create: rows %lld..%lld hold %llu triplets, more than one panel (%lld) holds",
                          (long long)(lo + 4 * k), (long long)std::min<int64_t>(m, lo + 4 * k + 4) - 1,
                          hg[k], (long long)limit);
                return SPMV_ERR_UNSUPPORTED;
            }
            if (cur > 0 && cur + (int64_t)hg[k] > limit) {
                bounds->push_back(lo + 4 * k);
                cur = 0;
            }
            cur += (int64_t)hg[k];
        }
    }
    bounds->push_back(m);
    return SPMV_OK;
}

int gather_panel(const int32_t *d_rows, const int32_t *d_cols, const void *d_vals, size_t vs, int64_t nnz,
                 int64_t r0, int64_t r1, int32_t **orow, int32_t **ocol, void **oval, int64_t *count,
                 cudaStream_t s) {
    *orow = *ocol = nullptr;
    *oval = nullptr;
    const int64_t ntiles = (nnz + PC_TILE - 1) / PC_TILE;
    Tmp<int> cnt, off;
    SPMV_TRY(cnt.alloc(ntiles, s));
    SPMV_TRY(off.alloc(ntiles, s));
    k_panel_tile_count<<<(unsigned)ntiles, PC_THREADS, 0, s>>>(d_rows, nnz, (int)r0, (int)r1, cnt.p);
    SPMV_CUDA_TRY(cudaGetLastError());
    int64_t total = 0;
    SPMV_TRY(exclusive_scan(cnt.p, off.p, ntiles, s, &total));
    *count = total;
    SPMV_TRY(dalloc(orow, (size_t)total));
    SPMV_TRY(dalloc(ocol, (size_t)total));
    SPMV_TRY(dalloc_bytes(oval, vs * (size_t)std::max<int64_t>(total, 1)));
    if (vs == 8)
        k_panel_scatter<uint64_t><<<(unsigned)ntiles, PC_THREADS, 0, s>>>(
            d_rows, d_cols, (const uint64_t *)d_vals, nnz, (int)r0, (int)r1, off.p, *orow, *ocol, (uint64_t *)*oval);
    else if (vs == 4)
        k_panel_scatter<uint32_t><<<(unsigned)ntiles, PC_THREADS, 0, s>>>(
            d_rows, d_cols, (const uint32_t *)d_vals, nnz, (int)r0, (int)r1, off.p, *orow, *ocol, (uint32_t *)*oval);
    else
        k_panel_scatter<uint16_t><<<(unsigned)ntiles, PC_THREADS, 0, s>>>(
            d_rows, d_cols, (const uint16_t *)d_vals, nnz, (int)r0, (int)r1, off.p, *orow, *ocol, (uint16_t *)*oval);
    SPMV_CUDA_TRY(cudaGetLastError());
    SPMV_CUDA_TRY(cudaStreamSynchronize(s));
    return SPMV_OK;
}

// The CSR arrays are allocated CSR_PAD entries longer than needed: the
// staged tile kernel copies whole multiples of 8 column/value entries and
// 16-byte windows of row pointers, so the last tile may read up to 7 entries
// past nnz and 3 past m (never used).
constexpr size_t CSR_PAD = 8;

int build_csr(spmv_matrix *h, const int32_t *d_rows, const int32_t *d_cols, const void *d_vals,
              cudaStream_t s) {
    const int64_t m = h->m, n = h->n, nnz_in = h->nnz;
    const size_t vs = value_size(h->vt);
    SPMV_TRY(dalloc(&h->rowptr, (size_t)m + 1 + CSR_PAD));  // staged windows may read 3 past m
    if (nnz_in == 0) {
        SPMV_CUDA_TRY(cudaMemsetAsync(h->rowptr, 0, sizeof(int) * (m + 1), s));
        SPMV_TRY(dalloc(&h->colidx, 1));
        SPMV_TRY(dalloc_bytes(&h->vals, vs));
        h->max_row = 0;
        SPMV_CUDA_TRY(cudaStreamSynchronize(s));
        return SPMV_OK;
    }
    Tmp<unsigned> flags;
    SPMV_TRY(flags.alloc(1, s));
    SPMV_CUDA_TRY(cudaMemsetAsync(flags.p, 0, sizeof(unsigned), s));
    k_check_triplets<<<grid1d(nnz_in, 256), 256, 0, s>>>(d_rows, d_cols, nnz_in, m, n, flags.p);
    SPMV_CUDA_TRY(cudaGetLastError());
    unsigned hflags = 0;
    SPMV_CUDA_TRY(cudaMemcpyAsync(&hflags, flags.p, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    SPMV_CUDA_TRY(cudaStreamSynchronize(s));
    if (hflags & 1u) {
        set_error("spmv_create: a triplet lies outside the %lld x %lld matrix", (long long)m,
                  (long long)n);
        return SPMV_ERR_INVALID;
    }
    if (!(hflags & 6u)) {
        // already sorted by (row, col) with no repeated pair: copy and index
        h->nnz = nnz_in;
        SPMV_TRY(dalloc(&h->colidx, (size_t)nnz_in + CSR_PAD));
        SPMV_TRY(dalloc_bytes(&h->vals, vs * (nnz_in + CSR_PAD)));
        SPMV_CUDA_TRY(cudaMemcpyAsync(h->colidx, d_cols, sizeof(int) * nnz_in, cudaMemcpyDeviceToDevice, s));
        SPMV_CUDA_TRY(cudaMemcpyAsync(h->vals, d_vals, vs * nnz_in, cudaMemcpyDeviceToDevice, s));
        k_rowptr_from_sorted<<<grid1d(m + 1, 256), 256, 0, s>>>(d_rows, nnz_in, m, h->rowptr);
        SPMV_CUDA_TRY(cudaGetLastError());
    } else {
        const int colbits = std::max(1, bits_for(n));
        const int total_bits = bits_for(m) + colbits;
        Tmp<uint64_t> k0, k1;
        Tmp<uint32_t> v0, v1;
        SPMV_TRY(k0.alloc(nnz_in, s));
        SPMV_TRY(k1.alloc(nnz_in, s));
        SPMV_TRY(v0.alloc(nnz_in, s));
        SPMV_TRY(v1.alloc(nnz_in, s));
        k_make_keys<<<grid1d(nnz_in, 256), 256, 0, s>>>(d_rows, d_cols, nnz_in, colbits, k0.p, v0.p);
        uint64_t *ks;
        uint32_t *vp;
        SPMV_TRY(radix_sort_pairs(k0.p, v0.p, k1.p, v1.p, nnz_in, total_bits, s, &ks, &vp));
        Tmp<int> head, pos, urows;
        SPMV_TRY(head.alloc(nnz_in, s));
        SPMV_TRY(pos.alloc(nnz_in, s));
        k_heads<<<grid1d(nnz_in, 256), 256, 0, s>>>(ks, nnz_in, head.p);
        int64_t nu = 0;
        SPMV_TRY(exclusive_scan(head.p, pos.p, nnz_in, s, &nu));
        h->nnz = nu;
        SPMV_TRY(urows.alloc(nu, s));
        SPMV_TRY(dalloc(&h->colidx, (size_t)nu + CSR_PAD));
        SPMV_TRY(dalloc_bytes(&h->vals, vs * (nu + CSR_PAD)));
        if (h->vt == SPMV_F64)
            merge_dispatch<double>(ks, vp, d_vals, head.p, pos.p, nnz_in, colbits, urows.p, h->colidx, h->vals, s);
        else if (h->vt == SPMV_F32)
            merge_dispatch<float>(ks, vp, d_vals, head.p, pos.p, nnz_in, colbits, urows.p, h->colidx, h->vals, s);
        else
            merge_dispatch<__nv_bfloat16>(ks, vp, d_vals, head.p, pos.p, nnz_in, colbits, urows.p, h->colidx,
                                          h->vals, s);
        k_rowptr_from_sorted<<<grid1d(m + 1, 256), 256, 0, s>>>(urows.p, nu, m, h->rowptr);
        SPMV_CUDA_TRY(cudaGetLastError());
    }
    Tmp<unsigned long long> mx;   // [0]: longest row, [1]: contiguous pairs
    SPMV_TRY(mx.alloc(2, s));
    SPMV_CUDA_TRY(cudaMemsetAsync(mx.p, 0, 2 * sizeof(unsigned long long), s));
    if (m > 0) k_max_row<<<grid1d(m, 256), 256, 0, s>>>(h->rowptr, m, reinterpret_cast<int *>(mx.p));
    if (h->nnz > 1) k_contiguous_pairs<<<grid1d(h->nnz, 256), 256, 0, s>>>(h->colidx, h->nnz, mx.p + 1);
    SPMV_CUDA_TRY(cudaGetLastError());
    unsigned long long hmx[2] = {0, 0};
    SPMV_CUDA_TRY(cudaMemcpyAsync(hmx, mx.p, sizeof(hmx), cudaMemcpyDeviceToHost, s));
    SPMV_CUDA_TRY(cudaStreamSynchronize(s));
    h->max_row = (int64_t)(hmx[0] & 0xffffffffull);
    h->contig = h->nnz > 1 ? (double)hmx[1] / (double)(h->nnz - 1) : 0.0;
    return SPMV_OK;
}

int alloc_partials(Partials *p, int64_t units, int stride, int vt, cudaStream_t s) {
    *p = Partials{};
    p->units = units;
    p->stride = stride;
    const int64_t n = (units + 1) * stride;
    const size_t ts = vec_size(vt);
    SPMV_TRY(dalloc_bytes(&p->head, ts * n));
    SPMV_TRY(dalloc_bytes(&p->tail, ts * n));
    SPMV_TRY(dalloc(&p->count, (size_t)n));
    SPMV_TRY(dalloc(&p->xslot, (size_t)n));
    SPMV_CUDA_TRY(cudaMemsetAsync(p->count, 0, sizeof(uint32_t) * n, s));
    const unsigned long long empty = vt == SPMV_F64 ? XEnc<double>::EMPTY : XEnc<float>::EMPTY;
    k_fill_u64<<<grid1d(n, 256), 256, 0, s>>>(p->xslot, n, empty);
    SPMV_CUDA_TRY(cudaGetLastError());
    return SPMV_OK;
}

void free_partials(Partials *p) {
    auto f = [](void *q) { if (q) cudaFree(q); };
    f(p->head); f(p->tail); f(p->count); f(p->xslot);
    *p = Partials{};
}

static void free_long_rows(spmv_matrix *h) {
    LongRows &L = h->lng;
    auto f = [](void *q) { if (q) cudaFree(q); };
    f(L.seg_row); f(L.seg_begin); f(L.seg_end); f(L.seg_c0); f(L.seg_c1);
    free_partials(&L.part);
    L = LongRows{};
}

int build_long_rows(spmv_matrix *h, const int32_t *rowptr, int64_t nrows, int64_t threshold, int64_t seg,
                    int stride, cudaStream_t s) {
    free_long_rows(h);
    LongRows &L = h->lng;
    L.threshold = threshold;
    if (nrows == 0) return SPMV_OK;
    Tmp<int> cnt, off;
    SPMV_TRY(cnt.alloc(nrows, s));
    SPMV_TRY(off.alloc(nrows, s));
    k_long_count<<<grid1d(nrows, 256), 256, 0, s>>>(rowptr, nrows, threshold, seg, cnt.p);
    SPMV_CUDA_TRY(cudaGetLastError());
    int64_t total = 0;
    SPMV_TRY(exclusive_scan(cnt.p, off.p, nrows, s, &total));
    L.nseg = total;
    if (total == 0) return SPMV_OK;
    SPMV_TRY(dalloc(&L.seg_row, (size_t)total));
    SPMV_TRY(dalloc(&L.seg_begin, (size_t)total));
    SPMV_TRY(dalloc(&L.seg_end, (size_t)total));
    SPMV_TRY(dalloc(&L.seg_c0, (size_t)total));
    SPMV_TRY(dalloc(&L.seg_c1, (size_t)total));
    k_long_fill<<<grid1d(nrows, 256), 256, 0, s>>>(rowptr, nrows, threshold, seg, off.p, L.seg_row, L.seg_begin,
                                                   L.seg_end, L.seg_c0, L.seg_c1);
    SPMV_CUDA_TRY(cudaGetLastError());
    SPMV_TRY(alloc_partials(&L.part, total, stride, h->vt, s));
    return SPMV_OK;
}

void free_packed(spmv_matrix *h) {
    auto f = [](void *p) { if (p) cudaFree(p); };
    f(h->coo_rows); h->coo_rows = nullptr;
    f(h->ell_col); h->ell_col = nullptr;
    f(h->ell_d16); h->ell_d16 = nullptr;
    f(h->ell_val); h->ell_val = nullptr;
    h->ell_width = h->ell_pitch = 0;
    f(h->hyb_rows); h->hyb_rows = nullptr;
    f(h->hyb_cols); h->hyb_cols = nullptr;
    f(h->hyb_vals); h->hyb_vals = nullptr;
    f(h->hyb_ptr); h->hyb_ptr = nullptr;
    h->hyb_nnz = 0;
    f(h->bsr_rowptr); h->bsr_rowptr = nullptr;
    f(h->bsr_col); h->bsr_col = nullptr;
    f(h->bsr_val); h->bsr_val = nullptr;
    f(h->sell_ptr); h->sell_ptr = nullptr;
    f(h->sell_col); h->sell_col = nullptr;
    f(h->sell_val); h->sell_val = nullptr;
    f(h->sell_perm); h->sell_perm = nullptr;
    h->sell_nslices = h->sell_slots = 0;
    h->bsr_r = 0;
    h->bsr_mb = h->bsr_blocks = 0;
    f(h->seg.meta0); f(h->seg.meta1);
    free_partials(&h->seg.part);
    h->seg = SegScratch{};
    free_long_rows(h);
}

namespace {

template <typename CI>
int launch_ell_pack(spmv_matrix *h, int64_t width, int64_t pitch, CI *cols, cudaStream_t s) {
    const unsigned g = grid1d(pitch, 256);
    const int64_t m = h->m;
    if (h->vt == SPMV_F64)
        k_ell_pack<double, CI><<<g, 256, 0, s>>>(h->rowptr, h->colidx, (const double *)h->vals, m, width, pitch,
                                                 cols, (double *)h->ell_val);
    else if (h->vt == SPMV_F32)
        k_ell_pack<float, CI><<<g, 256, 0, s>>>(h->rowptr, h->colidx, (const float *)h->vals, m, width, pitch,
                                                cols, (float *)h->ell_val);
    else
        k_ell_pack<__nv_bfloat16, CI><<<g, 256, 0, s>>>(h->rowptr, h->colidx, (const __nv_bfloat16 *)h->vals, m,
                                                        width, pitch, cols, (__nv_bfloat16 *)h->ell_val);
    SPMV_CUDA_TRY(cudaGetLastError());
    return SPMV_OK;
}

// bf16 values: columns are stored as 16-bit offsets from the row when
// every |column - row| of the matrix is at most 32767 (stencils, banded and
// block-diagonal matrices), 2 index bytes per slot instead of 4.  Measured
// on GB300 at the default unroll: bf16 13% faster (27-point stencil 76.5
// against 88.1 us); fp32 only gains at unroll 8 and loses 18% at its
// default 4; fp64 loses 8-10% (its ELL kernel is held by the fp64 pipe and
// the decode sits between the column load and the x gather).  fp32 and
// fp64 keep int32 columns.
int pack_ell(spmv_matrix *h, int64_t width, bool hyb, cudaStream_t s) {
    const int64_t m = h->m;
    const int64_t pitch = (m + 31) / 32 * 32;
    const size_t vs = value_size(h->vt);
    h->ell_width = width;
    h->ell_pitch = pitch;
    int maxoff = 0x7fffffff;
    if (width > 0 && m > 0 && h->vt == SPMV_BF16) {
        Tmp<int> mo;
        SPMV_TRY(mo.alloc(1, s));
        SPMV_CUDA_TRY(cudaMemsetAsync(mo.p, 0, sizeof(int), s));
        k_max_offset<<<grid1d(m, 256), 256, 0, s>>>(h->rowptr, h->colidx, m, mo.p);
        SPMV_CUDA_TRY(cudaGetLastError());
        SPMV_CUDA_TRY(cudaMemcpyAsync(&maxoff, mo.p, sizeof(int), cudaMemcpyDeviceToHost, s));
        SPMV_CUDA_TRY(cudaStreamSynchronize(s));
    }
    SPMV_TRY(dalloc_bytes(&h->ell_val, vs * width * pitch));
    if (maxoff <= 32767) {
        SPMV_TRY(dalloc(&h->ell_d16, (size_t)(width * pitch)));
        if (width > 0 && pitch > 0) SPMV_TRY(launch_ell_pack<int16_t>(h, width, pitch, h->ell_d16, s));
    } else {
        SPMV_TRY(dalloc(&h->ell_col, (size_t)(width * pitch)));
        if (width > 0 && pitch > 0) SPMV_TRY(launch_ell_pack<int>(h, width, pitch, h->ell_col, s));
    }
    (void)hyb;
    return SPMV_OK;
}

// HYB ELL width: the largest k >= 1 with at least max(4096, m/3) rows of
// length >= k (0 if none)
int hyb_width_rule(spmv_matrix *h, cudaStream_t s, int64_t *width) {
    const int64_t m = h->m;
    const int cap = (int)std::min<int64_t>(h->max_row, 1 << 20);
    if (m == 0 || cap == 0) { *width = 0; return SPMV_OK; }
    Tmp<unsigned> hist;
    SPMV_TRY(hist.alloc(cap + 1, s));
    SPMV_CUDA_TRY(cudaMemsetAsync(hist.p, 0, sizeof(unsigned) * (cap + 1), s));
    k_len_hist<<<grid1d(m, 256), 256, 0, s>>>(h->rowptr, m, cap, hist.p);
    std::vector<unsigned> hh(cap + 1);
    SPMV_CUDA_TRY(cudaMemcpyAsync(hh.data(), hist.p, sizeof(unsigned) * (cap + 1), cudaMemcpyDeviceToHost, s));
    SPMV_CUDA_TRY(cudaStreamSynchronize(s));
    int64_t ge = m;  // rows with length >= k, k = 0
    int64_t best = 0;
    for (int k = 1; k <= cap; ++k) {
        ge -= hh[k - 1];
        if (ge >= 4096 && 3 * ge >= m) best = k;
        else break;
    }
    *width = best;
    return SPMV_OK;
}

int pack_hyb(spmv_matrix *h, int64_t width, cudaStream_t s) {
    const int64_t m = h->m;
    SPMV_TRY(pack_ell(h, width, true, s));
    SPMV_TRY(dalloc(&h->hyb_ptr, (size_t)m + 1));
    Tmp<int> cnt;
    SPMV_TRY(cnt.alloc(m + 1, s));
    SPMV_CUDA_TRY(cudaMemsetAsync(cnt.p, 0, sizeof(int) * (m + 1), s));
    if (m > 0) k_tail_counts<<<grid1d(m, 256), 256, 0, s>>>(h->rowptr, m, (int)width, cnt.p);
    int64_t tail = 0;
    SPMV_TRY(exclusive_scan(cnt.p, h->hyb_ptr, m + 1, s, &tail));
    h->hyb_nnz = tail;
    const size_t vs = value_size(h->vt);
    SPMV_TRY(dalloc(&h->hyb_rows, (size_t)tail));
    SPMV_TRY(dalloc(&h->hyb_cols, (size_t)tail));
    SPMV_TRY(dalloc_bytes(&h->hyb_vals, vs * tail));
    if (tail > 0) {
        unsigned g = grid1d(tail, 256);
        if (h->vt == SPMV_F64)
            k_hyb_tail<double><<<g, 256, 0, s>>>(h->rowptr, h->colidx, (const double *)h->vals, m, (int)width,
                                                 h->hyb_ptr, tail, h->hyb_rows, h->hyb_cols, (double *)h->hyb_vals);
        else if (h->vt == SPMV_F32)
            k_hyb_tail<float><<<g, 256, 0, s>>>(h->rowptr, h->colidx, (const float *)h->vals, m, (int)width,
                                                h->hyb_ptr, tail, h->hyb_rows, h->hyb_cols, (float *)h->hyb_vals);
        else
            k_hyb_tail<__nv_bfloat16><<<g, 256, 0, s>>>(h->rowptr, h->colidx, (const __nv_bfloat16 *)h->vals, m,
                                                        (int)width, h->hyb_ptr, tail, h->hyb_rows, h->hyb_cols,
                                                        (__nv_bfloat16 *)h->hyb_vals);
        SPMV_CUDA_TRY(cudaGetLastError());
    }
    return SPMV_OK;
}

int pack_bsr(spmv_matrix *h, int r, cudaStream_t s) {
    const int64_t m = h->m, n = h->n, nnz = h->nnz;
    const int64_t mb = (m + r - 1) / r, nb = (n + r - 1) / r;
    const size_t vs = value_size(h->vt);
    h->bsr_r = r;
    h->bsr_mb = mb;
    SPMV_TRY(dalloc(&h->bsr_rowptr, (size_t)mb + 1));
    if (nnz == 0) {
        h->bsr_blocks = 0;
        SPMV_CUDA_TRY(cudaMemsetAsync(h->bsr_rowptr, 0, sizeof(int) * (mb + 1), s));
        SPMV_TRY(dalloc(&h->bsr_col, 1));
        SPMV_TRY(dalloc_bytes(&h->bsr_val, vs));
        return SPMV_OK;
    }
    const int bcbits = std::max(1, bits_for(nb));
    const int total_bits = bits_for(mb) + bcbits;
    Tmp<int> rows;
    SPMV_TRY(rows.alloc(nnz, s));
    SPMV_TRY(expand_rows(h->rowptr, m, nnz, rows.p, s));
    Tmp<uint64_t> k0, k1;
    Tmp<uint32_t> v0, v1;
    SPMV_TRY(k0.alloc(nnz, s));
    SPMV_TRY(k1.alloc(nnz, s));
    SPMV_TRY(v0.alloc(nnz, s));
    SPMV_TRY(v1.alloc(nnz, s));
    k_block_keys<<<grid1d(nnz, 256), 256, 0, s>>>(rows.p, h->colidx, nnz, r, bcbits, k0.p, v0.p);
    uint64_t *ks;
    uint32_t *vp;
    SPMV_TRY(radix_sort_pairs(k0.p, v0.p, k1.p, v1.p, nnz, total_bits, s, &ks, &vp));
    Tmp<int> head, pos;
    SPMV_TRY(head.alloc(nnz, s));
    SPMV_TRY(pos.alloc(nnz, s));
    k_heads<<<grid1d(nnz, 256), 256, 0, s>>>(ks, nnz, head.p);
    int64_t nblk = 0;
    SPMV_TRY(exclusive_scan(head.p, pos.p, nnz, s, &nblk));
    h->bsr_blocks = nblk;
    if ((double)nblk * r * r > 8.0 * (double)nnz + (double)(1 << 24)) {
        set_error("BSR: %lld blocks of %dx%d exceed 8 x nnz + 2^24 value slots", (long long)nblk, r, r);
        return SPMV_ERR_UNSUPPORTED;
    }
    SPMV_TRY(dalloc(&h->bsr_col, (size_t)nblk));
    SPMV_TRY(dalloc_bytes(&h->bsr_val, vs * nblk * r * r));
    SPMV_CUDA_TRY(cudaMemsetAsync(h->bsr_val, 0, vs * nblk * r * r, s));
    Tmp<int> brow;
    SPMV_TRY(brow.alloc(nblk, s));
    unsigned g = grid1d(nnz, 256);
    if (h->vt == SPMV_F64)
        k_bsr_fill<double><<<g, 256, 0, s>>>(ks, vp, head.p, pos.p, nnz, rows.p, h->colidx, (const double *)h->vals,
                                             r, bcbits, h->bsr_col, brow.p, (double *)h->bsr_val);
    else if (h->vt == SPMV_F32)
        k_bsr_fill<float><<<g, 256, 0, s>>>(ks, vp, head.p, pos.p, nnz, rows.p, h->colidx, (const float *)h->vals,
                                            r, bcbits, h->bsr_col, brow.p, (float *)h->bsr_val);
    else
        k_bsr_fill<__nv_bfloat16><<<g, 256, 0, s>>>(ks, vp, head.p, pos.p, nnz, rows.p, h->colidx,
                                                    (const __nv_bfloat16 *)h->vals, r, bcbits, h->bsr_col, brow.p,
                                                    (__nv_bfloat16 *)h->bsr_val);
    k_rowptr_from_sorted<<<grid1d(mb + 1, 256), 256, 0, s>>>(brow.p, nblk, mb, h->bsr_rowptr);
    SPMV_CUDA_TRY(cudaGetLastError());
    SPMV_CUDA_TRY(cudaStreamSynchronize(s));
    return SPMV_OK;
}

}  // namespace

namespace {

// kmax: columns of a slice per work item (wider slices become several items)
int pack_sell(spmv_matrix *h, int kmax, bool grouped, cudaStream_t s) {
    const int64_t m = h->m;
    const int64_t nslices = (m + 31) / 32;
    const size_t vs = value_size(h->vt);
    h->sell_nslices = nslices;
    h->sell_grouped = grouped;
    SPMV_TRY(dalloc(&h->sell_ptr, (size_t)nslices + 1));
    SPMV_TRY(dalloc(&h->sell_perm, (size_t)std::max<int64_t>(m, 1)));
    if (m == 0) {
        SPMV_CUDA_TRY(cudaMemsetAsync(h->sell_ptr, 0, sizeof(int), s));
        SPMV_TRY(dalloc(&h->sell_col, 1));
        SPMV_TRY(dalloc_bytes(&h->sell_val, vs));
        h->sell_slots = 0;
        return SPMV_OK;
    }
    // sort all rows by descending length (stable): slices group rows of
    // similar length, so padding stays small even for power-law rows
    Tmp<uint64_t> k0, k1;
    Tmp<uint32_t> v0, v1;
    SPMV_TRY(k0.alloc(m, s));
    SPMV_TRY(k1.alloc(m, s));
    SPMV_TRY(v0.alloc(m, s));
    SPMV_TRY(v1.alloc(m, s));
    k_sell_keys<<<grid1d(m, 256), 256, 0, s>>>(h->rowptr, m, k0.p, v0.p);
    uint64_t *ks;
    uint32_t *perm;
    SPMV_TRY(radix_sort_pairs(k0.p, v0.p, k1.p, v1.p, m, 32, s, &ks, &perm));
    Tmp<int> slots;
    SPMV_TRY(slots.alloc(nslices + 1, s));
    SPMV_CUDA_TRY(cudaMemsetAsync(slots.p, 0, sizeof(int) * (nslices + 1), s));
    k_sell_widths<<<grid1d(nslices, 256), 256, 0, s>>>(h->rowptr, perm, m, nslices, slots.p);
    int64_t total = 0;
    SPMV_TRY(exclusive_scan(slots.p, h->sell_ptr, nslices + 1, s, &total));
    if ((double)total > 8.0 * (double)h->nnz + (double)(1 << 24) || total >= (int64_t(1) << 31)) {
        set_error("SELL: %lld padded slots exceed min(8 x nnz + 2^24, 2^31 - 1)", (long long)total);
        return SPMV_ERR_UNSUPPORTED;
    }
    h->sell_slots = total;
    SPMV_TRY(dalloc(&h->sell_col, (size_t)total));
    SPMV_TRY(dalloc_bytes(&h->sell_val, vs * total));
    const unsigned g = grid1d(std::max<int64_t>(total, m), 256);
    if (h->vt == SPMV_F64)
        k_sell_fill<double><<<g, 256, 0, s>>>(h->rowptr, h->colidx, (const double *)h->vals, perm, m, nslices,
                                              h->sell_ptr, total, h->sell_col, (double *)h->sell_val, h->sell_perm,
                                              grouped);
    else if (h->vt == SPMV_F32)
        k_sell_fill<float><<<g, 256, 0, s>>>(h->rowptr, h->colidx, (const float *)h->vals, perm, m, nslices,
                                             h->sell_ptr, total, h->sell_col, (float *)h->sell_val, h->sell_perm,
                                             grouped);
    else
        k_sell_fill<__nv_bfloat16><<<g, 256, 0, s>>>(h->rowptr, h->colidx, (const __nv_bfloat16 *)h->vals, perm, m,
                                                     nslices, h->sell_ptr, total, h->sell_col,
                                                     (__nv_bfloat16 *)h->sell_val, h->sell_perm, grouped);
    SPMV_CUDA_TRY(cudaGetLastError());
    // work items (slice, first slot, column count <= 256) and the partials
    // joining the items of one slice
    LongRows &L = h->lng;
    Tmp<int> cnt, off;
    SPMV_TRY(cnt.alloc(nslices, s));
    SPMV_TRY(off.alloc(nslices, s));
    k_sell_item_count<<<grid1d(nslices, 256), 256, 0, s>>>(h->sell_ptr, nslices, kmax, cnt.p);
    int64_t nitems = 0;
    SPMV_TRY(exclusive_scan(cnt.p, off.p, nslices, s, &nitems));
    L.nseg = nitems;
    L.threshold = kmax;
    SPMV_TRY(dalloc(&L.seg_row, (size_t)nitems));
    SPMV_TRY(dalloc(&L.seg_begin, (size_t)nitems));
    SPMV_TRY(dalloc(&L.seg_end, (size_t)nitems));
    SPMV_TRY(dalloc(&L.seg_c0, (size_t)nitems));
    SPMV_TRY(dalloc(&L.seg_c1, (size_t)nitems));
    k_sell_item_fill<<<grid1d(nslices, 256), 256, 0, s>>>(h->sell_ptr, nslices, kmax, off.p, L.seg_row,
                                                           L.seg_begin, L.seg_end, L.seg_c0, L.seg_c1);
    SPMV_CUDA_TRY(cudaGetLastError());
    SPMV_TRY(alloc_partials(&L.part, nitems, 32, h->vt, s));
    // rows of the zero-width slices are written by a grid-stride pass
    Tmp<int> sz;
    SPMV_TRY(sz.alloc(1, s));
    k_sell_first_empty<<<1, 1, 0, s>>>(h->sell_ptr, nslices, sz.p);
    SPMV_CUDA_TRY(cudaGetLastError());
    int hz = 0;
    SPMV_CUDA_TRY(cudaMemcpyAsync(&hz, sz.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    SPMV_CUDA_TRY(cudaStreamSynchronize(s));
    L.nrows = hz;
    return SPMV_OK;
}
}  // namespace

int build_coo_meta(const int32_t *rows, const int32_t *rowptr, int64_t nnz, int C, int32_t *meta0, int32_t *meta1,
                   cudaStream_t s) {
    const int64_t nchunks = (nnz + C - 1) / C;
    if (nchunks == 0) return SPMV_OK;
    k_seg_meta_coo<<<grid1d(nchunks + 1, 256), 256, 0, s>>>(rows, rowptr, nnz, C, nchunks, meta0, meta1);
    SPMV_CUDA_TRY(cudaGetLastError());
    return SPMV_OK;
}

int build_merge_meta(const int32_t *rowptr, int64_t m, int64_t nnz, int C, int32_t *meta, cudaStream_t s) {
    const int64_t nchunks = (nnz + C - 1) / C;
    k_seg_meta_merge<<<grid1d(nchunks + 1, 256), 256, 0, s>>>(rowptr, m, C, nchunks, meta);
    SPMV_CUDA_TRY(cudaGetLastError());
    return SPMV_OK;
}

int ensure_seg_scratch(spmv_matrix *h, int items, int kind, cudaStream_t s) {
    SegScratch &g = h->seg;
    const int64_t nnz = kind != SEG_COO ? h->nnz : (h->cfg.format == SPMV_FMT_HYB ? h->hyb_nnz : h->nnz);
    const int C = 32 * items;
    const int64_t nchunks = (nnz + C - 1) / C;
    auto f = [](void *p) { if (p) cudaFree(p); };
    f(g.meta0); f(g.meta1);
    free_partials(&g.part);
    g = SegScratch{};
    g.items = items;
    g.nchunks = nchunks;
    SPMV_TRY(dalloc(&g.meta0, (size_t)nchunks + 1));
    SPMV_TRY(dalloc(&g.meta1, (size_t)nchunks + 1));
    SPMV_TRY(alloc_partials(&g.part, nchunks, 1, h->vt, s));
    if (nchunks > 0) {
        unsigned grid = grid1d(nchunks + 1, 256);
        if (kind == SEG_TILES) {
            k_seg_meta_split<<<grid, 256, 0, s>>>(h->rowptr, h->m, nnz, C, nchunks, g.meta0);
        } else if (kind == SEG_MERGE) {
            k_seg_meta_merge<<<grid, 256, 0, s>>>(h->rowptr, h->m, C, nchunks, g.meta0);
        } else if (h->cfg.format == SPMV_FMT_HYB) {
            k_seg_meta_coo<<<grid, 256, 0, s>>>(h->hyb_rows, h->hyb_ptr, nnz, C, nchunks, g.meta0, g.meta1);
        } else {
            k_seg_meta_coo<<<grid, 256, 0, s>>>(h->coo_rows, h->rowptr, nnz, C, nchunks, g.meta0, g.meta1);
        }
        SPMV_CUDA_TRY(cudaGetLastError());
    }
    return SPMV_OK;
}

int pack_format(spmv_matrix *h, const spmv_config &cfg, cudaStream_t s) {
    // a solver graph captured the old launches
    free_cg(h);
    // a change of launch parameters only (block size, register cap, carveout)
    // keeps the packed arrays
    const spmv_config &p = h->packed_req;
    if (h->packed && p.format == cfg.format && p.threads_per_row == cfg.threads_per_row &&
        p.unroll == cfg.unroll && p.bsr_block == cfg.bsr_block && p.hyb_ell_width == cfg.hyb_ell_width) {
        const int32_t width = h->cfg.hyb_ell_width;
        h->cfg = cfg;
        if (cfg.format == SPMV_FMT_HYB) h->cfg.hyb_ell_width = width;
        return SPMV_OK;
    }
    free_packed(h);
    h->packed = false;
    h->packed_req = cfg;
    h->cfg = cfg;
    const int items = 4 * (cfg.unroll > 4 ? 4 : cfg.unroll);  // COO parts: at most 16 entries per lane
    switch (cfg.format) {
    case SPMV_FMT_CSR:
        if (cfg.threads_per_row == SPMV_TPR_SPLIT) {
            // hyb_ell_width 0: warp chunks of 32 * items entries; else staged
            // tiles of hyb_ell_width nonzeros (a multiple of 256)
            if (cfg.hyb_ell_width == 0) SPMV_TRY(ensure_seg_scratch(h, items, SEG_MERGE, s));
            else SPMV_TRY(ensure_seg_scratch(h, cfg.hyb_ell_width / 32, SEG_TILES, s));
        } else {
            // rows needing more than 32 steps of their lane group go to whole blocks
            const int64_t thr = std::max<int64_t>(512, 32LL * cfg.threads_per_row * cfg.unroll);
            SPMV_TRY(build_long_rows(h, h->rowptr, h->m, thr, 4096, 1, s));
        }
        break;
    case SPMV_FMT_ELL: {
        const int64_t width = h->max_row;
        const int64_t pitch = (h->m + 31) / 32 * 32;
        if ((double)width * (double)pitch > 8.0 * (double)h->nnz + (double)(1 << 24)) {
            set_error("ELL: padded size %lld x %lld exceeds 8 x nnz + 2^24 entries", (long long)width,
                      (long long)pitch);
            return SPMV_ERR_UNSUPPORTED;
        }
        SPMV_TRY(pack_ell(h, width, false, s));
        break;
    }
    case SPMV_FMT_COO:
        SPMV_TRY(dalloc(&h->coo_rows, (size_t)h->nnz));
        SPMV_TRY(expand_rows(h->rowptr, h->m, h->nnz, h->coo_rows, s));
        SPMV_TRY(ensure_seg_scratch(h, items, SEG_COO, s));
        break;
    case SPMV_FMT_HYB: {
        int64_t width = cfg.hyb_ell_width;
        if (width <= 0) SPMV_TRY(hyb_width_rule(h, s, &width));
        width = std::min<int64_t>(width, h->max_row);
        SPMV_TRY(pack_hyb(h, width, s));
        h->cfg.hyb_ell_width = (int32_t)width;
        SPMV_TRY(ensure_seg_scratch(h, items, SEG_COO, s));
        break;
    }
    case SPMV_FMT_SELL:
        SPMV_TRY(pack_sell(h, cfg.hyb_ell_width, cfg.bsr_block == 4, s));
        break;
    case SPMV_FMT_BSR: {
        SPMV_TRY(pack_bsr(h, cfg.bsr_block, s));
        const int64_t thr = 256LL * cfg.threads_per_row;
        SPMV_TRY(build_long_rows(h, h->bsr_rowptr, h->bsr_mb, thr, 16LL * (256 / cfg.bsr_block), cfg.bsr_block, s));
        break;
    }
    default:
        set_error("unknown format %d", cfg.format);
        return SPMV_ERR_INVALID;
    }
    SPMV_CUDA_TRY(cudaStreamSynchronize(s));
    h->packed = true;
    return SPMV_OK;
}

}  // namespace spmv

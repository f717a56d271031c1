// Sparsity features on the device (Table 2, Section 5.5: n, nnz, Avg_nnz,
// Var_nnz, ELL_ratio, Median, Mode, Std_nnz) plus the selector's structural
// extras, and the fused inference kernel of the 2-layer selector MLP
// (Section 5.4: a multi-class classifier over the features).
//
// The paper extracts features on the CPU with NumPy (Section 7.5 reports
// seconds per matrix); here three kernels read the CSR arrays once:
//   k_feat_rows     row lengths: sum of squares, min, max, empty rows and a
//                   histogram of lengths;
//   k_feat_entries  per nonzero, in equal chunks of nonzeros: |i - j| (max
//                   and sum), diagonal entries and whether the entry opens a
//                   new 2x2 / 4x4 block;
//   k_feat_finish   one block: median, mode, Gini and the HYB width from the
//                   histogram, then the 20 feature values.
// Counts are exact 64-bit integers; ratios are formed once at the end.
#include <cmath>

#include "internal.cuh"

namespace spmv {

namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o);
    return v;  // valid in lane 0
}

struct FeatAcc {
    unsigned long long sum_len2;   // sum of squared row lengths
    unsigned long long empty;      // rows of length 0
    unsigned long long sum_dist;   // sum |i - j|
    unsigned long long diag;       // entries with i == j
    unsigned long long blocks4;    // nonempty 4x4 blocks
    unsigned long long blocks2;    // nonempty 2x2 blocks
    int min_len, max_len, max_dist, pad;
};

__global__ void k_feat_init(FeatAcc *acc) {
    acc->sum_len2 = acc->empty = acc->sum_dist = acc->diag = acc->blocks4 = acc->blocks2 = 0ull;
    acc->min_len = 0x7fffffff;
    acc->max_len = 0;
    acc->max_dist = 0;
}

__global__ void k_feat_rows(const int *rowptr, int64_t m, unsigned *hist, FeatAcc *acc) {
    unsigned long long s2 = 0, emp = 0;
    int mn = 0x7fffffff, mx = 0;
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t mr = (m + 31) / 32 * 32;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < mr; r += stride) {
        const bool valid = r < m;
        const int len = valid ? rowptr[r + 1] - rowptr[r] : -1;
        if (valid) {
            s2 += (unsigned long long)len * (unsigned long long)len;
            emp += len == 0;
            mn = min(mn, len);
            mx = max(mx, len);
        }
        const unsigned peers = __match_any_sync(FULL, len);
        if (valid && lane == 31 - __clz(peers)) atomicAdd(hist + len, (unsigned)__popc(peers));
    }
    s2 = warp_sum_u64(s2);
    emp = warp_sum_u64(emp);
    mn = __reduce_min_sync(FULL, mn);
    mx = __reduce_max_sync(FULL, mx);
    if (lane == 0) {
        atomicAdd(&acc->sum_len2, s2);
        atomicAdd(&acc->empty, emp);
        atomicMin(&acc->min_len, mn);
        atomicMax(&acc->max_len, mx);
    }
}

// first column position >= c in the sorted column list [b, e)
__device__ __forceinline__ int lower_col(const int *colidx, int b, int e, int c) {
    while (b < e) {
        const int mid = b + ((e - b) >> 1);  // b + e overflows int past 2^30 offsets
        if (colidx[mid] < c) b = mid + 1; else e = mid;
    }
    return b;
}

// does any of rows [r0, i) hold a column in [c0, c0 + w)?
__device__ __forceinline__ bool earlier_rows_hit(const int *rowptr, const int *colidx, int64_t r0, int64_t i,
                                                 int c0, int w) {
    for (int64_t q = r0; q < i; ++q) {
        const int b = rowptr[q], e = rowptr[q + 1];
        const int p = lower_col(colidx, b, e, c0);
        if (p < e && colidx[p] < c0 + w) return true;
    }
    return false;
}

// largest r in [lo, hi] with rowptr[r] <= k (the row holding entry k)
__device__ __forceinline__ int64_t row_in(const int *rowptr, int64_t lo, int64_t hi, int64_t k) {
    while (lo < hi) {
        const int64_t mid = lo + ((hi - lo + 1) >> 1);
        if (rowptr[mid] <= k) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Nonzero chunks of FEAT_CHUNK entries, one warp each, so a power-law row
// costs no more than the same number of entries in short rows: lane 0 finds
// the rows of the chunk's first and last entries, every lane then finds the
// row of each of its entries by a binary search between them.  Per entry:
// |i - j|, the diagonal, and whether the entry opens a new r x r block (no
// earlier entry of its block: neither the previous entry of its own row nor
// an entry of an earlier row of the same block row).
// row0: the global index of local row 0 (a multiple of 4 for row panels)
constexpr int FEAT_CHUNK = 256;

__global__ void k_feat_entries(const int *rowptr, const int *colidx, int64_t m, int64_t nnz, int64_t row0,
                               FeatAcc *acc) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nchunks = (nnz + FEAT_CHUNK - 1) / FEAT_CHUNK;
    unsigned long long sd = 0, dg = 0, b4 = 0, b2 = 0;
    int md = 0;
    for (int64_t c = warp; c < nchunks; c += nwarps) {
        const int64_t k0 = c * FEAT_CHUNK, k1 = k0 + FEAT_CHUNK < nnz ? k0 + FEAT_CHUNK : nnz;
        int64_t r0 = 0, r1 = 0;
        if (lane == 0) {
            r0 = row_in(rowptr, 0, m - 1, k0);
            r1 = row_in(rowptr, r0, m - 1, k1 - 1);
        }
        r0 = __shfl_sync(FULL, r0, 0);
        r1 = __shfl_sync(FULL, r1, 0);
        for (int64_t k = k0 + lane; k < k1; k += 32) {
            const int64_t i = row_in(rowptr, r0, r1, k);
            const int b = rowptr[i];
            const int j = colidx[k];
            const int64_t gi = row0 + i;
            const int64_t d = gi > j ? gi - j : j - gi;
            sd += (unsigned long long)d;
            md = max(md, (int)d);
            dg += d == 0;
            const int prev = k > b ? colidx[k - 1] : -1;
            if (prev < 0 || prev / 4 != j / 4) b4 += !earlier_rows_hit(rowptr, colidx, i / 4 * 4, i, j / 4 * 4, 4);
            if (prev < 0 || prev / 2 != j / 2) b2 += !earlier_rows_hit(rowptr, colidx, i / 2 * 2, i, j / 2 * 2, 2);
        }
    }
    sd = warp_sum_u64(sd);
    dg = warp_sum_u64(dg);
    b4 = warp_sum_u64(b4);
    b2 = warp_sum_u64(b2);
    md = __reduce_max_sync(FULL, md);
    if (lane == 0) {
        atomicAdd(&acc->sum_dist, sd);
        atomicAdd(&acc->diag, dg);
        atomicAdd(&acc->blocks4, b4);
        atomicAdd(&acc->blocks2, b2);
        atomicMax(&acc->max_dist, md);
    }
}

constexpr int FIN_THREADS = 1024;

__device__ long long block_sum_ll(long long v, long long *sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o);
    if (lane == 0) sh[w] = v;
    __syncthreads();
    long long t = 0;
    if (threadIdx.x == 0)
        for (int k = 0; k < FIN_THREADS / 32; ++k) t += sh[k];
    __syncthreads();
    if (threadIdx.x == 0) sh[0] = t;
    __syncthreads();
    t = sh[0];
    __syncthreads();
    return t;
}

// Single block over the histogram h[0..maxlen]: P(L) = #rows shorter than L.
__global__ void __launch_bounds__(FIN_THREADS)
k_feat_finish(const unsigned *hist, int maxlen, int64_t m, int64_t n, int64_t nnz, const FeatAcc *acc,
              double *out) {
    __shared__ long long sh[FIN_THREADS / 32];
    __shared__ long long carry;
    __shared__ long long median_s;
    __shared__ unsigned long long mode_key_s, K_s;
    if (threadIdx.x == 0) {
        carry = 0;
        median_s = 0;
        mode_key_s = 0ull;
        K_s = 0ull;
    }
    __syncthreads();
    const long long target = (m - 1) / 2;  // 0-based index of the lower middle
    long long gini_num = 0;
    for (int base = 0; base <= maxlen; base += FIN_THREADS) {
        const int L = base + threadIdx.x;
        const long long h = L <= maxlen ? (long long)hist[L] : 0;
        // exclusive prefix over this chunk (warp shuffles + shared totals)
        long long incl = h;
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        for (int o = 1; o < 32; o <<= 1) {
            const long long t = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) sh[w] = incl;
        __syncthreads();
        long long wpre = 0;
        for (int k = 0; k < w; ++k) wpre += sh[k];
        const long long P = carry + wpre + incl - h;  // rows shorter than L
        __syncthreads();
        if (L <= maxlen) {
            if (h > 0 && P <= target && target < P + h) median_s = L;
            if (h > 0) {
                // mode: largest count, smallest length on ties (64-bit key)
                const unsigned long long key = ((unsigned long long)h << 32) | (unsigned)(0x7fffffff - L);
                atomicMax(&mode_key_s, key);
            }
            gini_num += (long long)L * h * (2 * P + h - m);
            // HYB width: rows with length >= L is m - P
            const long long ge = m - P;
            if (L >= 1 && ge >= 4096 && 3 * ge >= m) atomicMax(&K_s, (unsigned long long)L);
        }
        __syncthreads();
        if (threadIdx.x == FIN_THREADS - 1) carry = P + h;
        __syncthreads();
    }
    gini_num = block_sum_ll(gini_num, sh);
    const long long K = (long long)K_s;
    long long tail = 0;
    for (int L = threadIdx.x; L <= maxlen; L += FIN_THREADS)
        if (L > K) tail += (long long)(L - K) * hist[L];
    tail = block_sum_ll(tail, sh);
    if (threadIdx.x == 0) {
        const double md = (double)m, nd = (double)n, zd = (double)nnz;
        const double mean = m ? zd / md : 0.0;
        // population variance from the exact integer numerator sum(l^2) m - nnz^2
        const __int128 num = (__int128)acc->sum_len2 * m - (__int128)nnz * nnz;
        const double var = m ? (double)num / (md * md) : 0.0;
        const double sd = sqrt(var > 0 ? var : 0.0);
        const long long mode_len = mode_key_s ? 0x7fffffff - (long long)(mode_key_s & 0xffffffffull) : 0;
        out[0] = md;
        out[1] = zd;
        out[2] = (m && n) ? zd / (md * nd) : 0.0;
        out[3] = mean;
        out[4] = var;
        out[5] = sd;
        out[6] = m ? (double)acc->min_len : 0.0;
        out[7] = (double)acc->max_len;
        out[8] = (double)median_s;
        out[9] = (double)mode_len;
        out[10] = (m && acc->max_len) ? zd / (md * (double)acc->max_len) : 0.0;
        out[11] = (m && nnz) ? (double)gini_num / (md * zd) : 0.0;
        out[12] = mean > 0 ? sd / mean : 0.0;
        out[13] = m ? (double)acc->empty / md : 0.0;
        out[14] = (double)acc->max_dist;
        out[15] = nnz ? (double)acc->sum_dist / zd : 0.0;
        out[16] = nnz ? (double)acc->diag / zd : 0.0;
        out[17] = nnz ? zd / (16.0 * (double)acc->blocks4) : 0.0;
        out[18] = nnz ? zd / (4.0 * (double)acc->blocks2) : 0.0;
        out[19] = nnz ? (double)tail / zd : 0.0;
    }
}

}  // namespace

// Features of the handle's matrix into d_out[SPMV_NUM_FEATURES] (device).
int compute_features(const spmv_matrix *h, double *d_out, cudaStream_t s) {
    const int64_t m = h->m;
    const int maxlen = (int)h->max_row;
    void *buf = nullptr;
    const size_t hist_bytes = sizeof(unsigned) * ((size_t)maxlen + 1);
    SPMV_CUDA_TRY(dev_malloc_async(&buf, hist_bytes + 256, s));
    unsigned *hist = static_cast<unsigned *>(buf);
    FeatAcc *acc = reinterpret_cast<FeatAcc *>(static_cast<char *>(buf) + (hist_bytes + 127) / 128 * 128);
    int st = SPMV_OK;
    cudaError_t e = cudaMemsetAsync(hist, 0, hist_bytes, s);
    if (e == cudaSuccess) {
        k_feat_init<<<1, 1, 0, s>>>(acc);
        // a matrix held in row panels accumulates every panel into one set
        const int np = h->npanels > 0 ? h->npanels : 1;
        for (int p = 0; p < np; ++p) {
            const spmv_matrix *q = h->npanels > 0 ? h->panels[p] : h;
            const int64_t row0 = h->npanels > 0 ? h->panel_row0[p] : 0;
            const int64_t mq = q->m;
            if (mq == 0) continue;
            const int64_t blocks = (mq + 255) / 256;
            k_feat_rows<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(q->rowptr, mq, hist, acc);
            const int64_t wblocks = ((q->nnz + FEAT_CHUNK - 1) / FEAT_CHUNK + 7) / 8;
            if (wblocks > 0)
                k_feat_entries<<<(unsigned)(wblocks < 8192 ? wblocks : 8192), 256, 0, s>>>(q->rowptr, q->colidx, mq,
                                                                                            q->nnz, row0, acc);
        }
        k_feat_finish<<<1, FIN_THREADS, 0, s>>>(hist, maxlen, m, h->n, h->nnz, acc, d_out);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) st = cuda_status(e, "feature kernels");
    cudaFreeAsync(buf, s);
    return st;
}

}  // namespace spmv

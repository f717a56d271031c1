// Nonzero-balanced SpMV kernels: COO (segmented reduction over row-sorted
// triplets), the COO part of HYB (accumulating into y), and split CSR
// (fixed nonzero chunks whose rows are recovered from the row pointers).
//
// All three cut the nonzeros into chunks of 32*ITEMS entries, one warp per
// chunk and ITEMS consecutive entries per lane, so a power-law row (the load
// imbalance the paper notes for CSR in Section 2.3) costs no more than the
// same number of nonzeros spread over short rows.  Each lane sums its runs
// of equal rows sequentially, a shuffle-based segmented scan joins runs
// that cross lanes, and a row that crosses chunks is finished by whichever
// of its chunks arrives last (an atomic counter per row, no waiting): that
// warp adds the chunks' partial sums in chunk order, so results do not
// depend on scheduling.  Counters reset themselves for the next product.
#pragma once

#include <climits>

#include "combine.cuh"

namespace spmv {

template <typename T, bool ACCUM>
__device__ __forceinline__ void seg_write(T *y, int64_t row, T acc, const Epi<T> &ep) {
    if (ACCUM) ep.add(y, row, acc);  // HYB: the ELL pass already wrote alpha*Ax_ell + beta*y
    else ep.store(y, row, acc);
}

// Chunk c adds `contrib` for a row spanning chunks c0..c1; the arrival that
// completes the row writes y.
template <typename T, bool ACCUM>
__device__ __forceinline__ void seg_arrive(int64_t row, int64_t c, int64_t c0, int64_t c1, T contrib,
                                           const PartialsT<T> &P, T *y, const Epi<T> &ep) {
    T total;
    if (join_partial<T>(c, c0, c1, 0, contrib, P, &total)) seg_write<T, ACCUM>(y, row, total, ep);
}

// Loads ITEMS consecutive entries of lane range [a, a+cnt): values, the
// gathered x entries and (for COO) rows.  Full chunks use 16-byte vector
// loads.  Products are formed later by one fused multiply-add per entry.
template <typename V, typename T, int ITEMS, bool HAS_ROWS>
__device__ __forceinline__ void seg_load(bool full, int64_t a, int cnt, const int *rows, const int *cols,
                                         const V *vals, const T *x, int (&r)[ITEMS], T (&v)[ITEMS],
                                         T (&xv)[ITEMS]) {
    if (full) {
        int cc[ITEMS];
        if (HAS_ROWS) ld_idx_vec<ITEMS>(rows + a, r);
        ld_idx_vec<ITEMS>(cols + a, cc);
        ld_vals_vec<ITEMS>(vals + a, v);
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) xv[j] = ld_x(x, cc[j]);
    } else {
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            if (j < cnt) {
                if (HAS_ROWS) r[j] = ld_s(rows + a + j);
                v[j] = ld_val(vals + a + j);
                xv[j] = ld_x(x, ld_s(cols + a + j));
            } else {
                if (HAS_ROWS) r[j] = INT_MAX;
                v[j] = T(0);
                xv[j] = T(0);
            }
        }
    }
}

// Inclusive segmented scan over lanes keyed by a nondecreasing row id.  A
// step whose add no lane needs (no run of equal keys that long) is skipped
// by a warp vote, so short rows pay no floating-point adds here.
template <typename T>
__device__ __forceinline__ T seg_scan(int key, T val) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int k = __shfl_up_sync(0xffffffffu, key, d);
        const bool need = lane >= d && k == key;
        if (!__any_sync(0xffffffffu, need)) break;   // runs are contiguous: longer steps add nothing
        const T v = __shfl_up_sync(0xffffffffu, val, d);
        if (need) val += v;
    }
    return val;
}

// Lane carry: a lane whose first row continues from the previous lane adds
// that lane's scanned run; the add is issued only if some lane needs it.
template <typename T>
__device__ __forceinline__ T seg_carry(bool need, T fs, T pval) {
    if (__any_sync(0xffffffffu, need)) return need ? fs + pval : fs;
    return fs;
}

// ---------------------------------------------------------------------------
// COO (ACCUM = false) and the COO part of HYB (ACCUM = true).
// meta0[c] = first chunk of the row of entry c*C; meta1[c] = last chunk of
// the row of the chunk's last entry.
// ---------------------------------------------------------------------------
// 16 items per lane need more than 64 registers: those variants are limited
// to 512-thread blocks.
template <typename V, typename T, int ITEMS, bool ACCUM>
__global__ void __launch_bounds__(ITEMS >= 16 ? 512 : 1024)
k_coo_seg(int64_t nnz, int64_t m, const int *__restrict__ rows, const int *__restrict__ cols,
          const V *__restrict__ vals, const T *__restrict__ x, T *__restrict__ y, T alpha, T beta,
          const int *__restrict__ meta0, const int *__restrict__ meta1, const PartialsT<T> P) {
    const Epi<T> ep(alpha, beta);
    constexpr int C = 32 * ITEMS;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nchunks = (nnz + C - 1) / C;
    for (int64_t c = warp; c < nchunks; c += nwarps) {
        const int64_t E0 = c * C, E1 = (E0 + C < nnz) ? E0 + C : nnz;
        const int64_t a = E0 + (int64_t)lane * ITEMS;
        const int cnt = E1 - a <= 0 ? 0 : (E1 - a >= ITEMS ? ITEMS : (int)(E1 - a));
        const int last_lane = (int)((E1 - E0 - 1) / ITEMS);
        int r[ITEMS];
        T v[ITEMS], xv[ITEMS];
        seg_load<V, T, ITEMS, true>(E1 - E0 == C, a, cnt, rows, cols, vals, x, r, v, xv);

        // row after this lane's range: next lane's first row, or the next
        // chunk's first row (m past the last entry)
        int nr = __shfl_down_sync(0xffffffffu, r[0], 1);
        if (lane == last_lane) nr = E1 < nnz ? ld_s(rows + E1) : (int)m;
        if (!ACCUM && c == 0 && lane == 0)
            for (int q = 0; q < r[0]; ++q) seg_write<T, false>(y, q, T(0), ep);

        int fr = r[0], cur = r[0];
        T fs = T(0), acc = T(0);
        bool fflush = false;
        if (cnt > 0) {
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) {
                if (j < cnt) {
                    if (r[j] != cur) {
                        if (!fflush) { fs = acc; fflush = true; }
                        else seg_write<T, ACCUM>(y, cur, acc, ep);
                        if (!ACCUM)
                            for (int q = cur + 1; q < r[j]; ++q) seg_write<T, false>(y, q, T(0), ep);
                        cur = r[j];
                        acc = T(0);
                    }
                    acc = fma(v[j], xv[j], acc);
                }
            }
            if (nr != cur) {  // the last row ends exactly at the lane's end
                if (!fflush) { fs = acc; fflush = true; }
                else seg_write<T, ACCUM>(y, cur, acc, ep);
                if (!ACCUM)
                    for (int q = cur + 1; q < nr; ++q) seg_write<T, false>(y, q, T(0), ep);
                cur = nr;
                acc = T(0);
            }
        }
        const int key = cnt > 0 ? cur : -1;
        const T sc = seg_scan<T>(key, cnt > 0 ? acc : T(0));
        const int pkey = __shfl_up_sync(0xffffffffu, key, 1);
        const T pval = __shfl_up_sync(0xffffffffu, sc, 1);
        const int H = __shfl_sync(0xffffffffu, r[0], 0);
        const int64_t hc0 = meta0[c], tc1 = meta1[c];
        const bool h_back = hc0 < c, t_fwd = tc1 > c;
        const T total = seg_carry<T>(cnt > 0 && fflush && lane > 0 && pkey == fr, fs, pval);
        if (cnt > 0 && fflush) {
            if (fr == H && h_back)  // H started in an earlier chunk and ends in this one
                seg_arrive<T, ACCUM>(fr, c, hc0, c, total, P, y, ep);
            else
                seg_write<T, ACCUM>(y, fr, total, ep);
        }
        if (lane == last_lane && t_fwd) {
            // the open row at the chunk end (cur == nr) continues into the next chunk
            const int64_t c0 = (cur == H && h_back) ? hc0 : c;
            seg_arrive<T, ACCUM>(cur, c, c0, tc1, sc, P, y, ep);
        }
    }
}

// ---------------------------------------------------------------------------
// Split CSR: chunks of C nonzeros; meta0[c] = row holding entry c*C,
// meta0[nchunks] = m-1.  Lanes find their start row by binary search in the
// row pointers and walk them, so empty rows are written on the way.
// csr_split_chunk processes chunk c with the whole warp; k_csr_split runs
// it over all chunks, the batched kernel over its work list.
// ---------------------------------------------------------------------------
template <typename V, typename T, int ITEMS>
__device__ __forceinline__ void csr_split_chunk(int64_t c, int64_t nnz, int64_t m, const int *__restrict__ rowptr,
                                                const int *__restrict__ cols, const V *__restrict__ vals,
                                                const T *__restrict__ x, T *__restrict__ y, const Epi<T> &ep,
                                                const int *__restrict__ meta0, const PartialsT<T> &P) {
    constexpr int C = 32 * ITEMS;
    const int lane = threadIdx.x & 31;
    const int64_t E0 = c * C, E1 = (E0 + C < nnz) ? E0 + C : nnz;
    const int64_t a = E0 + (int64_t)lane * ITEMS;
    const int cnt = E1 - a <= 0 ? 0 : (E1 - a >= ITEMS ? ITEMS : (int)(E1 - a));
    const int last_lane = (int)((E1 - E0 - 1) / ITEMS);
    int r_unused[ITEMS];
    T v[ITEMS], xv[ITEMS];
    seg_load<V, T, ITEMS, false>(E1 - E0 == C, a, cnt, nullptr, cols, vals, x, r_unused, v, xv);
    const int H = __ldg(meta0 + c);
    // Row pointers rowptr[H .. H+32] of the chunk's first rows, staged per
    // warp in shared memory with one coalesced load: the start-row search
    // and the walk over short or empty rows read them from there.
    __shared__ int s_win[32][33];
    int *win = s_win[threadIdx.x >> 5];
    __syncwarp();  // the previous chunk's reads of the window are done
    if ((int64_t)H + lane <= m) win[lane] = __ldg(rowptr + H + lane);
    if (lane == 0 && (int64_t)H + 32 <= m) win[32] = __ldg(rowptr + H + 32);
    __syncwarp();
    // rows before H (the empty rows that lane 0 of chunk 0 walks from row 0)
    // and rows past the window come from global memory
    auto rp = [&](int64_t r) -> int {
        const int64_t d = r - H;
        return d >= 0 && d <= 32 ? win[d] : __ldg(rowptr + r);
    };
    int cur = 0;
    if (cnt > 0 && a > 0) {  // largest row r in [H, H_next] with rowptr[r] <= a
        int lo = H, hi = __ldg(meta0 + c + 1);
        while (lo < hi) {
            const int mid = lo + ((hi - lo + 1) >> 1);  // lo + hi overflows int past 2^30 rows
            if (rp(mid) <= a) lo = mid; else hi = mid - 1;
        }
        cur = lo;
    }
    const int fr = cur;
    int next_end = cnt > 0 ? rp(cur + 1) : 0;
    T fs = T(0), acc = T(0);
    bool fflush = false;
    if (cnt > 0) {
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            if (j < cnt) {
                while (a + j >= next_end) {
                    if (!fflush) { fs = acc; fflush = true; }
                    else seg_write<T, false>(y, cur, acc, ep);
                    acc = T(0);
                    ++cur;
                    next_end = rp(cur + 1);
                }
                acc = fma(v[j], xv[j], acc);
            }
        }
        const int64_t b = a + cnt;
        while (cur < m && next_end <= b) {
            if (!fflush) { fs = acc; fflush = true; }
            else seg_write<T, false>(y, cur, acc, ep);
            acc = T(0);
            ++cur;
            if (cur < m) next_end = rp(cur + 1);
        }
    }
    const int key = (cnt > 0 && cur < m) ? cur : -1;
    const T sc = seg_scan<T>(key, key >= 0 ? acc : T(0));
    const int pkey = __shfl_up_sync(0xffffffffu, key, 1);
    const T pval = __shfl_up_sync(0xffffffffu, sc, 1);
    const int hstart = rp(H);
    const bool h_back = hstart < E0;
    const T total = seg_carry<T>(cnt > 0 && fflush && lane > 0 && pkey == fr, fs, pval);
    if (cnt > 0 && fflush) {
        if (fr == H && h_back) {
            const int64_t c0 = hstart / C, c1 = (rp(H + 1) - 1) / C;
            seg_arrive<T, false>(fr, c, c0, c1, total, P, y, ep);
        } else {
            seg_write<T, false>(y, fr, total, ep);
        }
    }
    if (lane == last_lane && cur < m) {
        const int s0 = rp(cur);
        if (s0 < E1 && next_end > E1) {  // open row continues into the next chunk
            const int64_t c0 = s0 / C, c1 = (next_end - 1) / C;
            seg_arrive<T, false>(cur, c, c0, c1, sc, P, y, ep);
        }
    }
}

template <typename V, typename T, int ITEMS>
__global__ void __launch_bounds__(ITEMS >= 16 ? 512 : 1024)
k_csr_split(int64_t nnz, int64_t m, const int *__restrict__ rowptr, const int *__restrict__ cols,
            const V *__restrict__ vals, const T *__restrict__ x, T *__restrict__ y, T alpha, T beta,
            const int *__restrict__ meta0, const PartialsT<T> P) {
    const Epi<T> ep(alpha, beta);
    constexpr int C = 32 * ITEMS;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nchunks = (nnz + C - 1) / C;
    for (int64_t c = warp; c < nchunks; c += nwarps)
        csr_split_chunk<V, T, ITEMS>(c, nnz, m, rowptr, cols, vals, x, y, ep, meta0, P);
}

}  // namespace spmv

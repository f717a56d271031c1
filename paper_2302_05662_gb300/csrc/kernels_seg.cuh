// Nonzero-balanced SpMV kernels: COO (segmented reduction over row-sorted
// triplets), the COO part of HYB (accumulating into y), and split CSR in two
// forms -- warp chunks whose rows are recovered by merging the row pointers
// with the chunk's positions, and nonzero tiles staged through shared memory
// by bulk copies.
//
// COO and the warp chunks cut the nonzeros into chunks of 32*ITEMS entries,
// one warp per chunk and ITEMS consecutive entries per lane, so a power-law
// row (the load imbalance the paper notes for CSR in Section 2.3) costs no
// more than the same number of nonzeros spread over short rows.  Each lane
// sums its runs of equal rows sequentially, a shuffle-based segmented scan
// joins runs that cross lanes, and a row that crosses chunks is finished by
// whichever of its chunks arrives last (an atomic counter per row, no
// waiting): that warp adds the chunks' partial sums in chunk order, so
// results do not depend on scheduling.  Counters reset themselves for the
// next product.
#pragma once

#include <climits>

#include "bulk.cuh"
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
// loads, or 32-byte loads with WIDE (arrays the library allocated, whose
// chunks start on 32-byte boundaries).  Products are formed later by one
// fused multiply-add per entry.
template <typename V, typename T, int ITEMS, bool HAS_ROWS, bool WIDE = false>
__device__ __forceinline__ void seg_load(bool full, int64_t a, int cnt, const int *rows, const int *cols,
                                         const V *vals, const T *x, int (&r)[ITEMS], T (&v)[ITEMS],
                                         T (&xv)[ITEMS]) {
    if (full) {
        int cc[ITEMS];
        if (HAS_ROWS) ld_idx_vec<ITEMS, WIDE>(rows + a, r);
        ld_idx_vec<ITEMS, WIDE>(cols + a, cc);
        ld_vals_vec<ITEMS, WIDE>(vals + a, v);
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
// One COO chunk c (ACCUM: the COO part of HYB, adding into y); the whole
// warp calls it.  WIDE: 32-byte loads (the handle's own arrays); the
// allocation-free entry point runs on caller arrays aligned to 16 bytes only.
template <typename V, typename T, int ITEMS, bool ACCUM, bool WIDE>
__device__ __forceinline__ void coo_chunk(int64_t c, int64_t nnz, int64_t m, const int *__restrict__ rows,
                                          const int *__restrict__ cols, const V *__restrict__ vals,
                                          const T *__restrict__ x, T *__restrict__ y, const Epi<T> &ep,
                                          const int *__restrict__ meta0, const int *__restrict__ meta1,
                                          const PartialsT<T> &P) {
    constexpr int C = 32 * ITEMS;
    const int lane = threadIdx.x & 31;
    const int64_t E0 = c * C, E1 = (E0 + C < nnz) ? E0 + C : nnz;
    const int64_t a = E0 + (int64_t)lane * ITEMS;
    const int cnt = E1 - a <= 0 ? 0 : (E1 - a >= ITEMS ? ITEMS : (int)(E1 - a));
    const int last_lane = (int)((E1 - E0 - 1) / ITEMS);
    int r[ITEMS];
    T v[ITEMS], xv[ITEMS];
    seg_load<V, T, ITEMS, true, WIDE>(E1 - E0 == C, a, cnt, rows, cols, vals, x, r, v, xv);

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

// 16 items per lane need more than 64 registers: those variants are limited
// to 512-thread blocks.
template <typename V, typename T, int ITEMS, bool ACCUM, bool WIDE = false>
__global__ void __launch_bounds__(ITEMS >= 16 ? 512 : 1024) __maxnreg__(ITEMS >= 16 ? 128 : 64)
k_coo_seg(int64_t nnz, int64_t m, const int *__restrict__ rows, const int *__restrict__ cols,
          const V *__restrict__ vals, const T *__restrict__ x, T *__restrict__ y, T alpha, T beta,
          const int *__restrict__ meta0, const int *__restrict__ meta1, const PartialsT<T> P) {
    const Epi<T> ep(alpha, beta);
    constexpr int C = 32 * ITEMS;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nchunks = (nnz + C - 1) / C;
    for (int64_t c = warp; c < nchunks; c += nwarps)
        coo_chunk<V, T, ITEMS, ACCUM, WIDE>(c, nnz, m, rows, cols, vals, x, y, ep, meta0, meta1, P);
}

// ---------------------------------------------------------------------------
// Nonzero tiles staged through shared memory (the nnz-balanced CSR kernel).
// Tile t holds the nonzeros [t TILE, (t+1) TILE); a thread block takes tiles
// t = blockIdx.x, + gridDim.x, ..., with two shared-memory stages: while it
// multiplies one tile, the copy engine brings the block's next tile (column
// indices and values, one bulk copy each) into the other stage.  Inside a
// tile, groups of TPR lanes take the tile's rows, each lane summing a strided
// part of its row from shared memory with one fused multiply-add per entry
// (UNROLL x gathers in flight) and the group adding its lanes' sums -- the
// row-sequential accumulation that keeps fp64 instructions at one per
// nonzero, with the loads of the row-major CSR arrays made contiguous by the
// bulk copies.  A row cut by a tile boundary is joined in tile order through
// the partials; a row segment longer than `long_len` is summed by the whole
// block after the groups finish.  meta0[t] = row holding entry t TILE,
// meta0[ntiles] = m - 1.  The column and value arrays must be readable up to
// the next multiple of 8 entries past nnz (their allocations are padded).
// ---------------------------------------------------------------------------
struct TileSmem {
    int stage_bytes, cols_off, vals_off, rows_off, hdr_off, bar_off, list_off, med_off, red_off, total;
};

// row segments per tile handed to whole warps (longer than a lane group
// should sum alone, shorter than the block-wide threshold); a tile whose
// medium segments overflow the list sends the rest to the block-wide pass
constexpr int TILE_MED = 256;

// Rows of a tile whose row pointers are staged with it: at most TILE_ROWS + 1
// pointers (a tile with more rows, i.e. many empty rows, reads them from
// global memory instead).
constexpr int TILE_ROWS = 1024;

template <typename V>
__host__ __device__ inline TileSmem tile_smem_layout(int tile, int long_max) {
    TileSmem L;
    const int cb = (tile * 4 + 127) / 128 * 128;
    const int vb = (tile * (int)sizeof(V) + 127) / 128 * 128;
    const int rb = ((TILE_ROWS + 8) * 4 + 127) / 128 * 128;
    L.cols_off = 0;
    L.vals_off = cb;
    L.rows_off = cb + vb;
    L.hdr_off = cb + vb + rb;                      // per stage: first row, last row, window base, staged
    L.stage_bytes = L.hdr_off + 128;
    L.bar_off = 2 * L.stage_bytes;                 // two stages, then 2 mbarriers
    L.list_off = L.bar_off + 16;                   // long segments: int4 (row, begin, end, -) + count
    L.med_off = L.list_off + 16 * long_max + 16;   // medium segments: int4 x TILE_MED + count
    L.red_off = L.med_off + 16 * TILE_MED + 16;    // block reduction scratch: 32 doubles
    L.total = L.red_off + 32 * 8;
    return L;
}

template <typename V, typename T, int TPR, int UNROLL>
__global__ void __launch_bounds__(1024)
k_csr_tiles(int64_t nnz, int64_t m, int64_t ntiles, int tile, int long_len, int long_max,
            const int *__restrict__ rowptr, const int *__restrict__ cols, const V *__restrict__ vals,
            const T *__restrict__ x, T *__restrict__ y, T alpha, T beta, const int *__restrict__ meta0,
            const PartialsT<T> P, unsigned *status) {
    extern __shared__ __align__(128) unsigned char smem[];
    const TileSmem L = tile_smem_layout<V>(tile, long_max);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + L.bar_off);
    int4 *list = reinterpret_cast<int4 *>(smem + L.list_off);
    int *nlist = reinterpret_cast<int *>(smem + L.list_off + 16 * long_max);
    int4 *med = reinterpret_cast<int4 *>(smem + L.med_off);
    int *nmed = reinterpret_cast<int *>(smem + L.med_off + 16 * TILE_MED);
    T *red = reinterpret_cast<T *>(smem + L.red_off);
    const Epi<T> ep(alpha, beta);
    const int tid = threadIdx.x, lane = tid & 31;
    const int G = blockDim.x / TPR, g = tid / TPR, sub = tid % TPR;
    const unsigned gmask = TPR == 32 ? 0xffffffffu : (((1u << TPR) - 1u) << (lane / TPR * TPR));

    // tile t's first and last rows (meta0 holds the row of entry t*tile)
    auto first_row = [&](int64_t t) -> int { return t == 0 ? 0 : __ldg(meta0 + t); };
    // one thread issues the copies of tile t (rows rb..re) into a stage: the
    // column indices and values of its nonzeros, the row pointers of its
    // rows (16-byte aligned window) when they fit, and a header the
    // barrier's completion publishes with them
    auto issue = [&](int64_t t, int st, int rb, int re) {
        const int64_t e0 = t * tile;
        const int64_t cnt = (e0 + tile < nnz ? tile : nnz - e0);
        const unsigned n8 = (unsigned)((cnt + 7) & ~int64_t(7));
        unsigned char *base = smem + st * L.stage_bytes;
        const int w0 = rb & ~3;
        const unsigned nw = (unsigned)((re + 2 - w0 + 3) & ~3);
        const bool staged = nw <= (unsigned)(TILE_ROWS + 8);
        int *hdr = reinterpret_cast<int *>(base + L.hdr_off);
        hdr[0] = rb;
        hdr[1] = re;
        hdr[2] = w0;
        hdr[3] = staged;
        const unsigned bytes = n8 * 4u + n8 * (unsigned)sizeof(V) + (staged ? nw * 4u : 0u);
        mbar_arrive_expect_tx(bar + st, bytes);
        bulk_copy_g2s(base + L.cols_off, cols + e0, n8 * 4u, bar + st);
        bulk_copy_g2s(base + L.vals_off, vals + e0, n8 * (unsigned)sizeof(V), bar + st);
        if (staged) bulk_copy_g2s(base + L.rows_off, rowptr + w0, nw * 4u, bar + st);
    };
    if (tid == 0) {
        mbar_init(bar, 1);
        mbar_init(bar + 1, 1);
        *nlist = 0;
        *nmed = 0;
        mbar_init_fence();
    }
    __syncthreads();
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            const int64_t t = blockIdx.x + (int64_t)i * gridDim.x;
            if (t < ntiles) issue(t, i, first_row(t), __ldg(meta0 + t + 1));
        }
    }
    int k = 0;  // tiles this block has taken
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
        const int st = k & 1;
        // rows of the block's tile after next, fetched now, used when its
        // copies are issued at the end of this tile
        const int64_t tn = t + 2 * (int64_t)gridDim.x;
        int nrb = 0, nre = 0;
        if (tid == 0 && tn < ntiles) {
            nrb = first_row(tn);
            nre = __ldg(meta0 + tn + 1);
        }
        const bool ok = mbar_wait_bounded(bar + st, (unsigned)(k >> 1) & 1u, MBAR_WAIT_NS);
        if (__syncthreads_or(!ok)) {
            // a copy did not complete in time: record it, let the copies
            // already issued finish (bounded), and stop
            if (tid == 0) {
                atomicOr(status, STATUS_TIMEOUT);
                mbar_wait_bounded(bar + (st ^ 1), (unsigned)((k + 1) >> 1) & 1u, MBAR_WAIT_NS);
            }
            return;
        }
        const unsigned char *base = smem + st * L.stage_bytes;
        const int *sc = reinterpret_cast<const int *>(base + L.cols_off);
        const V *sv = reinterpret_cast<const V *>(base + L.vals_off);
        const int *srp = reinterpret_cast<const int *>(base + L.rows_off);
        const int *hdr = reinterpret_cast<const int *>(base + L.hdr_off);
        const int rb = hdr[0], re = hdr[1], wbase = hdr[2];
        const bool staged = hdr[3] != 0;
        auto rp = [&](int r) -> int { return staged ? srp[r - wbase] : __ldg(rowptr + r); };
        const int64_t E0 = t * tile, E1 = E0 + tile < nnz ? E0 + tile : nnz;
        for (int r = rb + g; r <= re; r += G) {
            const int rs = rp(r), rend = rp(r + 1);
            if (rs == rend) {  // empty row: written by the one tile whose range ends at or after it
                if (sub == 0 && ((rs > E0 && rs <= E1) || (rs == 0 && t == 0))) ep.store(y, r, T(0));
                continue;
            }
            const int s = rs > E0 ? rs : (int)E0, e = rend < E1 ? rend : (int)E1;
            if (s >= e) continue;
            if (e - s > 8 * TPR * UNROLL && TPR < 32) {  // left to a whole warp, or the whole block
                if (sub == 0) {
                    int i = e - s > long_len ? TILE_MED : atomicAdd(nmed, 1);
                    if (i < TILE_MED) med[i] = make_int4(r, s, e, 0);
                    else if ((i = atomicAdd(nlist, 1)) < long_max) list[i] = make_int4(r, s, e, 0);
                }
                continue;
            }
            T acc = T(0);
            for (int q = s + sub; q < e; q += TPR * UNROLL) {
                int c[UNROLL];
                T v[UNROLL], xv[UNROLL];
#pragma unroll
                for (int u = 0; u < UNROLL; ++u) {
                    const int qq = q + u * TPR;
                    c[u] = qq < e ? sc[qq - E0] : -1;
                    v[u] = qq < e ? (T)sv[qq - E0] : T(0);
                }
#pragma unroll
                for (int u = 0; u < UNROLL; ++u) xv[u] = c[u] >= 0 ? ld_x(x, c[u]) : T(0);
#pragma unroll
                for (int u = 0; u < UNROLL; ++u)
                    if (c[u] >= 0) acc = fma(v[u], xv[u], acc);
            }
#pragma unroll
            for (int off = TPR / 2; off > 0; off >>= 1) acc += __shfl_down_sync(gmask, acc, off, TPR);
            if (sub == 0) {
                T total = acc;
                if (rs >= E0 && rend <= E1) ep.store(y, r, total);
                else if (join_partial<T>(t, rs / tile, (rend - 1) / tile, 0, acc, P, &total)) ep.store(y, r, total);
            }
        }
        __syncthreads();
        // medium segments: one warp each, lanes striding, a shuffle sum
        const int nm = *nmed < TILE_MED ? *nmed : TILE_MED;
        for (int i = tid >> 5; i < nm; i += (int)(blockDim.x >> 5)) {
            const int4 d = med[i];
            T acc = T(0);
            for (int q = d.y + lane; q < d.z; q += 32 * UNROLL) {
                int c[UNROLL];
                T v[UNROLL], xv[UNROLL];
#pragma unroll
                for (int u = 0; u < UNROLL; ++u) {
                    const int qq = q + 32 * u;
                    c[u] = qq < d.z ? sc[qq - E0] : -1;
                    v[u] = qq < d.z ? (T)sv[qq - E0] : T(0);
                }
#pragma unroll
                for (int u = 0; u < UNROLL; ++u) xv[u] = c[u] >= 0 ? ld_x(x, c[u]) : T(0);
#pragma unroll
                for (int u = 0; u < UNROLL; ++u)
                    if (c[u] >= 0) acc = fma(v[u], xv[u], acc);
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
            if (lane == 0) {
                const int rs = rp(d.x), rend = rp(d.x + 1);
                T total = acc;
                if (rs >= E0 && rend <= E1) ep.store(y, d.x, total);
                else if (join_partial<T>(t, rs / tile, (rend - 1) / tile, 0, acc, P, &total))
                    ep.store(y, d.x, total);
            }
        }
        __syncthreads();  // every warp is done with the medium list before its reset and the stage refill
        const int nl = *nlist < long_max ? *nlist : long_max;
        for (int i = 0; i < nl; ++i) {  // long row segments: every thread strides, then a block sum
            const int4 d = list[i];
            T acc = T(0);
            for (int q = d.y + tid; q < d.z; q += blockDim.x) acc = fma((T)sv[q - E0], ld_x(x, sc[q - E0]), acc);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
            if (lane == 0) red[tid >> 5] = acc;
            __syncthreads();
            if (tid == 0) {
                T sum = T(0);
                for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += red[w];
                const int rs = rp(d.x), rend = rp(d.x + 1);
                T total = sum;
                if (rs >= E0 && rend <= E1) ep.store(y, d.x, total);
                else if (join_partial<T>(t, rs / tile, (rend - 1) / tile, 0, sum, P, &total))
                    ep.store(y, d.x, total);
            }
            __syncthreads();
        }
        // stage st is free: the block's tile after next goes into it
        if (tid == 0) {
            *nlist = 0;
            *nmed = 0;
            if (tn < ntiles) {
                fence_proxy_async_smem();
                issue(tn, st, nrb, nre);
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Split CSR by warp chunks: the nonzeros cut into chunks of C = 32 ITEMS
// entries, one warp per chunk, ITEMS consecutive entries per lane loaded as
// COO loads them but without a row index per entry -- the warp recovers the
// rows by merging the row pointers with the chunk's positions.
//
// meta[c] = first row r with rowptr[r] >= c C (meta[nchunks] = m), so the
// rows [meta[c], meta[c+1]) start inside chunk c (the last chunk also holds
// the empty rows at the end), and row meta[c] - 1 may continue into it from
// before.  A rows pass reads those row pointers 32 rows at a time (coalesced
// loads), writes the empty rows among them, and lists the rows that have
// entries in the chunk, in order: list index k -> row id in `lr`, and the
// position inside the chunk where row k starts sets a bit of `bits`.  A lane
// finds the list index of its first entry's row by counting the set bits up
// to its first position, and walks its entries, moving to the next list row
// at each set bit -- one integer test per entry, no search.  Runs that cross
// lanes are joined by the same segmented scan as COO (keyed by list index),
// and a row crossing chunks by the same fixed-order partials.
// ---------------------------------------------------------------------------
template <int ITEMS>
struct MergeSmem {
    int lr[32 * ITEMS];     // row id of each list index
    unsigned bits[ITEMS];   // bit p: a listed row starts at chunk position p
};

template <typename V, typename T, int ITEMS>
__device__ __forceinline__ void csr_merge_chunk(int64_t c, int64_t nnz, int64_t m, const int *__restrict__ rowptr,
                                                const int *__restrict__ cols, const V *__restrict__ vals,
                                                const T *__restrict__ x, T *__restrict__ y, const Epi<T> &ep,
                                                int m0, int m1, const PartialsT<T> &P,
                                                MergeSmem<ITEMS> &W) {
    static_assert(32 % ITEMS == 0, "a lane's positions must sit in one word of the bitmap");
    constexpr int C = 32 * ITEMS;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    // offsets and rows fit in 32 bits: a handle holds fewer than 2^31 nonzeros
    const int E0 = (int)(c * C), E1 = (int)((c * C + C < nnz) ? c * C + C : nnz);
    const int n = E1 - E0;
    const int pos = lane * ITEMS;
    const int cnt = n - pos <= 0 ? 0 : (n - pos >= ITEMS ? ITEMS : n - pos);
    const int last_lane = (n - 1) / ITEMS;
    // rows [rb, m1) are read 32 at a time (rb < m1: row m1 - 1 holds or
    // follows entry E1 - 1); the first 32 row pointers are loaded before the
    // entries so that both latencies overlap
    const int rb = m0 > 0 ? m0 - 1 : 0;
    const bool v1 = rb + lane < m1;
    const int s1 = v1 ? __ldg(rowptr + rb + lane) : 0;
    const int e1 = v1 ? __ldg(rowptr + rb + lane + 1) : 0;
    int r_unused[ITEMS];
    T v[ITEMS], xv[ITEMS];
    seg_load<V, T, ITEMS, false, true>(n == C, (int64_t)E0 + pos, cnt, nullptr, cols, vals, x, r_unused, v, xv);

    // rows pass
    __syncwarp();  // the previous chunk's reads of W are done
    if (lane < ITEMS) W.bits[lane] = 0u;
    __syncwarp();
    int K = 0;
    int hs = 0, he = 0, te = 0;  // head row's start and end, tail row's end (whole rows)
    auto round = [&](int r0, int s, int e) {
        const int r = r0 + lane;
        const bool valid = r < m1;
        if (valid && s == e && r >= m0) ep.store(y, (int64_t)r, T(0));
        const int cs = s > E0 ? s : E0, ce = e < E1 ? e : E1;
        const bool in = valid && cs < ce;
        const unsigned bal = __ballot_sync(FULL, in);
        if (bal) {  // warp-uniform
            if (in) {
                const int k = K + __popc(bal & ((1u << lane) - 1u));
                W.lr[k] = r;
                const int p = cs - E0;
                atomicOr(&W.bits[p >> 5], 1u << (p & 31));
            }
            const int f = __ffs(bal) - 1, l = 31 - __clz(bal);
            if (K == 0) {
                hs = __shfl_sync(FULL, s, f);
                he = __shfl_sync(FULL, e, f);
            }
            te = __shfl_sync(FULL, e, l);
            K += __popc(bal);
        }
    };
    round(rb, s1, e1);
    // chunks of short rows span many rows: the row pointers of up to four
    // rounds are loaded together
    constexpr int RB = 4;
    for (int r0 = rb + 32; r0 < m1; r0 += 32 * RB) {
        int sv[RB], ev[RB];
#pragma unroll
        for (int q = 0; q < RB; ++q) {
            const int r = r0 + 32 * q + lane;
            sv[q] = r < m1 ? __ldg(rowptr + r) : 0;
            ev[q] = r < m1 ? __ldg(rowptr + r + 1) : 0;
        }
#pragma unroll
        for (int q = 0; q < RB; ++q)
            if (r0 + 32 * q < m1) round(r0 + 32 * q, sv[q], ev[q]);
    }
    __syncwarp();

    // list index of the row holding this lane's first entry: set bits in
    // positions [0, pos], minus one (position 0 always starts list row 0)
    const int w = pos >> 5, b = pos & 31;
    const int pc = lane < ITEMS ? __popc(W.bits[lane]) : 0;
    int incl = pc;
#pragma unroll
    for (int d = 1; d < ITEMS; d <<= 1) {
        const int t = __shfl_up_sync(FULL, incl, d);
        if (lane >= d) incl += t;
    }
    const int before = __shfl_sync(FULL, incl - pc, w);  // set bits in words before w
    const unsigned word = W.bits[w];
    const int k0 = before + __popc(word & ((2u << b) - 1u)) - 1;
    const unsigned mb = ITEMS == 32 ? (word >> b) : ((word >> b) & ((1u << ITEMS) - 1u));

    int cur = k0;
    const int fr = k0;
    T fs = T(0), acc = T(0);
    bool fflush = false;
    if (cnt > 0) {
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            if (j < cnt) {
                if (j > 0 && ((mb >> j) & 1u)) {  // entry pos + j starts the next list row
                    if (!fflush) { fs = acc; fflush = true; }
                    else seg_write<T, false>(y, W.lr[cur], acc, ep);
                    ++cur;
                    acc = T(0);
                }
                acc = fma(v[j], xv[j], acc);
            }
        }
    }
    // list row after this lane's range: the next lane's first row; after
    // the chunk's last entry, the tail row again if it continues past E1,
    // else K (no row)
    const int k0n = __shfl_down_sync(FULL, k0, 1);
    const bool t_fwd = te > E1;
    const int nr = lane == last_lane ? (t_fwd ? K - 1 : K) : k0n;
    if (cnt > 0 && nr != cur) {  // the lane's last row ends exactly at its end
        if (!fflush) { fs = acc; fflush = true; }
        else seg_write<T, false>(y, W.lr[cur], acc, ep);
        cur = nr;
        acc = T(0);
    }
    const int key = cnt > 0 ? cur : -1;
    const T sc = seg_scan<T>(key, cnt > 0 ? acc : T(0));
    const int pkey = __shfl_up_sync(FULL, key, 1);
    const T pval = __shfl_up_sync(FULL, sc, 1);
    const bool h_back = hs < E0;  // list row 0 started in an earlier chunk
    const T total = seg_carry<T>(cnt > 0 && fflush && lane > 0 && pkey == fr, fs, pval);
    if (cnt > 0 && fflush) {
        if (fr == 0 && h_back)
            seg_arrive<T, false>(W.lr[0], c, hs / C, (he - 1) / C, total, P, y, ep);
        else
            seg_write<T, false>(y, W.lr[fr], total, ep);
    }
    if (lane == last_lane && t_fwd) {  // the tail row continues into the next chunk
        const int64_t c0 = (cur == 0 && h_back) ? hs / C : c;
        seg_arrive<T, false>(W.lr[cur], c, c0, (te - 1) / C, sc, P, y, ep);
    }
}

// one MergeSmem per warp in dynamic shared memory; 16 items per lane need
// more than 64 registers, so those variants take at most 512 threads per
// block
template <typename V, typename T, int ITEMS>
__global__ void __launch_bounds__(ITEMS >= 16 ? 512 : 1024) __maxnreg__(ITEMS >= 16 ? 128 : 64)
k_csr_merge(int64_t nnz, int64_t m, const int *__restrict__ rowptr, const int *__restrict__ cols,
            const V *__restrict__ vals, const T *__restrict__ x, T *__restrict__ y, T alpha, T beta,
            const int *__restrict__ meta, const PartialsT<T> P) {
    extern __shared__ __align__(16) unsigned char merge_smem[];
    MergeSmem<ITEMS> &W = reinterpret_cast<MergeSmem<ITEMS> *>(merge_smem)[threadIdx.x >> 5];
    const Epi<T> ep(alpha, beta);
    constexpr int C = 32 * ITEMS;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nchunks = (nnz + C - 1) / C;
    // each chunk's row range is loaded one chunk ahead
    int m0 = 0, m1 = 0;
    if (warp < nchunks) {
        m0 = __ldg(meta + warp);
        m1 = __ldg(meta + warp + 1);
    }
    for (int64_t c = warp; c < nchunks; c += nwarps) {
        const int64_t cn = c + nwarps;
        const int n0 = cn < nchunks ? __ldg(meta + cn) : 0, n1 = cn < nchunks ? __ldg(meta + cn + 1) : 0;
        csr_merge_chunk<V, T, ITEMS>(c, nnz, m, rowptr, cols, vals, x, y, ep, m0, m1, P, W);
        m0 = n0;
        m1 = n1;
    }
}

}  // namespace spmv

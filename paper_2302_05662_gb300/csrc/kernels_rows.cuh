// Row-parallel SpMV kernels: CSR vector (threads-per-row lanes per row),
// column-major ELL (thread per row) and BSR (lanes per block row).
//
// Each computes y = alpha * A x + beta * y (Section 2.2) for the storage
// layouts of Section 2.3.  Kernel parameters are template arguments, so the
// paper's compile-time knobs (Section 4: register cap, block size) and the
// threads-per-row / unroll knobs become pre-built variants selected at run
// time instead of recompilation.
#pragma once

#include "combine.cuh"

namespace spmv {

constexpr unsigned FULLMASK = 0xffffffffu;

// ---------------------------------------------------------------------------
// CSR: TPR lanes share a row (Section 2.3: warp lanes coordinate to add the
// per-thread partial sums).  A warp takes 32 consecutive rows, reads their
// bounds with one coalesced load, then works through them RPW = 32/TPR rows
// at a time, each lane keeping UNROLL loads in flight.  Rows longer than
// long_threshold are left to k_csr_long.  All loops are warp-uniform, so the
// shuffle reduction always has every lane.
// ---------------------------------------------------------------------------
// 4 stored values starting at a multiple of 4 entries, L1-allocating (a
// lane walks its own row: the group after this one sits in the same sector)
__device__ __forceinline__ void ld_vals4_c(const double *p, double (&o)[4]) {
    const double2 a = __ldg(reinterpret_cast<const double2 *>(p));
    const double2 b = __ldg(reinterpret_cast<const double2 *>(p) + 1);
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}
__device__ __forceinline__ void ld_vals4_c(const float *p, float (&o)[4]) {
    const float4 a = __ldg(reinterpret_cast<const float4 *>(p));
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
}
__device__ __forceinline__ void ld_vals4_c(const __nv_bfloat16 *p, float (&o)[4]) {
    const uint2 w = __ldg(reinterpret_cast<const uint2 *>(p));
    o[0] = bf16lo(w.x); o[1] = bf16hi(w.x); o[2] = bf16lo(w.y); o[3] = bf16hi(w.y);
}

// 8 stored entries starting at a multiple of 8: 32-byte loads (the 256-bit
// global loads of sm_100 and later), L1-allocating as above
__device__ __forceinline__ void ld_idx8_c(const int *p, int (&o)[8]) {
    asm("ld.global.nc.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=r"(o[0]), "=r"(o[1]), "=r"(o[2]), "=r"(o[3]), "=r"(o[4]), "=r"(o[5]), "=r"(o[6]), "=r"(o[7])
        : "l"(p));
}
__device__ __forceinline__ void ld_vals8_c(const double *p, double (&o)[8]) {
    asm("ld.global.nc.v4.f64 {%0, %1, %2, %3}, [%4];" : "=d"(o[0]), "=d"(o[1]), "=d"(o[2]), "=d"(o[3]) : "l"(p));
    asm("ld.global.nc.v4.f64 {%0, %1, %2, %3}, [%4];" : "=d"(o[4]), "=d"(o[5]), "=d"(o[6]), "=d"(o[7]) : "l"(p + 4));
}
__device__ __forceinline__ void ld_vals8_c(const float *p, float (&o)[8]) {
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(o[0]), "=f"(o[1]), "=f"(o[2]), "=f"(o[3]), "=f"(o[4]), "=f"(o[5]), "=f"(o[6]), "=f"(o[7])
        : "l"(p));
}
__device__ __forceinline__ void ld_vals8_c(const __nv_bfloat16 *p, float (&o)[8]) {
    const uint4 w = __ldg(reinterpret_cast<const uint4 *>(p));
    o[0] = bf16lo(w.x); o[1] = bf16hi(w.x); o[2] = bf16lo(w.y); o[3] = bf16hi(w.y);
    o[4] = bf16lo(w.z); o[5] = bf16hi(w.z); o[6] = bf16lo(w.w); o[7] = bf16hi(w.w);
}

// one aligned group of GW entries: columns and values
template <int GW, typename V, typename T>
__device__ __forceinline__ void ld_group_c(const int *cp, const V *vp, int (&c)[GW], T (&v)[GW]) {
    if constexpr (GW == 8) {
        ld_idx8_c(cp, c);
        ld_vals8_c(vp, v);
    } else {
        const int4 w = __ldg(reinterpret_cast<const int4 *>(cp));
        c[0] = w.x; c[1] = w.y; c[2] = w.z; c[3] = w.w;
        ld_vals4_c(vp, v);
    }
}

// Entries [a, b) of one row summed by one lane with wide loads: the lane
// walks the aligned groups of GW entries (4: 16-byte loads; 8: 32-byte
// loads) covering its range, the first and last group masked, G groups in
// flight.  The column and value arrays are padded to a multiple of 8
// entries past nnz, so the last group's load stays inside them.
template <typename V, typename T, int G, int GW>
__device__ __forceinline__ T csr_lane_range(int a, int b, const int *__restrict__ colidx, const V *__restrict__ vals,
                                            const T *__restrict__ x) {
    T acc = T(0);
    for (int q = a & ~(GW - 1); q < b; q += GW * G) {
        int c[G][GW];
        T v[G][GW], xv[G][GW];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int gq = q + GW * g;
            if (gq < b) ld_group_c<GW>(colidx + gq, vals + gq, c[g], v[g]);
#pragma unroll
            for (int t = 0; t < GW; ++t)
                if (gq >= b || gq + t < a || gq + t >= b) c[g][t] = -1;
        }
#pragma unroll
        for (int g = 0; g < G; ++g)
#pragma unroll
            for (int t = 0; t < GW; ++t) xv[g][t] = c[g][t] >= 0 ? ld_x(x, c[g][t]) : T(0);
#pragma unroll
        for (int g = 0; g < G; ++g)
#pragma unroll
            for (int t = 0; t < GW; ++t)
                if (c[g][t] >= 0) acc = fma(v[g][t], xv[g][t], acc);
    }
    return acc;
}

// Rows [base, base + 32) with TPR lanes per row; the whole warp calls it.
// With one or two lanes per row each lane sums a contiguous part of its row
// with 16- or 32-byte loads (csr_lane_range); with more lanes, the lanes of a row
// take interleaved entries, so a warp's loads of a row are contiguous.
template <typename V, typename T, int TPR, int UNROLL, int GW = 4>
__device__ __forceinline__ void csr_vector_rows(int64_t base, int64_t m, const int *__restrict__ rowptr,
                                                const int *__restrict__ colidx, const V *__restrict__ vals,
                                                const T *__restrict__ x, T *__restrict__ y, const Epi<T> &ep,
                                                int long_threshold) {
    constexpr int RPW = 32 / TPR;  // rows per warp per step
    const int lane = threadIdx.x & 31;
    const int sub = lane % TPR, grp = lane / TPR;
    const int64_t rr = base + lane;
    const int my_s = rr < m ? __ldg(rowptr + rr) : 0;
    const int my_e = rr < m ? __ldg(rowptr + rr + 1) : 0;
#pragma unroll 1
    for (int g = 0; g < TPR; ++g) {
        const int src = g * RPW + grp;
        const int s = __shfl_sync(FULLMASK, my_s, src);
        const int e = __shfl_sync(FULLMASK, my_e, src);
        const int64_t row = base + src;
        const bool skip = row >= m || e - s > long_threshold;
        T acc = T(0);
        if constexpr (TPR <= 2) {
            if (!skip) {
                // lane sub takes [s, mid) or [mid, e), mid on a group boundary
                int mid = TPR == 1 ? e : ((s + (e - s) / 2 + GW - 1) & ~(GW - 1));
                mid = mid < s ? s : (mid > e ? e : mid);
                const int a = sub == 0 ? s : mid, b = sub == 0 ? mid : e;
                acc = csr_lane_range<V, T, (UNROLL >= 4 ? 2 : 1), GW>(a, b, colidx, vals, x);
            }
        } else if (!skip) {
            for (int k = s + sub; k < e; k += TPR * UNROLL) {
                int c[UNROLL];
                T v[UNROLL];
#pragma unroll
                for (int u = 0; u < UNROLL; ++u) {
                    const int kk = k + u * TPR;
                    c[u] = kk < e ? ld_s(colidx + kk) : -1;
                    v[u] = kk < e ? ld_val(vals + kk) : T(0);
                }
#pragma unroll
                for (int u = 0; u < UNROLL; ++u)
                    if (c[u] >= 0) acc += v[u] * ld_x(x, c[u]);
            }
        }
#pragma unroll
        for (int off = TPR / 2; off > 0; off >>= 1) acc += __shfl_down_sync(FULLMASK, acc, off, TPR);
        if (sub == 0 && !skip) ep.store(y, row, acc);
    }
}

// GW: entries per lane load with one or two lanes per row (4: 16-byte
// loads, 8: 32-byte loads; wider groups read fewer load instructions per
// entry but mask more slots at a lane's first and last group)
template <typename V, typename T, int TPR, int UNROLL, int REGCAP, int GW>
__global__ void __launch_bounds__(1024) __maxnreg__(REGCAP)
k_csr_vector(int64_t m, const int *__restrict__ rowptr, const int *__restrict__ colidx,
             const V *__restrict__ vals, const T *__restrict__ x, T *__restrict__ y, T alpha, T beta,
             int long_threshold) {
    const Epi<T> ep(alpha, beta);
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = warp * 32; base < m; base += nwarps * 32)
        csr_vector_rows<V, T, TPR, UNROLL, GW>(base, m, rowptr, colidx, vals, x, y, ep, long_threshold);
}

// Long CSR rows: one thread block per segment of a long row; segments of one
// row are joined through the partials (fixed order).
template <typename V, typename T>
__global__ void __launch_bounds__(256)
k_csr_long(int64_t nseg, const int *__restrict__ seg_row, const int *__restrict__ seg_begin,
           const int *__restrict__ seg_end, const int *__restrict__ seg_c0, const int *__restrict__ seg_c1,
           const int *__restrict__ colidx, const V *__restrict__ vals, const T *__restrict__ x, T *__restrict__ y,
           T alpha, T beta, const PartialsT<T> P) {
    const Epi<T> ep(alpha, beta);
    __shared__ T red[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t k = blockIdx.x; k < nseg; k += gridDim.x) {
        const int b = __ldg(seg_begin + k), e = __ldg(seg_end + k);
        T acc = T(0);
        for (int i = b + threadIdx.x; i < e; i += 256 * 4) {
            int c[4];
            T v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int ii = i + u * 256;
                c[u] = ii < e ? ld_s(colidx + ii) : -1;
                v[u] = ii < e ? ld_val(vals + ii) : T(0);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (c[u] >= 0) acc += v[u] * ld_x(x, c[u]);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(FULLMASK, acc, off);
        if (lane == 0) red[warp] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            T t = T(0);
#pragma unroll
            for (int w = 0; w < 8; ++w) t += red[w];
            const int row = __ldg(seg_row + k);
            const int64_t c0 = __ldg(seg_c0 + k), c1 = __ldg(seg_c1 + k);
            T total = t;
            if (c0 == c1 || join_partial<T>(k, c0, c1, 0, t, P, &total)) ep.store(y, row, total);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// ELL, column-major [width][pitch] (Section 2.3: m x max_nnz Data and Column
// Index matrices).  Padding has column -1 and rows are left-packed, so a
// thread stops at its first padding slot and reads no padding values.
// ---------------------------------------------------------------------------
// a stored ELL column: int32 (padding -1) or a 16-bit offset from the row
// (padding INT16_MIN)
__device__ __forceinline__ int ell_col_at(const int *p, int64_t r) { return ld_s(p); }
__device__ __forceinline__ int ell_col_at(const int16_t *p, int64_t r) {
    const int d = (int16_t)ld_s(reinterpret_cast<const unsigned short *>(p));
    return d == INT16_MIN ? -1 : (int)r + d;
}

// One ELL row r (thread per row), shared by k_ell and the batched kernel.
template <typename V, typename T, int UNROLL, typename CI>
__device__ __forceinline__ void ell_row(int64_t r, int64_t width, int64_t pitch, const CI *__restrict__ col,
                                        const V *__restrict__ val, const T *__restrict__ x, T *__restrict__ y,
                                        const Epi<T> &ep) {
    T acc = T(0);
    int64_t k = 0;
    bool done = false;
    for (; !done && k + UNROLL <= width; k += UNROLL) {
        // all loads of the group go out together: padding slots hold a
        // zero value and column -1 (gathered at column 0, not added)
        int c[UNROLL];
        T v[UNROLL], xv[UNROLL];
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) c[u] = ell_col_at(col + (k + u) * pitch + r, r);
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
            v[u] = ld_val(val + (k + u) * pitch + r);
            xv[u] = ld_x(x, c[u] >= 0 ? c[u] : 0);
        }
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
            if (c[u] >= 0) acc = fma(v[u], xv[u], acc);
            else done = true;
        }
    }
    for (; !done && k < width; ++k) {
        const int c = ell_col_at(col + k * pitch + r, r);
        if (c < 0) break;
        acc += ld_val(val + k * pitch + r) * ld_x(x, c);
    }
    ep.store(y, r, acc);
}

template <typename V, typename T, int UNROLL, int REGCAP, typename CI>
__global__ void __launch_bounds__(1024) __maxnreg__(REGCAP)
k_ell(int64_t m, int64_t width, int64_t pitch, const CI *__restrict__ col, const V *__restrict__ val,
      const T *__restrict__ x, T *__restrict__ y, T alpha, T beta) {
    const Epi<T> ep(alpha, beta);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < m; r += stride)
        ell_row<V, T, UNROLL, CI>(r, width, pitch, col, val, x, y, ep);
}

// Two adjacent rows per thread (fp32/bf16 values): rows r, r + 1 sit side by
// side in every column-major slice, so each load fetches both rows' entries
// in one 8-byte (int32 columns, fp32 values) or 4-byte (16-bit offsets, bf16
// values) access and a warp request covers 64 rows instead of 32.
__device__ __forceinline__ void ell_cols2(const int *p, int64_t r, int &a, int &b) {
    const int2 w = ld_s(reinterpret_cast<const int2 *>(p));
    a = w.x;
    b = w.y;
}
__device__ __forceinline__ void ell_cols2(const int16_t *p, int64_t r, int &a, int &b) {
    const uint32_t w = (uint32_t)ld_s(reinterpret_cast<const int *>(p));
    const int d0 = (int16_t)(w & 0xffffu), d1 = (int16_t)(w >> 16);
    a = d0 == INT16_MIN ? -1 : (int)r + d0;
    b = d1 == INT16_MIN ? -1 : (int)r + 1 + d1;
}
__device__ __forceinline__ void ell_vals2(const float *p, float &a, float &b) {
    const float2 w = ld_s(reinterpret_cast<const float2 *>(p));
    a = w.x;
    b = w.y;
}
__device__ __forceinline__ void ell_vals2(const __nv_bfloat16 *p, float &a, float &b) {
    const uint32_t w = (uint32_t)ld_s(reinterpret_cast<const int *>(p));
    a = bf16lo(w);
    b = bf16hi(w);
}

template <typename V, typename T, int UNROLL, int REGCAP, typename CI>
__global__ void __launch_bounds__(1024) __maxnreg__(REGCAP)
k_ell2(int64_t m, int64_t width, int64_t pitch, const CI *__restrict__ col, const V *__restrict__ val,
       const T *__restrict__ x, T *__restrict__ y, T alpha, T beta) {
    const Epi<T> ep(alpha, beta);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // pairs of rows up to the pitch (a multiple of 32): padding rows past m
    // hold padding slots, so every pair load stays inside the arrays
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; 2 * q < m; q += stride) {
        const int64_t r = 2 * q;
        T acc0 = T(0), acc1 = T(0);
        bool done0 = false, done1 = false;
        int64_t k = 0;
        for (; !(done0 && done1) && k + UNROLL <= width; k += UNROLL) {
            int c0[UNROLL], c1[UNROLL];
            T v0[UNROLL], v1[UNROLL], x0[UNROLL], x1[UNROLL];
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) ell_cols2(col + (k + u) * pitch + r, r, c0[u], c1[u]);
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) {
                ell_vals2(val + (k + u) * pitch + r, v0[u], v1[u]);
                x0[u] = ld_x(x, c0[u] >= 0 ? c0[u] : 0);
                x1[u] = ld_x(x, c1[u] >= 0 ? c1[u] : 0);
            }
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) {
                if (c0[u] >= 0) acc0 = fma(v0[u], x0[u], acc0);
                else done0 = true;
                if (c1[u] >= 0) acc1 = fma(v1[u], x1[u], acc1);
                else done1 = true;
            }
        }
        for (; !(done0 && done1) && k < width; ++k) {
            int c0, c1;
            T v0, v1;
            ell_cols2(col + k * pitch + r, r, c0, c1);
            ell_vals2(val + k * pitch + r, v0, v1);
            if (c0 >= 0) acc0 = fma(v0, ld_x(x, c0), acc0);
            else done0 = true;
            if (c1 >= 0) acc1 = fma(v1, ld_x(x, c1), acc1);
            else done1 = true;
        }
        ep.store(y, r, acc0);
        if (r + 1 < m) ep.store(y, r + 1, acc1);
    }
}

// ---------------------------------------------------------------------------
// BSR with R x R row-major blocks (the blocked ELL of Section 2.3 stored by
// block rows).  A group of R*S lanes owns a block row: lane (s, i) takes
// row i of every S-th block, so a warp reads whole blocks contiguously.
// ---------------------------------------------------------------------------
template <int R, typename V, typename T> struct BlockRow;
template <> struct BlockRow<4, double, double> {
    static __device__ __forceinline__ void load(const double *p, double (&o)[4]) {
        double2 a = ld_s(reinterpret_cast<const double2 *>(p));
        double2 b = ld_s(reinterpret_cast<const double2 *>(p) + 1);
        o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
    }
};
template <> struct BlockRow<2, double, double> {
    static __device__ __forceinline__ void load(const double *p, double (&o)[2]) {
        double2 a = ld_s(reinterpret_cast<const double2 *>(p));
        o[0] = a.x; o[1] = a.y;
    }
};
template <> struct BlockRow<4, float, float> {
    static __device__ __forceinline__ void load(const float *p, float (&o)[4]) {
        float4 a = ld_s(reinterpret_cast<const float4 *>(p));
        o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
    }
};
template <> struct BlockRow<2, float, float> {
    static __device__ __forceinline__ void load(const float *p, float (&o)[2]) {
        float2 a = ld_s(reinterpret_cast<const float2 *>(p));
        o[0] = a.x; o[1] = a.y;
    }
};
template <> struct BlockRow<4, __nv_bfloat16, float> {
    static __device__ __forceinline__ void load(const __nv_bfloat16 *p, float (&o)[4]) {
        uint2 w = ld_s(reinterpret_cast<const uint2 *>(p));
        o[0] = bf16lo(w.x); o[1] = bf16hi(w.x); o[2] = bf16lo(w.y); o[3] = bf16hi(w.y);
    }
};
template <> struct BlockRow<2, __nv_bfloat16, float> {
    static __device__ __forceinline__ void load(const __nv_bfloat16 *p, float (&o)[2]) {
        uint32_t w = (uint32_t)ld_s(reinterpret_cast<const int *>(p));
        o[0] = bf16lo(w); o[1] = bf16hi(w);
    }
};

// Block rows [base, base + 32 / (R S)) of a BSR matrix, R S lanes per block
// row (S blocks at once, two steps in flight); block rows longer than
// long_threshold blocks are left to k_bsr_long.  The whole warp calls it.
template <typename V, typename T, int R, int S>
__device__ __forceinline__ void bsr_rows(int64_t base, int64_t mb, int64_t m, int64_t n,
                                         const int *__restrict__ browptr, const int *__restrict__ bcol,
                                         const V *__restrict__ bval, const T *__restrict__ x, T *__restrict__ y,
                                         const Epi<T> &ep, int long_threshold) {
    constexpr int G = R * S;  // lanes per block row
    const int lane = threadIdx.x & 31;
    const int sub = lane % G, sblk = sub / R, i = sub % R;
    const int64_t br = base + lane / G;
    T acc = T(0);
    bool skip = br >= mb;
    if (!skip) {
        const int bs = __ldg(browptr + br), be = __ldg(browptr + br + 1);
        skip = be - bs > long_threshold;
        // two blocks per step keep more loads in flight
        for (int b = bs + sblk; !skip && b < be; b += 2 * S) {
            const bool two = b + S < be;
            const int64_t c0 = (int64_t)ld_s(bcol + b) * R;
            const int64_t c1 = two ? (int64_t)ld_s(bcol + b + S) * R : c0;
            T v0[R], v1[R];
            BlockRow<R, V, T>::load(bval + (int64_t)b * R * R + i * R, v0);
            if (two) BlockRow<R, V, T>::load(bval + (int64_t)(b + S) * R * R + i * R, v1);
#pragma unroll
            for (int j = 0; j < R; ++j)
                if (c0 + j < n) acc += v0[j] * ld_x(x, (int)(c0 + j));
            if (two) {
#pragma unroll
                for (int j = 0; j < R; ++j)
                    if (c1 + j < n) acc += v1[j] * ld_x(x, (int)(c1 + j));
            }
        }
    }
#pragma unroll
    for (int off = G / 2; off >= R; off >>= 1) acc += __shfl_down_sync(FULLMASK, acc, off, G);
    if (sblk == 0 && !skip) {
        const int64_t row = br * R + i;
        if (row < m) ep.store(y, row, acc);
    }
}

template <typename V, typename T, int R, int S>
__global__ void __launch_bounds__(1024)
k_bsr(int64_t mb, int64_t m, int64_t n, const int *__restrict__ browptr, const int *__restrict__ bcol,
      const V *__restrict__ bval, const T *__restrict__ x, T *__restrict__ y, T alpha, T beta, int long_threshold) {
    const Epi<T> ep(alpha, beta);
    constexpr int GPW = 32 / (R * S);  // block rows per warp per step
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = warp * GPW; base < mb; base += nwarps * GPW)
        bsr_rows<V, T, R, S>(base, mb, m, n, browptr, bcol, bval, x, y, ep, long_threshold);
}

// Long BSR block rows: one thread block per segment of blocks; lane (g, i)
// takes row i of every (256/R)-th block; rows of a block row are joined
// across segments through the partials with stride R.
template <typename V, typename T, int R>
__global__ void __launch_bounds__(256)
k_bsr_long(int64_t nseg, const int *__restrict__ seg_row, const int *__restrict__ seg_begin,
           const int *__restrict__ seg_end, const int *__restrict__ seg_c0, const int *__restrict__ seg_c1,
           int64_t m, int64_t n, const int *__restrict__ bcol, const V *__restrict__ bval,
           const T *__restrict__ x, T *__restrict__ y, T alpha, T beta, const PartialsT<T> P) {
    const Epi<T> ep(alpha, beta);
    constexpr int G = 256 / R;
    __shared__ T red[256];
    const int i = threadIdx.x % R, g = threadIdx.x / R;
    for (int64_t k = blockIdx.x; k < nseg; k += gridDim.x) {
        const int b = __ldg(seg_begin + k), e = __ldg(seg_end + k);
        T acc = T(0);
        for (int j = b + g; j < e; j += G) {
            const int64_t c0 = (int64_t)ld_s(bcol + j) * R;
            T v[R];
            BlockRow<R, V, T>::load(bval + (int64_t)j * R * R + i * R, v);
#pragma unroll
            for (int q = 0; q < R; ++q)
                if (c0 + q < n) acc += v[q] * ld_x(x, (int)(c0 + q));
        }
        red[threadIdx.x] = acc;
        __syncthreads();
        for (int st = G / 2; st > 0; st >>= 1) {
            if (g < st) red[g * R + i] += red[(g + st) * R + i];
            __syncthreads();
        }
        if (threadIdx.x < R) {
            const int64_t row = (int64_t)__ldg(seg_row + k) * R + i;
            if (row < m) {
                const int64_t c0 = __ldg(seg_c0 + k), c1 = __ldg(seg_c1 + k);
                T total = red[i];
                if (c0 == c1 || join_partial<T>(k, c0, c1, i, red[i], P, &total))
                    ep.store(y, row, total);
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// SELL (Section 2.3: slices of rows stored as small ELL matrices with a slice
// pointer array).  Slices are 32 rows -- one warp, one lane per row -- of
// rows sorted by descending length, so a slice's rows have similar lengths
// and little padding.  Inside a slice the columns come in groups of four,
// each group with a lane's four entries side by side, so a lane loads four
// column indices with one 16-byte access and a warp's request is 512
// contiguous bytes; a slice's last (width mod 4) columns are stored
// column-major, so no slot of padding is added.  A work item covers at most the item width (128
// columns by default) of one slice: a wider slice becomes several items whose
// per-row partials are joined in item order, so a slice of power-law rows is
// not left to one warp.  Slices of empty rows get no work item.
// ---------------------------------------------------------------------------
// 4 stored values of one lane's group (16-byte aligned for fp32 columns;
// 32-byte for fp64, 8-byte for bf16), through the streaming path
__device__ __forceinline__ void ld_vals4_s(const double *p, double (&o)[4]) {
    const double2 a = ld_s(reinterpret_cast<const double2 *>(p));
    const double2 b = ld_s(reinterpret_cast<const double2 *>(p) + 1);
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}
__device__ __forceinline__ void ld_vals4_s(const float *p, float (&o)[4]) {
    const float4 a = ld_s(reinterpret_cast<const float4 *>(p));
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
}
__device__ __forceinline__ void ld_vals4_s(const __nv_bfloat16 *p, float (&o)[4]) {
    const uint2 w = ld_s(reinterpret_cast<const uint2 *>(p));
    o[0] = bf16lo(w.x); o[1] = bf16hi(w.x); o[2] = bf16lo(w.y); o[3] = bf16hi(w.y);
}

// Work item `it` of a SELL matrix (the whole warp), shared by k_sell and the
// batched kernel.  An item is `len` columns of one slice starting at slot
// `ib`: len >> 2 groups of four columns (lane l's four entries of a group
// contiguous at ib + 128 g + 4 l: one 16-byte column load per lane and
// group), then len & 3 column-major columns (the slice's last item only).
template <typename V, typename T, int UNROLL, bool GROUPED>
__device__ __forceinline__ void sell_item(int64_t it, int64_t m, const int *__restrict__ it_slice,
                                          const int *__restrict__ it_base, const int *__restrict__ it_len,
                                          const int *__restrict__ it_c0, const int *__restrict__ it_c1,
                                          const int *__restrict__ col, const V *__restrict__ val,
                                          const int *__restrict__ perm, const T *__restrict__ x, T *__restrict__ y,
                                          const Epi<T> &ep, const PartialsT<T> &P) {
    constexpr int UG = UNROLL >= 8 ? 2 : 1;  // groups of four in flight per lane
    const int lane = threadIdx.x & 31;
    // an item is three independent loads: slice, slot offset, columns (the
    // row and join range are read after the loop: requesting them up front
    // slowed the fp64 banded product by 4%)
    const int sl = __ldg(it_slice + it), ib = __ldg(it_base + it), len = __ldg(it_len + it);
    T acc = T(0);
    if constexpr (!GROUPED) {  // every column column-major: entry k at ib + 32 k + lane
        const int64_t base = (int64_t)ib + lane;
        int k = 0;
        for (; k + UNROLL <= len; k += UNROLL) {
            int c[UNROLL];
            T v[UNROLL], xv[UNROLL];
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) c[u] = ld_s(col + base + 32LL * (k + u));
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) {
                v[u] = ld_val(val + base + 32LL * (k + u));
                xv[u] = ld_x(x, c[u] >= 0 ? c[u] : 0);
            }
#pragma unroll
            for (int u = 0; u < UNROLL; ++u)
                if (c[u] >= 0) acc = fma(v[u], xv[u], acc);
        }
        for (; k < len; ++k) {
            const int c = ld_s(col + base + 32LL * k);
            if (c >= 0) acc = fma(ld_val(val + base + 32LL * k), ld_x(x, c), acc);
        }
    } else {
    const int ng = len >> 2;
    const int64_t gbase = (int64_t)ib + 4 * lane;
    int g = 0;
    for (; g + UG <= ng; g += UG) {
        int c[UG][4];
        T v[UG][4], xv[UG][4];
#pragma unroll
        for (int u = 0; u < UG; ++u) {
            const int4 w = ld_s(reinterpret_cast<const int4 *>(col + gbase + 128LL * (g + u)));
            c[u][0] = w.x; c[u][1] = w.y; c[u][2] = w.z; c[u][3] = w.w;
            ld_vals4_s(val + gbase + 128LL * (g + u), v[u]);
        }
#pragma unroll
        for (int u = 0; u < UG; ++u)
#pragma unroll
            for (int t = 0; t < 4; ++t) xv[u][t] = ld_x(x, c[u][t] >= 0 ? c[u][t] : 0);
#pragma unroll
        for (int u = 0; u < UG; ++u)
#pragma unroll
            for (int t = 0; t < 4; ++t)
                if (c[u][t] >= 0) acc = fma(v[u][t], xv[u][t], acc);
    }
    for (; g < ng; ++g) {
        const int4 w = ld_s(reinterpret_cast<const int4 *>(col + gbase + 128LL * g));
        T v[4];
        ld_vals4_s(val + gbase + 128LL * g, v);
        const int c[4] = {w.x, w.y, w.z, w.w};
        T xv[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) xv[t] = ld_x(x, c[t] >= 0 ? c[t] : 0);
#pragma unroll
        for (int t = 0; t < 4; ++t)
            if (c[t] >= 0) acc = fma(v[t], xv[t], acc);
    }
    const int tail = len & 3;
    if (tail) {  // the slice's last columns, column-major
        const int64_t tb = (int64_t)ib + 128LL * ng + lane;
        int c[3];
        T v[3];
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            c[t] = t < tail ? ld_s(col + tb + 32 * t) : -1;
            v[t] = t < tail ? ld_val(val + tb + 32 * t) : T(0);
        }
#pragma unroll
        for (int t = 0; t < 3; ++t)
            if (c[t] >= 0) acc = fma(v[t], ld_x(x, c[t]), acc);
    }
    }
    const int64_t p = (int64_t)sl * 32 + lane;
    if (p < m) {
        const int row = __ldg(perm + p);
        const int64_t c0 = __ldg(it_c0 + it), c1 = __ldg(it_c1 + it);
        T total = acc;
        if (c0 == c1 || join_partial<T>(it, c0, c1, lane, acc, P, &total)) ep.store(y, row, total);
    }
}

template <typename V, typename T, int UNROLL, int REGCAP, bool GROUPED>
__global__ void __launch_bounds__(1024) __maxnreg__(REGCAP)
k_sell(int64_t m, int64_t nitems, int64_t s_zero, const int *__restrict__ it_slice, const int *__restrict__ it_base,
       const int *__restrict__ it_len, const int *__restrict__ it_c0, const int *__restrict__ it_c1,
       const int *__restrict__ col, const V *__restrict__ val, const int *__restrict__ perm,
       const T *__restrict__ x, T *__restrict__ y, T alpha, T beta, const PartialsT<T> P) {
    const Epi<T> ep(alpha, beta);
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t warp = gtid >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    // empty rows (sorted last, in slices s_zero and after): no item, one
    // grid-stride pass; the stable sort keeps their order, so the writes
    // of consecutive threads go to increasing rows
    for (int64_t p = s_zero * 32 + gtid; p < m; p += nwarps * 32) ep.store(y, __ldg(perm + p), T(0));
    // items come widest slice first; passes over the warps alternate
    // direction (warp w takes item w of pass 0, item 2N-1-w of pass 1, ...),
    // so the warps that drew the widest items draw the narrowest next
    for (int64_t j = 0; j * nwarps < nitems; ++j) {
        const int64_t it = j * nwarps + ((j & 1) ? nwarps - 1 - warp : warp);
        if (it >= nitems) continue;
        sell_item<V, T, UNROLL, GROUPED>(it, m, it_slice, it_base, it_len, it_c0, it_c1, col, val, perm, x, y, ep,
                                         P);
    }
}

template <typename T>
__global__ void k_scale_y(int64_t m, T *y, T beta) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < m; r += stride)
        y[r] = beta == T(0) ? T(0) : beta * y[r];
}

}  // namespace spmv

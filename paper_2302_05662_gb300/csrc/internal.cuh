// Internal declarations shared by the CUDA translation units of the SpMV
// library.  Nothing here is part of the public C ABI (include/spmv.h).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>
#include <vector>

#include "spmv.h"

namespace spmv {

// ---------------------------------------------------------------------------
// error reporting
// ---------------------------------------------------------------------------
void set_error(const char *fmt, ...);
int cuda_status(cudaError_t e, const char *what);

// Every device allocation of the library goes through these two, so that
// the host-side fault injector can fail one of them: with the environment
// variable SPMV_FAULT_ALLOC=k, the k-th allocation of an entry-point call
// returns cudaErrorMemoryAllocation without allocating (the call must then
// return SPMV_ERR_OOM and release what it had allocated).  entry_reset(),
// called first by every entry point that allocates, clears the thread's
// error message and its allocation count.
cudaError_t dev_malloc(void **p, size_t bytes);
cudaError_t dev_malloc_async(void **p, size_t bytes, cudaStream_t s);
template <typename T>
inline cudaError_t dev_malloc(T **p, size_t bytes) {
    return dev_malloc(reinterpret_cast<void **>(p), bytes);
}
template <typename T>
inline cudaError_t dev_malloc_async(T **p, size_t bytes, cudaStream_t s) {
    return dev_malloc_async(reinterpret_cast<void **>(p), bytes, s);
}
void entry_reset();

#define SPMV_CUDA_TRY(expr)                                       \
    do {                                                          \
        cudaError_t _e = (expr);                                  \
        if (_e != cudaSuccess) return ::spmv::cuda_status(_e, #expr); \
    } while (0)

#define SPMV_TRY(expr)                 \
    do {                               \
        int _s = (expr);               \
        if (_s != SPMV_OK) return _s;  \
    } while (0)

// ---------------------------------------------------------------------------
// value-type traits: V = stored value, T = x/y/accumulator type
// ---------------------------------------------------------------------------
template <int VT> struct VT_;
template <> struct VT_<SPMV_F64> { using V = double; using T = double; };
template <> struct VT_<SPMV_F32> { using V = float; using T = float; };
template <> struct VT_<SPMV_BF16> { using V = __nv_bfloat16; using T = float; };

inline size_t value_size(int vt) { return vt == SPMV_F64 ? 8 : vt == SPMV_F32 ? 4 : 2; }
inline size_t vec_size(int vt) { return vt == SPMV_F64 ? 8 : 4; }

// ---------------------------------------------------------------------------
// device load helpers.  Matrix arrays are streamed once per product: they
// are read through the non-coherent path without L1 allocation so that L1
// keeps the gathered x entries.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int ld_s(const int *p) {
    int r;
    asm("ld.global.nc.L1::no_allocate.s32 %0, [%1];" : "=r"(r) : "l"(p));
    return r;
}
__device__ __forceinline__ int2 ld_s(const int2 *p) {
    int2 r;
    asm("ld.global.nc.L1::no_allocate.v2.s32 {%0,%1}, [%2];"
        : "=r"(r.x), "=r"(r.y) : "l"(p));
    return r;
}
__device__ __forceinline__ int4 ld_s(const int4 *p) {
    int4 r;
    asm("ld.global.nc.L1::no_allocate.v4.s32 {%0,%1,%2,%3}, [%4];"
        : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w) : "l"(p));
    return r;
}
__device__ __forceinline__ double ld_s(const double *p) {
    double r;
    asm("ld.global.nc.L1::no_allocate.f64 %0, [%1];" : "=d"(r) : "l"(p));
    return r;
}
__device__ __forceinline__ double2 ld_s(const double2 *p) {
    double2 r;
    asm("ld.global.nc.L1::no_allocate.v2.f64 {%0,%1}, [%2];"
        : "=d"(r.x), "=d"(r.y) : "l"(p));
    return r;
}
__device__ __forceinline__ float ld_s(const float *p) {
    float r;
    asm("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(r) : "l"(p));
    return r;
}
__device__ __forceinline__ float4 ld_s(const float4 *p) {
    float4 r;
    asm("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
        : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w) : "l"(p));
    return r;
}
__device__ __forceinline__ float2 ld_s(const float2 *p) {
    float2 r;
    asm("ld.global.nc.L1::no_allocate.v2.f32 {%0,%1}, [%2];"
        : "=f"(r.x), "=f"(r.y) : "l"(p));
    return r;
}
__device__ __forceinline__ unsigned short ld_s(const unsigned short *p) {
    unsigned short r;
    asm("ld.global.nc.L1::no_allocate.u16 %0, [%1];" : "=h"(r) : "l"(p));
    return r;
}
__device__ __forceinline__ uint2 ld_s(const uint2 *p) {
    uint2 r;
    asm("ld.global.nc.L1::no_allocate.v2.u32 {%0,%1}, [%2];"
        : "=r"(r.x), "=r"(r.y) : "l"(p));
    return r;
}
__device__ __forceinline__ uint4 ld_s(const uint4 *p) {
    uint4 r;
    asm("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
        : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w) : "l"(p));
    return r;
}

__device__ __forceinline__ float bf16lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }

// one stored value, converted to the accumulator type
__device__ __forceinline__ double ld_val(const double *p) { return ld_s(p); }
__device__ __forceinline__ float ld_val(const float *p) { return ld_s(p); }
__device__ __forceinline__ float ld_val(const __nv_bfloat16 *p) {
    return __uint_as_float((uint32_t)ld_s(reinterpret_cast<const unsigned short *>(p)) << 16);
}

// cached variants (L1-allocating), for access patterns where one lane reads
// consecutive entries across successive instructions
__device__ __forceinline__ double ld_val_c(const double *p) { return __ldg(p); }
__device__ __forceinline__ float ld_val_c(const float *p) { return __ldg(p); }
__device__ __forceinline__ float ld_val_c(const __nv_bfloat16 *p) {
    return __uint_as_float((uint32_t)__ldg(reinterpret_cast<const unsigned short *>(p)) << 16);
}

// N consecutive entries from a 16-byte aligned address with 16-byte loads,
// or, with WIDE, from a 32-byte aligned address with 32-byte loads (the
// 256-bit global loads of sm_100 and later: half the load instructions and
// L1 wavefronts for the same bytes).
__device__ __forceinline__ void ld_s8(const int *p, int *o) {
    asm("ld.global.nc.L1::no_allocate.v8.s32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=r"(o[0]), "=r"(o[1]), "=r"(o[2]), "=r"(o[3]), "=r"(o[4]), "=r"(o[5]), "=r"(o[6]), "=r"(o[7])
        : "l"(p));
}
__device__ __forceinline__ void ld_s4(const double *p, double *o) {
    asm("ld.global.nc.L1::no_allocate.v4.f64 {%0,%1,%2,%3}, [%4];"
        : "=d"(o[0]), "=d"(o[1]), "=d"(o[2]), "=d"(o[3]) : "l"(p));
}
__device__ __forceinline__ void ld_s8(const float *p, float *o) {
    asm("ld.global.nc.L1::no_allocate.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(o[0]), "=f"(o[1]), "=f"(o[2]), "=f"(o[3]), "=f"(o[4]), "=f"(o[5]), "=f"(o[6]), "=f"(o[7])
        : "l"(p));
}

template <int N, bool WIDE = false>
__device__ __forceinline__ void ld_vals_vec(const double *p, double (&o)[N]) {
    static_assert(N % 2 == 0, "");
    if constexpr (WIDE && N % 4 == 0) {
#pragma unroll
        for (int i = 0; i < N / 4; ++i) ld_s4(p + 4 * i, o + 4 * i);
    } else {
#pragma unroll
        for (int i = 0; i < N / 2; ++i) {
            double2 d = ld_s(reinterpret_cast<const double2 *>(p) + i);
            o[2 * i] = d.x;
            o[2 * i + 1] = d.y;
        }
    }
}
template <int N, bool WIDE = false>
__device__ __forceinline__ void ld_vals_vec(const float *p, float (&o)[N]) {
    static_assert(N % 4 == 0, "");
    if constexpr (WIDE && N % 8 == 0) {
#pragma unroll
        for (int i = 0; i < N / 8; ++i) ld_s8(p + 8 * i, o + 8 * i);
    } else {
#pragma unroll
        for (int i = 0; i < N / 4; ++i) {
            float4 d = ld_s(reinterpret_cast<const float4 *>(p) + i);
            o[4 * i] = d.x; o[4 * i + 1] = d.y; o[4 * i + 2] = d.z; o[4 * i + 3] = d.w;
        }
    }
}
template <int N, bool WIDE = false>
__device__ __forceinline__ void ld_vals_vec(const __nv_bfloat16 *p, float (&o)[N]) {
    static_assert(N % 4 == 0, "");
    if constexpr (N % 8 == 0) {  // 8 bf16 values are one 16-byte load
#pragma unroll
        for (int i = 0; i < N / 8; ++i) {
            uint4 w = ld_s(reinterpret_cast<const uint4 *>(p) + i);
            o[8 * i + 0] = bf16lo(w.x); o[8 * i + 1] = bf16hi(w.x);
            o[8 * i + 2] = bf16lo(w.y); o[8 * i + 3] = bf16hi(w.y);
            o[8 * i + 4] = bf16lo(w.z); o[8 * i + 5] = bf16hi(w.z);
            o[8 * i + 6] = bf16lo(w.w); o[8 * i + 7] = bf16hi(w.w);
        }
    } else {
#pragma unroll
        for (int i = 0; i < N / 4; ++i) {
            uint2 w = ld_s(reinterpret_cast<const uint2 *>(p) + i);
            o[4 * i + 0] = bf16lo(w.x); o[4 * i + 1] = bf16hi(w.x);
            o[4 * i + 2] = bf16lo(w.y); o[4 * i + 3] = bf16hi(w.y);
        }
    }
}
template <int N, bool WIDE = false>
__device__ __forceinline__ void ld_idx_vec(const int *p, int (&o)[N]) {
    static_assert(N % 4 == 0, "");
    if constexpr (WIDE && N % 8 == 0) {
#pragma unroll
        for (int i = 0; i < N / 8; ++i) ld_s8(p + 8 * i, o + 8 * i);
    } else {
#pragma unroll
        for (int i = 0; i < N / 4; ++i) {
            int4 d = ld_s(reinterpret_cast<const int4 *>(p) + i);
            o[4 * i] = d.x; o[4 * i + 1] = d.y; o[4 * i + 2] = d.z; o[4 * i + 3] = d.w;
        }
    }
}

// gathered x entry (read-only path, cached in L1)
template <typename T>
__device__ __forceinline__ T ld_x(const T *x, int col) { return __ldg(x + col); }

// y epilogue of Section 2.2 extended with BLAS scalars.  The tests on alpha
// and beta are made once per thread, so the common alpha = 1, beta = 0 case
// costs no floating-point instruction per row (fp64 issue slots are scarce
// on this GPU); beta == 0 never reads y.
template <typename T>
struct Epi {
    T alpha, beta;
    bool unit_alpha, zero_beta;
    __device__ __forceinline__ Epi(T a, T b) : alpha(a), beta(b), unit_alpha(a == T(1)), zero_beta(b == T(0)) {}
    __device__ __forceinline__ void store(T *y, int64_t row, T acc) const {
        if (unit_alpha && zero_beta) {
            y[row] = acc;
        } else {
            T r = unit_alpha ? acc : alpha * acc;
            if (!zero_beta) r += beta * y[row];
            y[row] = r;
        }
    }
    // y += alpha * acc (a second pass adding to rows a first pass wrote)
    __device__ __forceinline__ void add(T *y, int64_t row, T acc) const {
        y[row] += unit_alpha ? acc : alpha * acc;
    }
};

// ---------------------------------------------------------------------------
// handle
// ---------------------------------------------------------------------------
// Device scratch that joins partial sums of rows split across work units
// (chunks of the segmented kernels, segments of long rows).  A row spanning
// exactly two units meets in one 64-bit exchange slot; a longer row leaves
// its partials in head/tail and the last unit to arrive (counter) adds them
// in unit order.  Slots and counters are restored by whoever consumes them,
// so they start each product in their initial state.
struct Partials {
    void *head = nullptr;                 // T[units * stride]
    void *tail = nullptr;                 // T[units * stride]
    uint32_t *count = nullptr;            // [units * stride], initially 0
    unsigned long long *xslot = nullptr;  // [units * stride], initially empty
    int64_t units = 0;
    int stride = 1;
};

struct SegScratch {
    int items = 0;            // items per lane (chunk = 32 * items entries)
    int64_t nchunks = 0;
    int32_t *meta0 = nullptr; // COO: first chunk of the chunk's head row;
                              // staged tiles: row of the tile's first entry;
                              // warp chunks: first row starting at or after it
    int32_t *meta1 = nullptr; // COO: last chunk of the chunk's tail row
    Partials part;
};

// Rows (CSR) or block rows (BSR) too long for one lane group: cut into
// segments handled by whole thread blocks after the main kernel.
struct LongRows {
    int64_t threshold = 0;    // rows longer than this are deferred
    int64_t nrows = 0, nseg = 0;
    int32_t *seg_row = nullptr, *seg_begin = nullptr, *seg_end = nullptr;
    int32_t *seg_c0 = nullptr, *seg_c1 = nullptr;  // first / last segment of the row
    Partials part;
};

}  // namespace spmv

namespace spmv {
struct CgPlan;
}

struct spmv_matrix {
    int64_t m = 0, n = 0, nnz = 0, max_row = 0;
    double contig = 0.0;  // fraction of consecutive stored entries with consecutive columns
    int32_t vt = SPMV_F64;
    spmv_config cfg{};
    spmv_config packed_req{};  // configuration the current packs were built for
    bool packed = false;
    int sm_count = 0;
    // CSR (always present: the base every other format is packed from)
    int32_t *rowptr = nullptr;
    int32_t *colidx = nullptr;
    void *vals = nullptr;
    // COO row array (COO format; column and value arrays alias the CSR ones)
    int32_t *coo_rows = nullptr;
    // ELL (also the ELL part of HYB)
    int64_t ell_width = 0, ell_pitch = 0;
    int32_t *ell_col = nullptr;   // int32 columns, padding -1 ...
    int16_t *ell_d16 = nullptr;   // ... or 16-bit column - row, padding INT16_MIN
    void *ell_val = nullptr;
    // HYB COO part
    int64_t hyb_nnz = 0;
    int32_t *hyb_rows = nullptr, *hyb_cols = nullptr, *hyb_ptr = nullptr;
    void *hyb_vals = nullptr;
    // BSR
    int32_t bsr_r = 0;
    int64_t bsr_mb = 0, bsr_blocks = 0;
    int32_t *bsr_rowptr = nullptr, *bsr_col = nullptr;
    void *bsr_val = nullptr;
    // SELL: 32-row slices, column-major inside a slice, all rows stably
    // sorted by descending length; work items = (slice, first slot, columns)
    int64_t sell_nslices = 0, sell_slots = 0;
    bool sell_grouped = false;  // columns in groups of four (else column-major)
    int32_t *sell_ptr = nullptr, *sell_col = nullptr, *sell_perm = nullptr;
    void *sell_val = nullptr;
    // scratch of the segmented-reduction kernels (COO, HYB tail, split CSR)
    spmv::SegScratch seg;
    // deferred long rows of vector CSR and BSR
    spmv::LongRows lng;
    // conjugate-gradient plan (cg.cu): scratch vectors and the solve's graph
    spmv::CgPlan *cg = nullptr;
    // device status word: kernels that wait on a copy record a timeout here
    // (bits STATUS_TIMEOUT, STATUS_BOUNDS); spmv_check reads and clears it
    unsigned *d_status = nullptr;
    // row panels: a matrix with more triplets than one handle indexes with
    // int32 offsets is held as sub-handles over rows [panel_row0[p],
    // panel_row0[p+1]); the parent then holds no arrays of its own
    int32_t npanels = 0;
    spmv_matrix **panels = nullptr;
    int64_t *panel_row0 = nullptr;
};

namespace spmv {

// conversion (convert.cu)
int build_csr(spmv_matrix *h, const int32_t *d_rows, const int32_t *d_cols,
              const void *d_vals, cudaStream_t s);
int pack_format(spmv_matrix *h, const spmv_config &cfg, cudaStream_t s);
void free_packed(spmv_matrix *h);
int expand_rows(const int32_t *rowptr, int64_t m, int64_t nnz, int32_t *rows_out,
                cudaStream_t s);
int decode_ell_columns(const spmv_matrix *h, int32_t *d_out, cudaStream_t s);
// chunk metadata kinds: COO / HYB tail, staged CSR tiles, CSR warp chunks
enum { SEG_COO = 0, SEG_TILES = 1, SEG_MERGE = 2 };
int ensure_seg_scratch(spmv_matrix *h, int items, int kind, cudaStream_t s);
int build_coo_meta(const int32_t *rows, const int32_t *rowptr, int64_t nnz, int C, int32_t *meta0, int32_t *meta1,
                   cudaStream_t s);
int build_merge_meta(const int32_t *rowptr, int64_t m, int64_t nnz, int C, int32_t *meta, cudaStream_t s);
int alloc_partials(Partials *p, int64_t units, int stride, int vt, cudaStream_t s);
void free_partials(Partials *p);
int build_long_rows(spmv_matrix *h, const int32_t *rowptr, int64_t nrows, int64_t threshold, int64_t seg,
                    int stride, cudaStream_t s);

// row panels (convert.cu): bounds check of every triplet; panel row bounds
// (multiples of 4 rows, at most `limit` triplets each); stable copy of the
// triplets of rows [r0, r1) with rows shifted by -r0 (device buffers the
// caller frees with cudaFree)
int check_triplet_bounds(const int32_t *d_rows, const int32_t *d_cols, int64_t nnz, int64_t m, int64_t n,
                         cudaStream_t s);
int plan_panels(const int32_t *d_rows, int64_t nnz, int64_t m, int64_t limit, cudaStream_t s,
                std::vector<int64_t> *bounds);
int gather_panel(const int32_t *d_rows, const int32_t *d_cols, const void *d_vals, size_t vs, int64_t nnz,
                 int64_t r0, int64_t r1, int32_t **orow, int32_t **ocol, void **oval, int64_t *count,
                 cudaStream_t s);

// checked products (checked.cu): SPMV_CHECKED=1 in the environment, and
// the verification of the active format's indices before a product
bool checked_mode();
int check_indices(const spmv_matrix *h, cudaStream_t s);

// y = alpha A x + beta y in the handle's current format (api.cu)
int run_product(const spmv_matrix *h, double alpha, const void *x, double beta, void *y, cudaStream_t s);
// release the conjugate-gradient plan (cg.cu); packs it captured go stale on re-pack
void free_cg(spmv_matrix *h);

// kernel launchers: one runner per value type (kernels_<type>.cu)
enum RunKind { RUN_CSR_VECTOR, RUN_CSR_SPLIT, RUN_ELL, RUN_COO, RUN_HYB, RUN_BSR, RUN_SCALE, RUN_SELL };
int run_kernels_f64(int kind, const spmv_matrix *h, double alpha, const void *x, double beta, void *y,
                    cudaStream_t s);
int run_kernels_f32(int kind, const spmv_matrix *h, double alpha, const void *x, double beta, void *y,
                    cudaStream_t s);
int run_kernels_bf16(int kind, const spmv_matrix *h, double alpha, const void *x, double beta, void *y,
                     cudaStream_t s);

// default lanes per row of vector CSR for this matrix (api.cu)
int default_tpr(const spmv_matrix *h);

// launch helpers (api.cu)
int resident_blocks(const void *kernel, int threads);
int apply_carveout(const void *kernel, int carveout);

}  // namespace spmv

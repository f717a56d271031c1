// Measurement kernels (include/spmv_probe.h): the gather floor of a matrix
// and the fp64 fused-multiply-add ceiling of the device.  Neither forms a
// product; the benchmark times them beside the SpMV kernels to tell a kernel
// held by its x gathers or by the fp64 pipe from one that is simply slow.
#include "launch.cuh"
#include "spmv_probe.h"

namespace spmv {
namespace {

template <typename T> struct Bits;
template <> struct Bits<double> {
    using U = unsigned long long;
    static __device__ __forceinline__ U of(double v) { return (U)__double_as_longlong(v); }
    static __device__ __forceinline__ double to(U u) { return __longlong_as_double((long long)u); }
};
template <> struct Bits<float> {
    using U = unsigned;
    static __device__ __forceinline__ U of(float v) { return __float_as_uint(v); }
    static __device__ __forceinline__ float to(U u) { return __uint_as_float(u); }
};

// The product's bytes with ideal access and no floating-point instruction:
// each thread takes groups of 4 consecutive nonzeros (one 16-byte column
// load, 16 or 32 bytes of values; two groups in flight), gathers x at the 4
// columns, and folds the bits in with integer adds and xors; then the row
// pointers are streamed and y written, both grid-stride.
template <typename V, typename T>
__global__ void __launch_bounds__(256)
k_gather_floor(int64_t m, int64_t nnz, const int *__restrict__ rowptr, const int *__restrict__ col,
               const V *__restrict__ val, const T *__restrict__ x, T *__restrict__ y) {
    using U = typename Bits<T>::U;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t groups = nnz / 4;
    U acc = 0;
    for (int64_t g = tid; g < groups; g += 2 * stride) {
        const bool two = g + stride < groups;
        int c0[4], c1[4];
        T v0[4], v1[4], x0[4], x1[4];
        ld_idx_vec<4>(col + 4 * g, c0);
        ld_vals_vec<4>(val + 4 * g, v0);
        if (two) {
            ld_idx_vec<4>(col + 4 * (g + stride), c1);
            ld_vals_vec<4>(val + 4 * (g + stride), v1);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            x0[u] = ld_x(x, c0[u]);
            x1[u] = two ? ld_x(x, c1[u]) : T(0);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            acc ^= Bits<T>::of(v0[u]) + Bits<T>::of(x0[u]);
            acc ^= Bits<T>::of(v1[u]) + Bits<T>::of(x1[u]);
        }
    }
    for (int64_t i = 4 * groups + tid; i < nnz; i += stride)
        acc ^= Bits<T>::of(ld_val(val + i)) + Bits<T>::of(ld_x(x, ld_s(col + i)));
    for (int64_t r = tid; r <= m; r += stride) {
        acc += (U)(unsigned)ld_s(rowptr + r);
        if (r < m) y[r] = Bits<T>::to(acc);
    }
}

// Eight independent fp64 FMA chains per thread; b and c arrive as arguments
// so the chains cannot be folded at compile time.
__global__ void __launch_bounds__(256) k_fp64_fma(int64_t iters, double b, double c, double *sink) {
    double a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = (double)(threadIdx.x + 32 * k) * 1e-3;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = fma(a[k], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    if (s == -1.0e300) *sink = s;
}

template <int VT>
int gather_floor_vt(const spmv_matrix *h, const void *x, void *y, cudaStream_t s) {
    using V = typename VT_<VT>::V;
    using T = typename VT_<VT>::T;
    auto kern = k_gather_floor<V, T>;
    const int64_t work = (h->nnz / 4 > h->m + 1 ? h->nnz / 4 : h->m + 1);
    const int grid = wave_grid((const void *)kern, 256, (work + 255) / 256, h->sm_count);
    kern<<<grid, 256, 0, s>>>(h->m, h->nnz, h->rowptr, h->colidx, (const V *)h->vals, (const T *)x, (T *)y);
    SPMV_LAUNCH_CHECK();
    return SPMV_OK;
}

}  // namespace
}  // namespace spmv

using namespace spmv;

extern "C" {

int spmv_probe_gather_floor(spmv_handle h, const void *d_x, void *d_y, void *stream) {
    if (!h) {
        set_error("spmv_probe_gather_floor: NULL handle");
        return SPMV_ERR_INVALID;
    }
    if (h->npanels > 0) {
        set_error("spmv_probe_gather_floor: the matrix is held in row panels");
        return SPMV_ERR_UNSUPPORTED;
    }
    if ((h->n > 0 && !d_x) || (h->m > 0 && !d_y)) {
        set_error("spmv_probe_gather_floor: NULL vector");
        return SPMV_ERR_INVALID;
    }
    if (h->m == 0) return SPMV_OK;
    cudaStream_t s = (cudaStream_t)stream;
    switch (h->vt) {
    case SPMV_F64: return gather_floor_vt<SPMV_F64>(h, d_x, d_y, s);
    case SPMV_F32: return gather_floor_vt<SPMV_F32>(h, d_x, d_y, s);
    default: return gather_floor_vt<SPMV_BF16>(h, d_x, d_y, s);
    }
}

int spmv_probe_fp64_fma(int64_t iterations, double *d_sink, int64_t *h_fma_count, void *stream) {
    if (iterations < 1 || !d_sink || !h_fma_count) {
        set_error("spmv_probe_fp64_fma: iterations must be >= 1 and the pointers non-NULL");
        return SPMV_ERR_INVALID;
    }
    int dev = 0, sms = 0;
    SPMV_CUDA_TRY(cudaGetDevice(&dev));
    SPMV_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int grid = resident_blocks((const void *)k_fp64_fma, 256) * sms;
    k_fp64_fma<<<grid, 256, 0, (cudaStream_t)stream>>>(iterations, 1.0 - 1e-9, 1e-9, d_sink);
    SPMV_CUDA_TRY(cudaGetLastError());
    *h_fma_count = (int64_t)grid * 256 * 8 * iterations;
    return SPMV_OK;
}

}  // extern "C"

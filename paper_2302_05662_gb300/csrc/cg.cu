// Conjugate gradients on the device with the handle's SpMV (spmv_cg).
//
// Section 7.5 of the paper names preconditioned CG as the iterative setting
// in which one matrix is multiplied many times, so that feature extraction,
// selection and conversion are paid once.  The iteration is Hestenes and
// Stiefel's (1952):
//
//   r0 = b - A x0, p0 = r0, rho_k = r_k.r_k
//   while k < maxit and rho_k > tol^2 (b.b):
//     q = A p_k; alpha = rho_k / (p_k.q)          (stop on p_k.q <= 0)
//     x_{k+1} = x_k + alpha p_k; r_{k+1} = r_k - alpha q
//     beta = rho_{k+1} / rho_k; p_{k+1} = r_{k+1} + beta p_k
//
// GB300 layout of the loop: the whole solve is one CUDA graph.  A prologue
// forms r0, p0, rho_0 and b.b; a WHILE conditional node repeats the body
//   SpMV (the handle's format) -> p.q partials -> x, r update + r.r partials
//   -> state update (sets the loop condition) -> p update
// and the device alone decides when to stop, so no iteration waits for the
// host.  Every dot product is a fixed-shape reduction in fp64 (per-block
// partials, then every consumer sums the partials in the same order), so
// results are bit-reproducible and every block sees the same alpha and beta.
// Vector updates round the product and the sum separately (no FMA), the
// arithmetic the iteration above spells out.
//
// Termination does not depend on the reductions: the one-block state kernel
// increments the iteration counter on every pass and clears the condition
// once it reaches maxit.

#include <cmath>
#include <cstring>
#include <new>

#include "internal.cuh"

namespace spmv {

namespace {

constexpr int CG_THREADS = 256;

struct CgState {
    double rho, rho_prev, stop, bb;
    int32_t iter, maxit, converged, breakdown;
};

// fixed-order sum over the block (every block with the same inputs returns
// the same value); result valid in every thread
__device__ double block_sum(double v) {
    __shared__ double s_w[CG_THREADS / 32];
    __shared__ double s_total;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) s_w[w] = v;
    __syncthreads();
    if (w == 0) {
        double t = lane < CG_THREADS / 32 ? s_w[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (lane == 0) s_total = t;
    }
    __syncthreads();
    const double r = s_total;
    __syncthreads();
    return r;
}

// sum of part[0..n) in one fixed order, identical in every block
__device__ double sum_parts(const double *part, int n) {
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += CG_THREADS) v += part[i];
    return block_sum(v);
}

__device__ __forceinline__ double wide(double v) { return v; }
__device__ __forceinline__ double wide(float v) { return (double)v; }

// a + s*b with the product and the sum rounded separately
__device__ __forceinline__ double axpy1(double a, double s, double b) { return __dadd_rn(a, __dmul_rn(s, b)); }
__device__ __forceinline__ float axpy1(float a, float s, float b) { return __fadd_rn(a, __fmul_rn(s, b)); }

template <typename T>
__global__ void __launch_bounds__(CG_THREADS) k_cg_start(int64_t m, const T *__restrict__ r, const T *__restrict__ b,
                                                         T *__restrict__ p, double *part_rr, double *part_bb) {
    double rr = 0.0, bb = 0.0;
    const int64_t stride = (int64_t)gridDim.x * CG_THREADS;
    for (int64_t i = (int64_t)blockIdx.x * CG_THREADS + threadIdx.x; i < m; i += stride) {
        const T ri = r[i];
        const double rw = wide(ri), bw = wide(b[i]);
        p[i] = ri;
        rr = fma(rw, rw, rr);
        bb = fma(bw, bw, bb);
    }
    rr = block_sum(rr);
    bb = block_sum(bb);
    if (threadIdx.x == 0) {
        part_rr[blockIdx.x] = rr;
        part_bb[blockIdx.x] = bb;
    }
}

__global__ void __launch_bounds__(CG_THREADS) k_cg_init(const double *part_rr, const double *part_bb, int nparts,
                                                        CgState *st, double *hist, double tol2, int32_t maxit,
                                                        cudaGraphConditionalHandle cond) {
    const double rr = sum_parts(part_rr, nparts);
    const double bb = sum_parts(part_bb, nparts);
    if (threadIdx.x == 0) {
        const double stop = tol2 * bb;
        st->rho = rr;
        st->rho_prev = rr;
        st->stop = stop;
        st->bb = bb;
        st->iter = 0;
        st->maxit = maxit;
        st->converged = rr <= stop;
        st->breakdown = 0;
        hist[0] = rr;
        cudaGraphSetConditional(cond, (maxit > 0 && rr > stop) ? 1u : 0u);
    }
}

template <typename T>
__global__ void __launch_bounds__(CG_THREADS) k_cg_dot(int64_t m, const T *__restrict__ p, const T *__restrict__ q,
                                                       double *part_pq) {
    double pq = 0.0;
    const int64_t stride = (int64_t)gridDim.x * CG_THREADS;
    for (int64_t i = (int64_t)blockIdx.x * CG_THREADS + threadIdx.x; i < m; i += stride)
        pq = fma(wide(p[i]), wide(q[i]), pq);
    pq = block_sum(pq);
    if (threadIdx.x == 0) part_pq[blockIdx.x] = pq;
}

template <typename T>
__global__ void __launch_bounds__(CG_THREADS) k_cg_update(int64_t m, T *__restrict__ x, T *__restrict__ r,
                                                          const T *__restrict__ p, const T *__restrict__ q,
                                                          const double *part_pq, double *part_rr, int nparts,
                                                          const CgState *st) {
    const double pq = sum_parts(part_pq, nparts);
    if (!(pq > 0.0)) return;  // breakdown: the state kernel records it, nothing moves
    const T alpha = (T)(st->rho / pq);
    double rr = 0.0;
    const int64_t stride = (int64_t)gridDim.x * CG_THREADS;
    for (int64_t i = (int64_t)blockIdx.x * CG_THREADS + threadIdx.x; i < m; i += stride) {
        x[i] = axpy1(x[i], alpha, p[i]);
        const T ri = axpy1(r[i], -alpha, q[i]);
        r[i] = ri;
        const double rw = wide(ri);
        rr = fma(rw, rw, rr);
    }
    rr = block_sum(rr);
    if (threadIdx.x == 0) part_rr[blockIdx.x] = rr;
}

__global__ void __launch_bounds__(CG_THREADS) k_cg_state(const double *part_pq, const double *part_rr, int nparts,
                                                         CgState *st, double *hist,
                                                         cudaGraphConditionalHandle cond) {
    const double pq = sum_parts(part_pq, nparts);
    const double rr = sum_parts(part_rr, nparts);
    if (threadIdx.x != 0) return;
    if (st->iter >= st->maxit || st->breakdown) {  // cannot happen when the loop is entered correctly
        cudaGraphSetConditional(cond, 0u);
        return;
    }
    if (!(pq > 0.0)) {
        st->breakdown = 1;
        st->converged = 0;
        cudaGraphSetConditional(cond, 0u);
        return;
    }
    st->rho_prev = st->rho;
    st->rho = rr;
    st->iter += 1;
    hist[st->iter] = rr;
    st->converged = rr <= st->stop;
    cudaGraphSetConditional(cond, (st->iter < st->maxit && rr > st->stop) ? 1u : 0u);
}

template <typename T>
__global__ void __launch_bounds__(CG_THREADS) k_cg_direction(int64_t m, T *__restrict__ p, const T *__restrict__ r,
                                                             const CgState *st) {
    if (st->breakdown) return;
    const T beta = (T)(st->rho / st->rho_prev);
    const int64_t stride = (int64_t)gridDim.x * CG_THREADS;
    for (int64_t i = (int64_t)blockIdx.x * CG_THREADS + threadIdx.x; i < m; i += stride)
        p[i] = axpy1(r[i], beta, p[i]);
}

int run_spmv(const spmv_matrix *h, double alpha, const void *x, double beta, void *y, cudaStream_t s) {
    return run_product(h, alpha, x, beta, y, s);
}

}  // namespace

struct CgPlan {
    const void *b = nullptr;
    void *x = nullptr;
    double tol = -1.0;
    int32_t maxit = -1;
    int nparts = 0;
    void *r = nullptr, *p = nullptr, *q = nullptr;
    double *part = nullptr;  // 3 x nparts: p.q, r.r, b.b
    double *hist = nullptr;  // maxit + 1
    CgState *st = nullptr;
    cudaStream_t cs = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

void free_cg(spmv_matrix *h) {
    CgPlan *c = h->cg;
    if (!c) return;
    if (c->exec) cudaGraphExecDestroy(c->exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    if (c->cs) cudaStreamDestroy(c->cs);
    cudaFree(c->r);
    cudaFree(c->p);
    cudaFree(c->q);
    cudaFree(c->part);
    cudaFree(c->hist);
    cudaFree(c->st);
    delete c;
    h->cg = nullptr;
}

namespace {

template <typename T>
int capture_cg(spmv_matrix *h, CgPlan *c) {
    const int64_t m = h->m;
    const int G = c->nparts;
    T *r = (T *)c->r, *p = (T *)c->p, *q = (T *)c->q;
    const T *b = (const T *)c->b;
    T *x = (T *)c->x;
    double *part_pq = c->part, *part_rr = c->part + G, *part_bb = c->part + 2 * G;
    cudaStream_t cs = c->cs;

    SPMV_CUDA_TRY(cudaGraphCreate(&c->graph, 0));
    cudaGraphConditionalHandle cond;
    SPMV_CUDA_TRY(cudaGraphConditionalHandleCreate(&cond, c->graph, 0, cudaGraphCondAssignDefault));

    // prologue: r = b - A x, p = r, rho_0, b.b, loop condition
    SPMV_CUDA_TRY(cudaStreamBeginCaptureToGraph(cs, c->graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    int st = SPMV_OK;
    cudaError_t e = cudaMemcpyAsync(r, b, sizeof(T) * m, cudaMemcpyDeviceToDevice, cs);
    if (e != cudaSuccess) st = cuda_status(e, "cudaMemcpyAsync(r <- b)");
    if (st == SPMV_OK) st = run_spmv(h, -1.0, x, 1.0, r, cs);
    if (st == SPMV_OK) {
        k_cg_start<T><<<G, CG_THREADS, 0, cs>>>(m, r, b, p, part_rr, part_bb);
        k_cg_init<<<1, CG_THREADS, 0, cs>>>(part_rr, part_bb, G, c->st, c->hist, c->tol * c->tol, c->maxit, cond);
        e = cudaGetLastError();
        if (e != cudaSuccess) st = cuda_status(e, "CG prologue launch");
    }
    cudaGraphNode_t loop = nullptr;
    if (st == SPMV_OK) {
        cudaStreamCaptureStatus cst;
        const cudaGraphNode_t *deps = nullptr;
        size_t ndeps = 0;
        e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, nullptr, &deps, nullptr, &ndeps);
        if (e != cudaSuccess) st = cuda_status(e, "cudaStreamGetCaptureInfo");
        if (st == SPMV_OK) {
            cudaGraphNodeParams np = {};
            np.type = cudaGraphNodeTypeConditional;
            np.conditional.handle = cond;
            np.conditional.type = cudaGraphCondTypeWhile;
            np.conditional.size = 1;
            e = cudaGraphAddNode(&loop, c->graph, deps, nullptr, ndeps, &np);
            if (e != cudaSuccess) st = cuda_status(e, "cudaGraphAddNode(while)");
            if (st == SPMV_OK) {
                e = cudaStreamUpdateCaptureDependencies(cs, &loop, nullptr, 1, cudaStreamSetCaptureDependencies);
                if (e != cudaSuccess) st = cuda_status(e, "cudaStreamUpdateCaptureDependencies");
            }
            if (st == SPMV_OK) {
                // body: one CG iteration
                cudaGraph_t body = np.conditional.phGraph_out[0];
                cudaStream_t bs = nullptr;
                e = cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking);
                if (e != cudaSuccess) st = cuda_status(e, "cudaStreamCreate(body)");
                if (st == SPMV_OK) {
                    e = cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
                    if (e != cudaSuccess) st = cuda_status(e, "cudaStreamBeginCaptureToGraph(body)");
                }
                if (st == SPMV_OK) {
                    st = run_spmv(h, 1.0, p, 0.0, q, bs);
                    if (st == SPMV_OK) {
                        k_cg_dot<T><<<G, CG_THREADS, 0, bs>>>(m, p, q, part_pq);
                        k_cg_update<T><<<G, CG_THREADS, 0, bs>>>(m, x, r, p, q, part_pq, part_rr, G, c->st);
                        k_cg_state<<<1, CG_THREADS, 0, bs>>>(part_pq, part_rr, G, c->st, c->hist, cond);
                        k_cg_direction<T><<<G, CG_THREADS, 0, bs>>>(m, p, r, c->st);
                        e = cudaGetLastError();
                        if (e != cudaSuccess) st = cuda_status(e, "CG body launch");
                    }
                    cudaGraph_t bout = nullptr;
                    e = cudaStreamEndCapture(bs, &bout);
                    if (e != cudaSuccess && st == SPMV_OK) st = cuda_status(e, "cudaStreamEndCapture(body)");
                }
                if (bs) cudaStreamDestroy(bs);
            }
        }
    }
    cudaGraph_t out = nullptr;
    e = cudaStreamEndCapture(cs, &out);
    if (e != cudaSuccess && st == SPMV_OK) st = cuda_status(e, "cudaStreamEndCapture");
    if (st != SPMV_OK) return st;
    SPMV_CUDA_TRY(cudaGraphInstantiate(&c->exec, c->graph, 0));
    return SPMV_OK;
}

int build_plan(spmv_matrix *h, const void *d_b, void *d_x, double tol, int32_t maxit, cudaStream_t s) {
    CgPlan *c = h->cg;
    if (c && c->b == d_b && c->x == d_x && c->tol == tol && c->maxit == maxit) return SPMV_OK;
    free_cg(h);
    c = new (std::nothrow) CgPlan();
    if (!c) {
        set_error("spmv_cg: host allocation failed");
        return SPMV_ERR_OOM;
    }
    h->cg = c;
    c->b = d_b;
    c->x = d_x;
    c->tol = tol;
    c->maxit = maxit;
    c->nparts = 4 * (h->sm_count > 0 ? h->sm_count : 152);
    const size_t vb = vec_size(h->vt) * (size_t)h->m;
    // a plan that fails half-built is released, so a later call with the
    // same arguments builds it again instead of reusing it
    auto fail = [&](int st) {
        free_cg(h);
        return st;
    };
    cudaError_t e = dev_malloc(&c->r, vb);
    if (e == cudaSuccess) e = dev_malloc(&c->p, vb);
    if (e == cudaSuccess) e = dev_malloc(&c->q, vb);
    if (e == cudaSuccess) e = dev_malloc(&c->part, sizeof(double) * 3 * c->nparts);
    if (e == cudaSuccess) e = dev_malloc(&c->hist, sizeof(double) * ((size_t)maxit + 1));
    if (e == cudaSuccess) e = dev_malloc(&c->st, sizeof(CgState));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return fail(cuda_status(e, "spmv_cg plan"));
    // one eager product before capture: occupancy and carveout settings of
    // the kernel are resolved outside the capture
    int st = run_spmv(h, 1.0, d_b, 0.0, c->q, s);
    if (st == SPMV_OK) {
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_status(e, "spmv_cg plan");
    }
    if (st == SPMV_OK) st = h->vt == SPMV_F64 ? capture_cg<double>(h, c) : capture_cg<float>(h, c);
    if (st != SPMV_OK) return fail(st);
    return SPMV_OK;
}

}  // namespace
}  // namespace spmv

using namespace spmv;

extern "C" int spmv_cg(spmv_handle h, const void *d_b, void *d_x, double tol, int32_t maxit, double *d_rho,
                       spmv_cg_result *out, void *stream) {
    entry_reset();
    if (!h || !out) {
        set_error("spmv_cg: NULL handle or result");
        return SPMV_ERR_INVALID;
    }
    std::memset(out, 0, sizeof *out);
    if (h->m != h->n) {
        set_error("spmv_cg: matrix is %lld x %lld, not square", (long long)h->m, (long long)h->n);
        return SPMV_ERR_INVALID;
    }
    if (!(tol >= 0.0) || !std::isfinite(tol) || maxit < 0 || maxit > SPMV_CG_MAX_ITERATIONS) {
        set_error("spmv_cg: need 0 <= tol < inf and 0 <= maxit <= %d", SPMV_CG_MAX_ITERATIONS);
        return SPMV_ERR_INVALID;
    }
    if (h->m > 0 && (!d_b || !d_x)) {
        set_error("spmv_cg: NULL vector");
        return SPMV_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (h->m == 0) {
        out->converged = 1;
        if (d_rho) SPMV_CUDA_TRY(cudaMemsetAsync(d_rho, 0, sizeof(double), s));
        return SPMV_OK;
    }
    SPMV_TRY(build_plan(h, d_b, d_x, tol, maxit, s));
    CgPlan *c = h->cg;
    SPMV_CUDA_TRY(cudaGraphLaunch(c->exec, s));
    CgState st;
    SPMV_CUDA_TRY(cudaMemcpyAsync(&st, c->st, sizeof st, cudaMemcpyDeviceToHost, s));
    SPMV_CUDA_TRY(cudaStreamSynchronize(s));
    if (d_rho)
        SPMV_CUDA_TRY(cudaMemcpyAsync(d_rho, c->hist, sizeof(double) * ((size_t)st.iter + 1), cudaMemcpyDeviceToDevice, s));
    out->iterations = st.iter;
    out->converged = st.converged;
    out->breakdown = st.breakdown;
    out->rho0 = 0.0;
    out->rho = st.rho;
    out->bb = st.bb;
    SPMV_CUDA_TRY(cudaMemcpyAsync(&out->rho0, c->hist, sizeof(double), cudaMemcpyDeviceToHost, s));
    SPMV_CUDA_TRY(cudaStreamSynchronize(s));
    return SPMV_OK;
}

// Format and launch-parameter selection (Section 5.3, run-time mode steps
// 1-2, and Section 5.2 for the kernel parameters): features of the matrix,
// then a trained multi-class classifier (Section 5.4) picks one entry of a
// label table of configurations.  The classifier is a 2-layer MLP evaluated
// by one fused kernel: input transform, hidden layer with ReLU, output
// layer and argmax in a single thread block.
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "internal.cuh"

namespace spmv {

int compute_features(const spmv_matrix *h, double *d_out, cudaStream_t s);

namespace {

constexpr float BLOB_MAGIC = 2302.0f;
constexpr int MAX_HIDDEN = 256, MAX_CLASSES = 512, NCFG = 8;

// Features entering the network as log1p(value): the counts and lengths
// (n_rows, nnz, mean, var, std, min, max, median, mode, bandwidth,
// mean |i - j|); the ratios enter unchanged.
__constant__ unsigned char c_logmask[SPMV_NUM_FEATURES] = {1, 1, 0, 1, 1, 1, 1, 1, 1, 1,
                                                            0, 0, 0, 0, 1, 1, 0, 0, 0, 0};

struct Selector {
    int F = 0, H = 0, K = 0;
    float *d_w = nullptr;  // mu[F] sigma[F] W1[H][F] b1[H] W2[K][H] b2[K]
    std::vector<spmv_config> labels;
};

std::mutex g_sel_mu;
Selector g_sel[64];

__global__ void __launch_bounds__(256)
k_mlp(const double *feat, const float *w, int F, int H, int K, int *choice, float *logits) {
    __shared__ float z[SPMV_NUM_FEATURES];
    __shared__ float hid[MAX_HIDDEN];
    __shared__ float lg[MAX_CLASSES];
    const float *mu = w, *sigma = w + F, *W1 = w + 2 * F, *b1 = W1 + H * F, *W2 = b1 + H, *b2 = W2 + K * H;
    const int t = threadIdx.x;
    if (t < F) {
        double f = feat[t];
        if (c_logmask[t]) f = log1p(f);
        z[t] = (float)((f - (double)mu[t]) / (double)sigma[t]);
    }
    __syncthreads();
    for (int j = t; j < H; j += blockDim.x) {
        float a = b1[j];
        for (int k = 0; k < F; ++k) a = fmaf(W1[j * F + k], z[k], a);
        hid[j] = a > 0.f ? a : 0.f;
    }
    __syncthreads();
    for (int o = t; o < K; o += blockDim.x) {
        float a = b2[o];
        for (int j = 0; j < H; ++j) a = fmaf(W2[o * H + j], hid[j], a);
        lg[o] = a;
        if (logits) logits[o] = a;
    }
    __syncthreads();
    if (t == 0) {
        int best = 0;
        for (int o = 1; o < K; ++o)
            if (lg[o] > lg[best]) best = o;
        *choice = best;
    }
}

Selector *current_selector(int *dev_out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    if (dev_out) *dev_out = dev;
    return &g_sel[dev];
}

void default_csr_config(spmv_config *c) {
    spmv_config_default(c, SPMV_FMT_CSR);
}

}  // namespace
}  // namespace spmv

using namespace spmv;

extern "C" {

int spmv_features(spmv_handle h, double *h_out, void *stream) {
    if (!h || !h_out) {
        set_error("spmv_features: NULL argument");
        return SPMV_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    double *d = nullptr;
    SPMV_CUDA_TRY(cudaMallocAsync((void **)&d, sizeof(double) * SPMV_NUM_FEATURES, s));
    int st = compute_features(h, d, s);
    if (st == SPMV_OK) {
        cudaError_t e = cudaMemcpyAsync(h_out, d, sizeof(double) * SPMV_NUM_FEATURES, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_status(e, "spmv_features copy");
    }
    cudaFreeAsync(d, s);
    return st;
}

int spmv_selector_load(const float *h_blob, int64_t count) {
    if (!h_blob && count == 0) {  // unload: spmv_select falls back to default CSR
        Selector *sel = current_selector(nullptr);
        if (!sel) {
            set_error("spmv_selector_load: no current device");
            return SPMV_ERR_CUDA;
        }
        std::lock_guard<std::mutex> lk(g_sel_mu);
        if (sel->d_w) cudaFree(sel->d_w);
        *sel = Selector{};
        return SPMV_OK;
    }
    if (!h_blob || count < 5) {
        set_error("spmv_selector_load: blob too short");
        return SPMV_ERR_INVALID;
    }
    if (h_blob[0] != BLOB_MAGIC || h_blob[1] != 1.0f) {
        set_error("spmv_selector_load: bad magic or version");
        return SPMV_ERR_INVALID;
    }
    const int F = (int)h_blob[2], H = (int)h_blob[3], K = (int)h_blob[4];
    if (F != SPMV_NUM_FEATURES || H < 1 || H > MAX_HIDDEN || K < 1 || K > MAX_CLASSES) {
        set_error("spmv_selector_load: sizes F=%d H=%d K=%d unsupported", F, H, K);
        return SPMV_ERR_INVALID;
    }
    const int64_t nw = 2LL * F + (int64_t)H * F + H + (int64_t)K * H + K;
    if (count != 5 + nw + (int64_t)K * NCFG) {
        set_error("spmv_selector_load: %lld floats, expected %lld", (long long)count,
                  (long long)(5 + nw + (int64_t)K * NCFG));
        return SPMV_ERR_INVALID;
    }
    for (int64_t i = 0; i < F; ++i)
        if (!(h_blob[5 + F + i] > 0.0f)) {
            set_error("spmv_selector_load: nonpositive feature scale");
            return SPMV_ERR_INVALID;
        }
    int dev = 0;
    Selector *sel = current_selector(&dev);
    if (!sel) {
        set_error("spmv_selector_load: no current device");
        return SPMV_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lk(g_sel_mu);
    if (sel->d_w) cudaFree(sel->d_w);
    sel->d_w = nullptr;
    sel->K = 0;
    SPMV_CUDA_TRY(cudaMalloc((void **)&sel->d_w, sizeof(float) * nw));
    SPMV_CUDA_TRY(cudaMemcpy(sel->d_w, h_blob + 5, sizeof(float) * nw, cudaMemcpyHostToDevice));
    sel->labels.assign(K, spmv_config{});
    for (int k = 0; k < K; ++k) {
        const float *c = h_blob + 5 + nw + (int64_t)k * NCFG;
        spmv_config &o = sel->labels[k];
        o.format = (int32_t)c[0];
        o.threads_per_block = (int32_t)c[1];
        o.threads_per_row = (int32_t)c[2];
        o.unroll = (int32_t)c[3];
        o.regcap = (int32_t)c[4];
        o.carveout = (int32_t)c[5];
        o.bsr_block = (int32_t)c[6];
        o.hyb_ell_width = (int32_t)c[7];
    }
    sel->F = F;
    sel->H = H;
    sel->K = K;
    return SPMV_OK;
}

int spmv_selector_infer(const double *h_features, float *h_logits, int32_t *choice, void *stream) {
    if (!h_features || !choice) {
        set_error("spmv_selector_infer: NULL argument");
        return SPMV_ERR_INVALID;
    }
    Selector *sel = current_selector(nullptr);
    if (!sel || sel->K == 0) {
        set_error("spmv_selector_infer: no selector loaded on this device");
        return SPMV_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    char *buf = nullptr;
    const size_t fb = sizeof(double) * SPMV_NUM_FEATURES, lb = sizeof(float) * sel->K;
    SPMV_CUDA_TRY(cudaMallocAsync((void **)&buf, fb + 16 + lb, s));
    double *d_f = reinterpret_cast<double *>(buf);
    int *d_c = reinterpret_cast<int *>(buf + fb);
    float *d_l = reinterpret_cast<float *>(buf + fb + 16);
    cudaError_t e = cudaMemcpyAsync(d_f, h_features, fb, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        k_mlp<<<1, 256, 0, s>>>(d_f, sel->d_w, sel->F, sel->H, sel->K, d_c, d_l);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(choice, d_c, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && h_logits) e = cudaMemcpyAsync(h_logits, d_l, lb, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFreeAsync(buf, s);
    if (e != cudaSuccess) return cuda_status(e, "spmv_selector_infer");
    return SPMV_OK;
}

int spmv_select(spmv_handle h, spmv_config *out_cfg, double *h_features, void *stream) {
    if (!h || !out_cfg) {
        set_error("spmv_select: NULL argument");
        return SPMV_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    Selector *sel = current_selector(nullptr);
    const bool have = sel && sel->K > 0;
    char *buf = nullptr;
    const size_t fb = sizeof(double) * SPMV_NUM_FEATURES;
    SPMV_CUDA_TRY(cudaMallocAsync((void **)&buf, fb + 16, s));
    double *d_f = reinterpret_cast<double *>(buf);
    int *d_c = reinterpret_cast<int *>(buf + fb);
    int st = compute_features(h, d_f, s);
    int choice = -1;
    double hf[SPMV_NUM_FEATURES];
    if (st == SPMV_OK) {
        cudaError_t e = cudaSuccess;
        if (have) {
            k_mlp<<<1, 256, 0, s>>>(d_f, sel->d_w, sel->F, sel->H, sel->K, d_c, nullptr);
            e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaMemcpyAsync(&choice, d_c, sizeof(int), cudaMemcpyDeviceToHost, s);
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(hf, d_f, fb, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_status(e, "spmv_select");
    }
    cudaFreeAsync(buf, s);
    if (st != SPMV_OK) return st;
    if (h_features) std::memcpy(h_features, hf, fb);
    if (have && choice >= 0 && choice < sel->K) *out_cfg = sel->labels[choice];
    else default_csr_config(out_cfg);  // no selector: default CSR (Section 3.1's baseline)
    return SPMV_OK;
}

}  // extern "C"

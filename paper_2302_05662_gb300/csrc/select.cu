// Format and launch-parameter selection (Section 5.3, run-time mode, and
// Section 5.2 for the kernel parameters): features of the matrix, then a
// trained multi-class classifier (Section 5.4) picks one entry of a label
// table of configurations.  The classifier is a 2-layer MLP evaluated by one
// fused kernel: input transform, hidden layer with ReLU, output layer and
// argmax in a single thread block.  A version-2 selector also carries a
// linear time head on the hidden layer (predicted log-time of every label
// configuration and of default CSR; the regression alternative of Section
// 5.4) and a per-format conversion-cost model, which together decide whether
// converting pays off over the expected number of products (Section 5.3
// steps 3-4).
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "internal.cuh"

namespace spmv {

int compute_features(const spmv_matrix *h, double *d_out, cudaStream_t s);

namespace {

constexpr float BLOB_MAGIC = 2302.0f;
constexpr int MAX_HIDDEN = 256, MAX_CLASSES = 512, NCFG = 8, NFMT = 6, NPACK = 3;

// Features entering the network as log1p(value): the counts and lengths
// (n_rows, nnz, mean, var, std, min, max, median, mode, bandwidth,
// mean |i - j|); the ratios enter unchanged.
__constant__ unsigned char c_logmask[SPMV_NUM_FEATURES] = {1, 1, 0, 1, 1, 1, 1, 1, 1, 1,
                                                            0, 0, 0, 0, 1, 1, 0, 0, 0, 0};

struct Selector {
    int F = 0, H = 0, K = 0, version = 0;
    // device: mu[F] sigma[F] W1[H][F] b1[H] W2[K][H] b2[K] (+ W3[K+1][H] b3[K+1])
    float *d_w = nullptr;
    std::vector<spmv_config> labels;
    std::vector<float> pack;  // version 2: NFMT x {a, b_per_nnz, c_per_row} in microseconds
};

std::mutex g_sel_mu;
// per device: slot 0 the selector for every value type, slots 1..3 one for
// fp64 / fp32 / bf16 values that takes precedence when loaded
Selector g_sel[64][4];

__global__ void __launch_bounds__(256)
k_mlp(const double *feat, const float *w, int F, int H, int K, int time_head, int *choice, float *logits,
      float *logt) {
    __shared__ float z[SPMV_NUM_FEATURES];
    __shared__ float hid[MAX_HIDDEN];
    __shared__ float lg[MAX_CLASSES];
    const float *mu = w, *sigma = w + F, *W1 = w + 2 * F, *b1 = W1 + H * F, *W2 = b1 + H, *b2 = W2 + K * H;
    const float *W3 = b2 + K, *b3 = W3 + (K + 1) * H;
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
    if (time_head && logt) {
        for (int o = t; o <= K; o += blockDim.x) {
            float a = b3[o];
            for (int j = 0; j < H; ++j) a = fmaf(W3[o * H + j], hid[j], a);
            logt[o] = a;
        }
    }
    __syncthreads();
    if (t == 0) {
        int best = 0;
        for (int o = 1; o < K; ++o)
            if (lg[o] > lg[best]) best = o;
        *choice = best;
    }
}

Selector *current_selector(int *dev_out, int slot = 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    if (dev_out) *dev_out = dev;
    return &g_sel[dev][slot];
}

// the selector a handle uses: its value type's if loaded, else the shared one
Selector *selector_for(const spmv_matrix *h) {
    Selector *own = current_selector(nullptr, 1 + h->vt);
    if (own && own->K > 0) return own;
    return current_selector(nullptr, 0);
}

void default_csr_config(spmv_config *c) { spmv_config_default(c, SPMV_FMT_CSR); }

// the label class whose (format, block size, lanes per row, block size r)
// matches a resolved configuration; -1 if none
int class_of(const Selector *sel, const spmv_config &c, int default_tpr) {
    for (int k = 0; k < sel->K; ++k) {
        const spmv_config &l = sel->labels[k];
        if (l.format != c.format || l.threads_per_block != c.threads_per_block) continue;
        const int ltpr = l.threads_per_row == 0 ? (c.format == SPMV_FMT_CSR ? default_tpr : 1) : l.threads_per_row;
        const int ctpr = c.format == SPMV_FMT_CSR || c.format == SPMV_FMT_BSR ? c.threads_per_row : 1;
        if (c.format == SPMV_FMT_CSR || c.format == SPMV_FMT_BSR) {
            if (ltpr != ctpr) continue;
        }
        if (c.format == SPMV_FMT_BSR && (l.bsr_block == 0 ? 4 : l.bsr_block) != c.bsr_block) continue;
        return k;
    }
    return -1;
}

// features, classifier (and time head) for one handle; choice/logt on host
int run_selector(const spmv_matrix *h, const Selector *sel, cudaStream_t s, double *hf, int *choice,
                 std::vector<float> *logt) {
    const bool have = sel && sel->K > 0;
    const bool th = have && sel->version >= 2 && logt;
    char *buf = nullptr;
    const size_t fb = sizeof(double) * SPMV_NUM_FEATURES;
    const size_t tb = th ? sizeof(float) * (sel->K + 1) : 0;
    SPMV_CUDA_TRY(dev_malloc_async((void **)&buf, fb + 16 + tb + 16, s));
    double *d_f = reinterpret_cast<double *>(buf);
    int *d_c = reinterpret_cast<int *>(buf + fb);
    float *d_t = reinterpret_cast<float *>(buf + fb + 16);
    int st = compute_features(h, d_f, s);
    *choice = -1;
    if (st == SPMV_OK) {
        cudaError_t e = cudaSuccess;
        if (have) {
            k_mlp<<<1, 256, 0, s>>>(d_f, sel->d_w, sel->F, sel->H, sel->K, th ? 1 : 0, d_c, nullptr,
                                    th ? d_t : nullptr);
            e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaMemcpyAsync(choice, d_c, sizeof(int), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess && th) {
                logt->resize(sel->K + 1);
                e = cudaMemcpyAsync(logt->data(), d_t, tb, cudaMemcpyDeviceToHost, s);
            }
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(hf, d_f, fb, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_status(e, "selector");
    }
    cudaFreeAsync(buf, s);
    return st;
}

}  // namespace
}  // namespace spmv

using namespace spmv;

extern "C" {

int spmv_features(spmv_handle h, double *h_out, void *stream) {
    entry_reset();
    if (!h || !h_out) {
        set_error("spmv_features: NULL argument");
        return SPMV_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    double *d = nullptr;
    SPMV_CUDA_TRY(dev_malloc_async((void **)&d, sizeof(double) * SPMV_NUM_FEATURES, s));
    int st = compute_features(h, d, s);
    if (st == SPMV_OK) {
        cudaError_t e = cudaMemcpyAsync(h_out, d, sizeof(double) * SPMV_NUM_FEATURES, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_status(e, "spmv_features copy");
    }
    cudaFreeAsync(d, s);
    return st;
}

namespace {
int selector_load_slot(int slot, const float *h_blob, int64_t count) {
    if (!h_blob && count == 0) {  // unload: spmv_select falls back to default CSR
        Selector *sel = current_selector(nullptr, slot);
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
    const int version = h_blob[1] == 1.0f ? 1 : h_blob[1] == 2.0f ? 2 : 0;
    if (h_blob[0] != BLOB_MAGIC || version == 0) {
        set_error("spmv_selector_load: bad magic or version");
        return SPMV_ERR_INVALID;
    }
    const int F = (int)h_blob[2], H = (int)h_blob[3], K = (int)h_blob[4];
    if (F != SPMV_NUM_FEATURES || H < 1 || H > MAX_HIDDEN || K < 1 || K > MAX_CLASSES) {
        set_error("spmv_selector_load: sizes F=%d H=%d K=%d unsupported", F, H, K);
        return SPMV_ERR_INVALID;
    }
    const int64_t nw1 = 2LL * F + (int64_t)H * F + H + (int64_t)K * H + K;
    const int64_t nw2 = version >= 2 ? (int64_t)(K + 1) * H + (K + 1) : 0;
    const int64_t npack = version >= 2 ? NFMT * NPACK : 0;
    const int64_t expect = 5 + nw1 + (int64_t)K * NCFG + nw2 + npack;
    if (count != expect) {
        set_error("spmv_selector_load: %lld floats, expected %lld", (long long)count, (long long)expect);
        return SPMV_ERR_INVALID;
    }
    for (int64_t i = 0; i < F; ++i)
        if (!(h_blob[5 + F + i] > 0.0f)) {
            set_error("spmv_selector_load: nonpositive feature scale");
            return SPMV_ERR_INVALID;
        }
    int dev = 0;
    Selector *sel = current_selector(&dev, slot);
    if (!sel) {
        set_error("spmv_selector_load: no current device");
        return SPMV_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lk(g_sel_mu);
    if (sel->d_w) cudaFree(sel->d_w);
    *sel = Selector{};
    // device layout: network weights, then (version 2) the time head
    std::vector<float> w(h_blob + 5, h_blob + 5 + nw1);
    const float *tail = h_blob + 5 + nw1 + (int64_t)K * NCFG;
    w.insert(w.end(), tail, tail + nw2);
    SPMV_CUDA_TRY(dev_malloc((void **)&sel->d_w, sizeof(float) * w.size()));
    SPMV_CUDA_TRY(cudaMemcpy(sel->d_w, w.data(), sizeof(float) * w.size(), cudaMemcpyHostToDevice));
    sel->labels.assign(K, spmv_config{});
    for (int k = 0; k < K; ++k) {
        const float *c = h_blob + 5 + nw1 + (int64_t)k * NCFG;
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
    if (version >= 2) sel->pack.assign(tail + nw2, tail + nw2 + npack);
    sel->F = F;
    sel->H = H;
    sel->K = K;
    sel->version = version;
    return SPMV_OK;
}
}  // namespace

int spmv_selector_load(const float *h_blob, int64_t count) {
    entry_reset();
    return selector_load_slot(0, h_blob, count);
}

int spmv_selector_load_vt(int32_t value_type, const float *h_blob, int64_t count) {
    entry_reset();
    if (value_type != SPMV_F64 && value_type != SPMV_F32 && value_type != SPMV_BF16) {
        set_error("spmv_selector_load_vt: unknown value type %d", value_type);
        return SPMV_ERR_INVALID;
    }
    return selector_load_slot(1 + value_type, h_blob, count);
}

int spmv_selector_infer(const double *h_features, float *h_logits, int32_t *choice, void *stream) {
    entry_reset();
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
    SPMV_CUDA_TRY(dev_malloc_async((void **)&buf, fb + 16 + lb, s));
    double *d_f = reinterpret_cast<double *>(buf);
    int *d_c = reinterpret_cast<int *>(buf + fb);
    float *d_l = reinterpret_cast<float *>(buf + fb + 16);
    cudaError_t e = cudaMemcpyAsync(d_f, h_features, fb, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        k_mlp<<<1, 256, 0, s>>>(d_f, sel->d_w, sel->F, sel->H, sel->K, 0, d_c, d_l, nullptr);
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
    entry_reset();
    if (!h || !out_cfg) {
        set_error("spmv_select: NULL argument");
        return SPMV_ERR_INVALID;
    }
    Selector *sel = selector_for(h);
    double hf[SPMV_NUM_FEATURES];
    int choice = -1;
    SPMV_TRY(run_selector(h, sel, (cudaStream_t)stream, hf, &choice, nullptr));
    if (h_features) std::memcpy(h_features, hf, sizeof hf);
    if (sel && sel->K > 0 && choice >= 0 && choice < sel->K) *out_cfg = sel->labels[choice];
    else default_csr_config(out_cfg);  // no selector: default CSR (Section 3.1's baseline)
    return SPMV_OK;
}

int spmv_select_runtime(spmv_handle h, int64_t expected_runs, spmv_config *out_cfg, spmv_runtime_decision *out,
                        void *stream) {
    entry_reset();
    if (!h || !out_cfg || !out || expected_runs < 0) {
        set_error("spmv_select_runtime: bad argument");
        return SPMV_ERR_INVALID;
    }
    Selector *sel = selector_for(h);
    if (!sel || sel->K == 0 || sel->version < 2) {
        set_error("spmv_select_runtime: needs a loaded selector with a time head (blob version 2)");
        return SPMV_ERR_INVALID;
    }
    const auto t0 = std::chrono::steady_clock::now();
    double hf[SPMV_NUM_FEATURES];
    int choice = -1;
    std::vector<float> logt;
    SPMV_TRY(run_selector(h, sel, (cudaStream_t)stream, hf, &choice, &logt));
    const double select_us =
        std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now() - t0).count();
    std::memset(out, 0, sizeof *out);
    const spmv_config &pick = sel->labels[choice];
    *out_cfg = pick;
    // the handle's current configuration: a label class, or default CSR
    const int dtpr = default_tpr(h);
    int cur = class_of(sel, h->cfg, dtpr);
    const bool is_default = h->cfg.format == SPMV_FMT_CSR && h->cfg.threads_per_block == 256 &&
                            h->cfg.threads_per_row == dtpr;
    double t_cur;
    if (is_default || cur < 0) {
        t_cur = std::exp((double)logt[sel->K]);  // default-CSR time head
        cur = -1;
    } else {
        t_cur = std::exp((double)logt[cur]);
    }
    const double t_sel = std::exp((double)logt[choice]);
    // conversion cost of the selected format; a change of launch parameters
    // only (same packed arrays) costs nothing
    double pack_us = 0.0;
    const bool same_pack = pick.format == h->cfg.format &&
                           (pick.format == SPMV_FMT_ELL || pick.format == SPMV_FMT_COO ||
                            pick.format == SPMV_FMT_HYB || pick.format == SPMV_FMT_SELL ||
                            (pick.format == SPMV_FMT_CSR && pick.threads_per_row == h->cfg.threads_per_row));
    if (!same_pack && pick.format >= 0 && pick.format < NFMT) {
        const float *c = sel->pack.data() + pick.format * NPACK;
        pack_us = std::max(0.0, (double)c[0] + (double)c[1] * (double)h->nnz + (double)c[2] * (double)h->m);
    }
    out->current_class = cur;
    out->selected_class = choice;
    out->predicted_us_current = t_cur;
    out->predicted_us_selected = t_sel;
    out->predicted_pack_us = pack_us;
    out->measured_select_us = select_us;
    const double gain = (t_cur - t_sel) * (double)expected_runs;
    out->convert = gain > select_us + pack_us ? 1 : 0;
    return SPMV_OK;
}

}  // extern "C"

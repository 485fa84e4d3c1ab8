// perf_lpc.cu -- C ABI of the learned block preconditioner (perf.h) and of
// the exact block-Jacobi baseline.
//
// The network (k_lpc.cu) maps per-voxel features of one Gauss-Newton system
// to P_v = D_v^{-1/2} (L_v L_v^T + eps I) D_v^{-1/2}; perf_pcg_set_blocks hands
// the blocks to Algorithm 2 (PERF_PRECOND_BLOCK4), with Jacobi for the shell
// texels.  Training runs entirely in this library's kernels: forward
// convolutions, the head and its loss, the backward convolutions, Adam.
#include <cmath>
#include <cstring>
#include <new>
#include <random>
#include <string>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "../../include/perf.h"
#include "perf_kernels.h"

namespace perf {
cudaError_t lpc_conv_fwd(const __nv_bfloat16* in, const __nv_bfloat16* W, const float* bias,
                         __nv_bfloat16* out, int G, int relu, cudaStream_t st);
cudaError_t lpc_conv_bwd_w(const __nv_bfloat16* in, const __nv_bfloat16* gpre, float* dW,
                           float* dB, int G, cudaStream_t st);
cudaError_t lpc_conv_flip(const __nv_bfloat16* W, __nv_bfloat16* Wt, cudaStream_t st);
int lpc_conv_error();
void lpc_conv_set_first_wait_limit(uint32_t rounds);
cudaError_t lpc_relu_bwd(__nv_bfloat16* g, const __nv_bfloat16* act, long long n, cudaStream_t st);
cudaError_t lpc_head_train(const __nv_bfloat16* o, const float* ahat, const float* xi,
                           const unsigned char* mask, __nv_bfloat16* gout, long long V, float scale,
                           double* loss, cudaStream_t st);
cudaError_t lpc_head_infer(const __nv_bfloat16* o, const float* diag, float* blocks, long long V,
                           cudaStream_t st);
cudaError_t lpc_features(const float* x, const float* grad, const float* diag, const float* cross,
                         double* stats, __nv_bfloat16* feat, long long V, cudaStream_t st);
cudaError_t lpc_adam(float* w, const float* gw, float* m, float* v2, __nv_bfloat16* wb, int n,
                     float lr, int step, cudaStream_t st);
cudaError_t lpc_to_bf16(const float* a, __nv_bfloat16* b, int n, cudaStream_t st);
cudaError_t launch_block_jacobi(const float* diag, const float* cross, float* blocks, long long V,
                                cudaStream_t st);
cudaError_t launch_dscale(const float* diag, const float* in, float* out, unsigned char* mask,
                          long long V, cudaStream_t st);
}  // namespace perf

namespace {
constexpr int kLayers = 4;
constexpr int kC = 16;
constexpr int kWPer = 27 * kC * kC;           // weights per layer
constexpr int kLayerSize = kWPer + kC;        // + bias
constexpr int kNW = kLayers * kLayerSize;
}  // namespace

struct perf_lpc {
    float* w = nullptr;        // FP32 master: per layer W[27][16][16] then b[16]
    float* gw = nullptr;       // gradient
    float* m = nullptr;
    float* v2 = nullptr;
    __nv_bfloat16* wb = nullptr;   // bf16 copy (same layout)
    __nv_bfloat16* wt = nullptr;   // flipped / transposed weights (one layer)
    float* zero_bias = nullptr;
    double* dloss = nullptr;
    double* stats = nullptr;   // feature normalisation (6 doubles)
    // activations for the largest G seen
    long long cap_v = 0;
    __nv_bfloat16* act[kLayers + 1] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    __nv_bfloat16* g0 = nullptr;
    __nv_bfloat16* g1 = nullptr;
    int step = 0;
    std::string err;
};

namespace {

#define LK(call)                                                                  \
    do {                                                                          \
        cudaError_t e_ = (call);                                                  \
        if (e_ != cudaSuccess) {                                                  \
            L->err = std::string(#call) + ": " + cudaGetErrorString(e_);          \
            return PERF_ERR_CUDA;                                                 \
        }                                                                         \
    } while (0)

inline cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

perf_status ensure_acts(perf_lpc* L, long long V) {
    if (V <= L->cap_v) return PERF_OK;
    for (auto& a : L->act) { if (a) cudaFree(a); a = nullptr; }
    if (L->g0) cudaFree(L->g0);
    if (L->g1) cudaFree(L->g1);
    L->g0 = L->g1 = nullptr;
    for (int i = 1; i <= kLayers; ++i) LK(cudaMalloc(&L->act[i], sizeof(__nv_bfloat16) * kC * (size_t)V));
    LK(cudaMalloc(&L->g0, sizeof(__nv_bfloat16) * kC * (size_t)V));
    LK(cudaMalloc(&L->g1, sizeof(__nv_bfloat16) * kC * (size_t)V));
    L->cap_v = V;
    return PERF_OK;
}

// Forward through all layers: act[0] = feat (borrowed), act[4] = head outputs.
perf_status forward(perf_lpc* L, int G, const __nv_bfloat16* feat, cudaStream_t st) {
    const long long V = (long long)G * G * G;
    perf_status ps = ensure_acts(L, V);
    if (ps != PERF_OK) return ps;
    const __nv_bfloat16* in = feat;
    for (int l = 0; l < kLayers; ++l) {
        const __nv_bfloat16* W = L->wb + (size_t)l * kLayerSize;
        const float* b = L->w + (size_t)l * kLayerSize + kWPer;
        LK(perf::lpc_conv_fwd(in, W, b, L->act[l + 1], G, l < kLayers - 1 ? 1 : 0, st));
        in = L->act[l + 1];
    }
    return PERF_OK;
}

// Loss and gradient of the weights (into L->gw) for one system.
perf_status loss_grad(perf_lpc* L, int G, const __nv_bfloat16* feat, const float* ahat,
                      const float* xi, const unsigned char* mask, double xi_norm2,
                      cudaStream_t st) {
    const long long V = (long long)G * G * G;
    perf_status ps = forward(L, G, feat, st);
    if (ps != PERF_OK) return ps;
    LK(cudaMemsetAsync(L->dloss, 0, sizeof(double), st));
    LK(cudaMemsetAsync(L->gw, 0, sizeof(float) * kNW, st));
    const float scale = xi_norm2 > 0.0 ? (float)(1.0 / xi_norm2) : 1.0f;
    LK(perf::lpc_head_train(L->act[kLayers], ahat, xi, mask, L->g0, V, scale, L->dloss, st));
    __nv_bfloat16* g = L->g0;
    __nv_bfloat16* gn = L->g1;
    for (int l = kLayers - 1; l >= 0; --l) {
        const __nv_bfloat16* in = l == 0 ? feat : L->act[l];
        float* dW = L->gw + (size_t)l * kLayerSize;
        LK(perf::lpc_conv_bwd_w(in, g, dW, dW + kWPer, G, st));
        if (l == 0) break;
        LK(perf::lpc_conv_flip(L->wb + (size_t)l * kLayerSize, L->wt, st));
        LK(perf::lpc_conv_fwd(g, L->wt, L->zero_bias, gn, G, 0, st));
        LK(perf::lpc_relu_bwd(gn, L->act[l], (long long)kC * V, st));
        __nv_bfloat16* t = g;
        g = gn;
        gn = t;
    }
    return PERF_OK;
}

double host_norm2(const float* d_xi, long long V, cudaStream_t st, bool& ok) {
    std::vector<float> h(4 * (size_t)V);
    ok = cudaMemcpyAsync(h.data(), d_xi, sizeof(float) * h.size(), cudaMemcpyDeviceToHost, st) ==
             cudaSuccess &&
         cudaStreamSynchronize(st) == cudaSuccess;
    double s = 0.0;
    for (float v : h) s += (double)v * v;
    return s;
}

}  // namespace

extern "C" {

int64_t perf_lpc_weight_count(void) { return kNW; }

perf_status perf_lpc_create(perf_lpc** out, uint64_t seed) {
    if (!out) return PERF_ERR_INVALID_ARG;
    *out = nullptr;
    perf_lpc* L = new (std::nothrow) perf_lpc();
    if (!L) return PERF_ERR_INVALID_ARG;
    std::vector<float> h(kNW, 0.0f);
    std::mt19937_64 rng(seed);
    std::normal_distribution<float> nd(0.0f, 1.0f);
    const int fan_in[kLayers] = {27 * 12, 27 * kC, 27 * kC, 27 * kC};
    for (int l = 0; l < kLayers; ++l) {
        float* W = h.data() + (size_t)l * kLayerSize;
        const float sd = (l < kLayers - 1) ? std::sqrt(2.0f / fan_in[l]) : 1e-3f;
        for (int i = 0; i < kWPer; ++i) W[i] = sd * nd(rng);
        float* b = W + kWPer;
        if (l == kLayers - 1)   // head starts at L = I: softplus(o) = 1 on the diagonal
            for (int c = 0; c < 4; ++c) b[c] = std::log(std::exp(1.0f) - 1.0f);
    }
    cudaError_t e = cudaMalloc(&L->w, sizeof(float) * kNW);
    if (e == cudaSuccess) e = cudaMalloc(&L->gw, sizeof(float) * kNW);
    if (e == cudaSuccess) e = cudaMalloc(&L->m, sizeof(float) * kNW);
    if (e == cudaSuccess) e = cudaMalloc(&L->v2, sizeof(float) * kNW);
    if (e == cudaSuccess) e = cudaMalloc(&L->wb, sizeof(__nv_bfloat16) * kNW);
    if (e == cudaSuccess) e = cudaMalloc(&L->wt, sizeof(__nv_bfloat16) * kWPer);
    if (e == cudaSuccess) e = cudaMalloc(&L->zero_bias, sizeof(float) * kC);
    if (e == cudaSuccess) e = cudaMalloc(&L->dloss, sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&L->stats, 6 * sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpy(L->w, h.data(), sizeof(float) * kNW, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(L->m, 0, sizeof(float) * kNW);
    if (e == cudaSuccess) e = cudaMemset(L->v2, 0, sizeof(float) * kNW);
    if (e == cudaSuccess) e = cudaMemset(L->zero_bias, 0, sizeof(float) * kC);
    if (e == cudaSuccess) e = perf::lpc_to_bf16(L->w, L->wb, kNW, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        perf_lpc_destroy(L);
        return PERF_ERR_CUDA;
    }
    *out = L;
    return PERF_OK;
}

perf_status perf_lpc_destroy(perf_lpc* L) {
    if (!L) return PERF_ERR_INVALID_ARG;
    void* bufs[] = {L->w, L->gw, L->m, L->v2, L->wb, L->wt, L->zero_bias, L->dloss, L->stats,
                    L->g0, L->g1};
    for (void* b : bufs)
        if (b) cudaFree(b);
    for (auto& a : L->act)
        if (a) cudaFree(a);
    delete L;
    return PERF_OK;
}

const char* perf_lpc_last_error(const perf_lpc* L) { return L ? L->err.c_str() : "null lpc"; }

perf_status perf_lpc_get_weights(perf_lpc* L, float* host_out) {
    if (!L || !host_out) return PERF_ERR_INVALID_ARG;
    LK(cudaMemcpy(host_out, L->w, sizeof(float) * kNW, cudaMemcpyDeviceToHost));
    return PERF_OK;
}

perf_status perf_lpc_set_weights(perf_lpc* L, const float* host_in) {
    if (!L || !host_in) return PERF_ERR_INVALID_ARG;
    LK(cudaMemcpy(L->w, host_in, sizeof(float) * kNW, cudaMemcpyHostToDevice));
    LK(perf::lpc_to_bf16(L->w, L->wb, kNW, nullptr));
    LK(cudaDeviceSynchronize());
    return PERF_OK;
}

perf_status perf_lpc_features(perf_lpc* L, int32_t G, const float* x, const float* grad,
                              const float* diag, const float* cross, void* feat_out, void* stream) {
    if (!L || G < 2 || !x || !grad || !diag || !feat_out) return PERF_ERR_INVALID_ARG;
    const long long V = (long long)G * G * G;
    LK(perf::lpc_features(x, grad, diag, cross, L->stats, static_cast<__nv_bfloat16*>(feat_out), V,
                          S(stream)));
    return PERF_OK;
}

perf_status perf_lpc_loss_grad(perf_lpc* L, int32_t G, const void* feat, const float* ahat,
                               const float* xi, const uint8_t* mask, double* loss_out,
                               float* grad_out, void* stream) {
    if (!L || G < 2 || !feat || !ahat || !xi) return PERF_ERR_INVALID_ARG;
    const long long V = (long long)G * G * G;
    bool ok = true;
    const double n2 = host_norm2(xi, V, S(stream), ok);
    if (!ok) return PERF_ERR_CUDA;
    perf_status ps = loss_grad(L, G, static_cast<const __nv_bfloat16*>(feat), ahat, xi, mask, n2,
                               S(stream));
    if (ps != PERF_OK) return ps;
    if (grad_out)
        LK(cudaMemcpyAsync(grad_out, L->gw, sizeof(float) * kNW, cudaMemcpyDeviceToDevice, S(stream)));
    if (loss_out) {
        LK(cudaMemcpyAsync(loss_out, L->dloss, sizeof(double), cudaMemcpyDeviceToHost, S(stream)));
        LK(cudaStreamSynchronize(S(stream)));
        // a convolution whose bounded waits ran out has left its outputs incomplete
        const int ce = perf::lpc_conv_error();
        if (ce != 0) {
            L->err = "loss_grad: a convolution's bounded wait gave up";
            return ce > 0 ? PERF_ERR_TIMEOUT : PERF_ERR_CUDA;
        }
    }
    return PERF_OK;
}

perf_status perf_lpc_train_step(perf_lpc* L, int32_t G, const void* feat, const float* ahat,
                                const float* xi, const uint8_t* mask, float lr, double* loss_out,
                                void* stream) {
    perf_status ps = perf_lpc_loss_grad(L, G, feat, ahat, xi, mask, loss_out, nullptr, stream);
    if (ps != PERF_OK) return ps;
    L->step += 1;
    LK(perf::lpc_adam(L->w, L->gw, L->m, L->v2, L->wb, kNW, lr, L->step, S(stream)));
    return PERF_OK;
}

perf_status perf_lpc_head_outputs(perf_lpc* L, int32_t G, const void* feat, void* out,
                                  void* stream) {
    if (!L || G < 2 || !feat || !out) return PERF_ERR_INVALID_ARG;
    perf_status ps = forward(L, G, static_cast<const __nv_bfloat16*>(feat), S(stream));
    if (ps != PERF_OK) return ps;
    const long long V = (long long)G * G * G;
    LK(cudaMemcpyAsync(out, L->act[kLayers], sizeof(__nv_bfloat16) * kC * (size_t)V,
                       cudaMemcpyDeviceToDevice, S(stream)));
    return PERF_OK;
}

perf_status perf_lpc_infer(perf_lpc* L, int32_t G, const void* feat, const float* diag,
                           float* blocks_out, void* stream) {
    if (!L || G < 2 || !feat || !diag || !blocks_out) return PERF_ERR_INVALID_ARG;
    perf_status ps = forward(L, G, static_cast<const __nv_bfloat16*>(feat), S(stream));
    if (ps != PERF_OK) return ps;
    const long long V = (long long)G * G * G;
    LK(perf::lpc_head_infer(L->act[kLayers], diag, blocks_out, V, S(stream)));
    return PERF_OK;
}

perf_status perf_lpc_conv_status(int32_t* timed_out) {
    if (!timed_out) return PERF_ERR_INVALID_ARG;
    const int v = perf::lpc_conv_error();
    if (v < 0) return PERF_ERR_CUDA;
    *timed_out = v;
    return PERF_OK;
}

perf_status perf_lpc_test_conv_wait_limit(uint32_t rounds) {
    perf::lpc_conv_set_first_wait_limit(rounds);
    return PERF_OK;
}

perf_status perf_lpc_dscale(int32_t G, const float* diag, const float* in, float* out,
                            uint8_t* mask_out, void* stream) {
    if (G < 2 || !diag || !in || !out) return PERF_ERR_INVALID_ARG;
    const long long V = (long long)G * G * G;
    return perf::launch_dscale(diag, in, out, mask_out, V, S(stream)) == cudaSuccess ? PERF_OK
                                                                                     : PERF_ERR_CUDA;
}

perf_status perf_block_jacobi(int32_t G, const float* diag, const float* cross, float* blocks_out,
                              void* stream) {
    if (G < 2 || !diag || !cross || !blocks_out) return PERF_ERR_INVALID_ARG;
    const long long V = (long long)G * G * G;
    return perf::launch_block_jacobi(diag, cross, blocks_out, V, S(stream)) == cudaSuccess
               ? PERF_OK
               : PERF_ERR_CUDA;
}

}  // extern "C"

namespace perf {
// Blocks of the learned preconditioner for one system (used by perf_gn_solve).
cudaError_t lpc_blocks_for(perf_lpc* L, int G, const float* x, const float* grad, const float* diag,
                           const float* cross, __nv_bfloat16* feat, float* blocks, cudaStream_t st) {
    const long long V = (long long)G * G * G;
    cudaError_t e = lpc_features(x, grad, diag, cross, L->stats, feat, V, st);
    if (e != cudaSuccess) return e;
    if (forward(L, G, feat, st) != PERF_OK) return cudaErrorUnknown;
    return lpc_head_infer(L->act[kLayers], diag, blocks, V, st);
}
}  // namespace perf

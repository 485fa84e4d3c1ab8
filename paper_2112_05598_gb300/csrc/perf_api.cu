// perf_api.cu -- the C ABI of libperf (declared in include/perf.h).
//
// Host orchestration of the Gauss-Newton step (PERF Eq. 7): residual and F,
// gradient with the Jacobi diagonal, Algorithm 2 on the context's workspace,
// and Algorithm 3 evaluating F(P(x + gamma Delta)) on the device with one
// FP64 scalar read back per trial step length.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "../../include/perf.h"
#include "perf_kernels.h"

using perf::DevScene;
using perf::PcgScalars;

namespace perf {
cudaError_t lpc_blocks_for(perf_lpc* L, int G, const float* x, const float* grad, const float* diag,
                           const float* cross, __nv_bfloat16* feat, float* blocks, cudaStream_t st);
cudaError_t launch_block_jacobi(const float* diag, const float* cross, float* blocks, long long V,
                                cudaStream_t st);
int lpc_conv_error();
}  // namespace perf

struct perf_ctx {
    perf_scene scene;
    perf_options opts;
    DevScene ds;
    long long n = 0, n_rays = 0;
    int device = 0;
    float* cams = nullptr;
    // workspace (allocated on first use)
    void* r = nullptr;          // residuals, scene storage type
    float* diag = nullptr;
    float* grad = nullptr;
    float* delta = nullptr;     // Algorithm 2 vectors (FP32; p is also gathered by A p)
    float* rho = nullptr;
    float* p = nullptr;
    float* xp = nullptr;        // paired (x, p) records for A p (FP32 scenes)
    bool pair = true;           // Gauss-Newton A p reads the paired records
    // brick order of a Gauss-Newton step's PCG vectors (LayoutKey shift; 0:
    // canonical), used when the step's A p runs wholly from the store
    int brick_s = 0;
    // the fixed-iteration PCG loop of perf_gn_solve as a CUDA graph, captured
    // on an internal stream and replayed on the caller's while everything it
    // captured (the key: pointers, scene descriptor, iteration count) holds
    bool pcg_graph_on = true;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t pcg_graph = nullptr;
    std::vector<unsigned char> pcg_graph_key;
    unsigned long long pcg_graph_launches = 0;   // kernels per replay
    // coefficient-cached A p: per-sample (w_i, dH/dsigma_i) of the current
    // Gauss-Newton step, stored by its diagonal march (see k_march.cu)
    long long coef_budget = -1;        // bytes; -1 automatic, 0 off
    long long* tile_off = nullptr;     // first row of every pixel tile (n_tiles + 1)
    float* coef = nullptr;
    size_t coef_bytes = 0;             // allocated
    int* keff = nullptr;               // per ray: length of its non-zero row prefix (DevScene::keff)
    // the last perf_gn_solve step filled keff for the rays of tiles
    // [0, keff_tiles) at tile width keff_tile_w and jitter epoch keff_epoch
    bool keff_valid = false;
    long long keff_tiles = 0;
    int keff_tile_w = 0;
    uint32_t keff_epoch = 0;
    unsigned long long* d_prefix = nullptr;   // perf_coef_prefix's two sums
    long long coef_rows = 0;           // rows needed by the current tiling
    std::vector<long long> tile_off_h; // host copy of tile_off
    long long coef_tiles = 0;          // tiles [0, coef_tiles) are in the store
    int tab_tile_w = 0, tab_max_samples = 0;
    long long tab_epoch = -1;          // epoch of a jittered table (-1: not jittered)
    bool coef_used = false;            // the last Gauss-Newton step used the store
    float* Ap = nullptr;
    // shell hits of every ray (n_rays x S entries, FP64 texel coordinates),
    // valid for jitter epoch shell_tab_epoch (-1: no jitter); see ensure_shells
    float4* shell_tab = nullptr;
    long long shell_tab_epoch = -2;
    // R after each PCG iteration of the last solve (perf_pcg_history)
    double* hist = nullptr;
    long long hist_cap = 0;
    float* x_trial = nullptr;
    __nv_bfloat16* x16 = nullptr;
    __nv_bfloat16* p16 = nullptr;
    __nv_bfloat16* t16 = nullptr;
    PcgScalars* s = nullptr;
    double* dF = nullptr;
    const float* blocks = nullptr;   // caller-owned 4x4 blocks per voxel (or null)
    long long n_block = 0;
    perf_lpc* lpc = nullptr;         // learned preconditioner (not owned)
    float* cross = nullptr;          // per voxel (a s_0, a s_1, a s_2, 0)
    float* blocks_ws = nullptr;      // blocks computed each GN step
    __nv_bfloat16* feat = nullptr;   // network input features
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::string err;
    // kernel timing
    bool timing = false;
    struct KTimer {
        std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
        size_t used = 0;
        double ms = 0.0;
        long long launches = 0;
    } kt[PERF_T_COUNT];
};

namespace {

perf_status fail(perf_ctx* c, perf_status st, const std::string& msg) {
    if (c) c->err = msg;
    return st;
}

perf_status cuda_fail(perf_ctx* c, cudaError_t e, const char* where) {
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    return fail(c, PERF_ERR_CUDA, m);
}

#define CK(call)                                                     \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);     \
    } while (0)

inline cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

perf_status check_options(const perf_options* o, std::string& why) {
    if (!o) { why = "options is NULL"; return PERF_ERR_INVALID_ARG; }
    if (o->max_samples < 1 || o->max_samples > (1 << 20)) { why = "max_samples out of range"; return PERF_ERR_INVALID_ARG; }
    if (o->pcg_iters < 0) { why = "pcg_iters < 0"; return PERF_ERR_INVALID_ARG; }
    if (!(o->ls_alpha > 0.0 && o->ls_alpha < 1.0)) { why = "ls_alpha must be in (0,1)"; return PERF_ERR_INVALID_ARG; }
    if (o->ls_max < 0 || o->ls_max > 200) { why = "ls_max out of range"; return PERF_ERR_INVALID_ARG; }
    if (o->precond != PERF_PRECOND_JACOBI && o->precond != PERF_PRECOND_BLOCK4 &&
        o->precond != PERF_PRECOND_BLOCK_JACOBI) { why = "unknown preconditioner"; return PERF_ERR_INVALID_ARG; }
    if (!(o->pcg_eps_rel >= 0.0) || !(o->pcg_stall > 0.0)) { why = "pcg_eps_rel / pcg_stall invalid"; return PERF_ERR_INVALID_ARG; }
    if ((o->aux != 0 && o->aux != 1) || !(o->aux_lambda >= 0.0) || !std::isfinite(o->aux_lambda)) {
        why = "aux must be 0 or 1 and aux_lambda finite and >= 0";
        return PERF_ERR_INVALID_ARG;
    }
    if (o->precond_judge != PERF_JUDGE_RESIDUAL && o->precond_judge != PERF_JUDGE_OBJECTIVE) {
        why = "unknown precond_judge";
        return PERF_ERR_INVALID_ARG;
    }
    return PERF_OK;
}

template <typename T>
cudaError_t alloc(T** p, long long count) {
    if (*p) return cudaSuccess;
    return cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * (size_t)(count > 0 ? count : 1));
}

// Room for the residual history of a solve of up to `iters` iterations.
perf_status ensure_hist(perf_ctx* ctx, long long iters) {
    if (iters <= ctx->hist_cap) return PERF_OK;
    if (ctx->hist) cudaFree(ctx->hist);
    ctx->hist = nullptr;
    ctx->hist_cap = 0;
    CK(cudaMalloc(&ctx->hist, sizeof(double) * (size_t)iters));
    ctx->hist_cap = iters;
    return PERF_OK;
}

perf_status ensure_pcg(perf_ctx* ctx) {
    CK(alloc(&ctx->diag, ctx->n));
    CK(alloc(&ctx->grad, ctx->n));
    CK(alloc(&ctx->delta, ctx->n));
    CK(alloc(&ctx->rho, ctx->n));
    CK(alloc(&ctx->p, ctx->n));
    CK(alloc(&ctx->Ap, ctx->n));
    if (ctx->scene.dtype == PERF_BF16) CK(alloc(&ctx->p16, ctx->n));
    else CK(alloc(&ctx->xp, 2 * ctx->n));
    return PERF_OK;
}

// Prepares the coefficient store for the context's current tiling; *use =
// whether it fits the budget (automatic: the free device memory minus 6 GiB).
perf_status ensure_coef(perf_ctx* ctx, cudaStream_t st, bool* use) {
    *use = false;
    if (ctx->coef_budget == 0 || ctx->n_rays == 0) return PERF_OK;
    const perf::DevScene& d = ctx->ds;
    // with pixel jitter the rays, and so the sample counts, change with the epoch
    const long long epoch = d.jitter ? (long long)d.epoch : -1;
    if (!ctx->tile_off || ctx->tab_tile_w != d.tile_w || ctx->tab_max_samples != d.max_samples ||
        ctx->tab_epoch != epoch) {
        if (ctx->tile_off) { cudaFree(ctx->tile_off); ctx->tile_off = nullptr; }
        int* rows = nullptr;
        CK(cudaMalloc(&rows, sizeof(int) * (size_t)d.n_tiles));
        cudaError_t e = perf::launch_tile_rows(d, rows, st);
        std::vector<int> h((size_t)d.n_tiles);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h.data(), rows, sizeof(int) * (size_t)d.n_tiles, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        cudaFree(rows);
        CK(e);
        std::vector<long long> off((size_t)d.n_tiles + 1);
        off[0] = 0;
        for (long long t = 0; t < d.n_tiles; ++t) off[(size_t)t + 1] = off[(size_t)t] + h[(size_t)t];
        CK(cudaMalloc(&ctx->tile_off, sizeof(long long) * off.size()));
        CK(cudaMemcpy(ctx->tile_off, off.data(), sizeof(long long) * off.size(), cudaMemcpyHostToDevice));
        ctx->coef_rows = off.back();
        ctx->tile_off_h.swap(off);
        ctx->tab_tile_w = d.tile_w;
        ctx->tab_max_samples = d.max_samples;
        ctx->tab_epoch = epoch;
    }
    const size_t row_bytes = 32 * sizeof(float4);
    // the per-ray prefix lengths (4 bytes per ray) come out of the budget too
    const size_t keff_bytes = sizeof(int) * (size_t)ctx->n_rays;
    size_t budget;
    if (ctx->coef_budget > 0) {
        budget = (size_t)ctx->coef_budget;
    } else {
        size_t fr = 0, tot = 0;
        CK(cudaMemGetInfo(&fr, &tot));
        const size_t avail = fr + ctx->coef_bytes + (ctx->keff ? keff_bytes : 0),
                     reserve = (size_t)6 << 30;
        budget = avail > reserve ? avail - reserve : 0;
    }
    budget = budget > keff_bytes ? budget - keff_bytes : 0;
    // the longest prefix of tiles whose rows fit: those tiles' A p reads the
    // store, the rest recompute
    const std::vector<long long>& off = ctx->tile_off_h;
    long long T1 = d.n_tiles;
    if ((size_t)off.back() * row_bytes > budget) {
        const long long max_rows = (long long)(budget / row_bytes);
        T1 = (long long)(std::upper_bound(off.begin(), off.end(), max_rows) - off.begin()) - 1;
    }
    const size_t need = (size_t)(T1 > 0 ? off[(size_t)T1] : 0) * row_bytes;
    if (T1 <= 0 || need == 0) {
        if (ctx->coef) { cudaFree(ctx->coef); ctx->coef = nullptr; ctx->coef_bytes = 0; }
        ctx->coef_tiles = 0;
        return PERF_OK;
    }
    if (ctx->coef_bytes < need) {
        if (ctx->coef) { cudaFree(ctx->coef); ctx->coef = nullptr; ctx->coef_bytes = 0; }
        if (cudaMalloc(&ctx->coef, need > 0 ? need : 16) != cudaSuccess) {
            // out of memory after all (fragmentation, another user): recompute,
            // and report no store (perf_coef_info)
            cudaGetLastError();
            ctx->coef = nullptr;
            ctx->coef_bytes = 0;
            ctx->coef_tiles = 0;
            return PERF_OK;
        }
        ctx->coef_bytes = need;
    }
    if (!ctx->keff && cudaMalloc(&ctx->keff, keff_bytes) != cudaSuccess) {
        // without the prefix lengths every row is written and read
        cudaGetLastError();
        ctx->keff = nullptr;
    }
    ctx->coef_tiles = T1;
    *use = true;
    return PERF_OK;
}

bool bad_ptr(const void* p) { return p == nullptr; }

// The shell-hit table of the context's rays at the current jitter epoch:
// built on first use and whenever the rays move (pixel jitter of a new
// epoch, new options); if it cannot be allocated the marches compute the hits
// themselves in FP32.
perf_status ensure_shells(perf_ctx* ctx, cudaStream_t st) {
    perf::DevScene& d = ctx->ds;
    if (d.S == 0 || ctx->n_rays == 0) {
        d.shell_tab = nullptr;
        return PERF_OK;
    }
    const long long epoch = d.jitter ? (long long)d.epoch : -1;
    if (ctx->shell_tab && ctx->shell_tab_epoch == epoch) {
        d.shell_tab = ctx->shell_tab;
        return PERF_OK;
    }
    if (!ctx->shell_tab &&
        cudaMalloc(&ctx->shell_tab, sizeof(float4) * (size_t)ctx->n_rays * (size_t)d.S) != cudaSuccess) {
        cudaGetLastError();
        ctx->shell_tab = nullptr;
        d.shell_tab = nullptr;
        return PERF_OK;
    }
    d.shell_tab = nullptr;
    CK(perf::launch_shell_table(d, ctx->shell_tab, st));
    ctx->shell_tab_epoch = epoch;
    d.shell_tab = ctx->shell_tab;
    return PERF_OK;
}

#define SHELLS(ctx, st)                                 \
    do {                                                \
        const perf_status ps_ = ensure_shells(ctx, st); \
        if (ps_ != PERF_OK) return ps_;                 \
    } while (0)

void t_begin(perf_ctx* c, int k, cudaStream_t st) {
    if (!c->timing) return;
    auto& t = c->kt[k];
    if (t.used == t.ev.size()) {
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        t.ev.emplace_back(a, b);
    }
    cudaEventRecord(t.ev[t.used].first, st);
}

void t_end(perf_ctx* c, int k, cudaStream_t st) {
    if (!c->timing) return;
    auto& t = c->kt[k];
    cudaEventRecord(t.ev[t.used].second, st);
    ++t.used;
}

void t_harvest(perf_ctx* c) {
    for (auto& t : c->kt) {
        for (size_t i = 0; i < t.used; ++i) {
            cudaEventSynchronize(t.ev[i].second);
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, t.ev[i].first, t.ev[i].second) == cudaSuccess) t.ms += ms;
        }
        t.launches += (long long)t.used;
        t.used = 0;
    }
}

}  // namespace

extern "C" {

perf_status perf_default_options(perf_options* o) {
    if (!o) return PERF_ERR_INVALID_ARG;
    std::memset(o, 0, sizeof(*o));
    o->max_samples = 512;
    o->jitter = 0;
    o->seed = 0;
    o->epoch = 0;
    o->pcg_iters = 20;
    o->pcg_fixed = 1;
    o->pcg_eps_rel = 1e-3;
    o->pcg_stall = 0.85;
    o->ls_alpha = 0.7;
    o->ls_max = 20;
    o->project = 1;
    o->precond = PERF_PRECOND_JACOBI;
    o->aux = 0;
    o->aux_lambda = 0.1;
    return PERF_OK;
}

perf_status perf_create(perf_ctx** out, const perf_scene* sc, const perf_cameras* cams,
                        const perf_options* opts) {
    if (!out) return PERF_ERR_INVALID_ARG;
    *out = nullptr;
    if (!sc || !cams || !opts) return PERF_ERR_INVALID_ARG;
    std::string why;
    if (check_options(opts, why) != PERF_OK) return PERF_ERR_INVALID_ARG;
    if (sc->grid_res < 2 || sc->grid_res > 1024) return PERF_ERR_INVALID_ARG;
    if (sc->n_shells < 0 || sc->n_shells > PERF_MAX_SHELLS) return PERF_ERR_INVALID_ARG;
    if (sc->dtype != PERF_F32 && sc->dtype != PERF_BF16) return PERF_ERR_INVALID_ARG;
    if (sc->n_shells > 0 && (sc->env_h < 2 || sc->env_w < 2)) return PERF_ERR_INVALID_ARG;
    if (sc->env_kind != PERF_ENV_EQUIRECT && sc->env_kind != PERF_ENV_CUBE) return PERF_ERR_INVALID_ARG;
    if (sc->env_kind == PERF_ENV_CUBE && sc->n_shells > 0 && sc->env_w != 6 * sc->env_h)
        return PERF_ERR_INVALID_ARG;
    for (int s = 0; s < sc->n_shells; ++s) {
        if (!(sc->shell_radii[s] > 1.7320508f)) return PERF_ERR_INVALID_ARG;
        if (s > 0 && !(sc->shell_radii[s] > sc->shell_radii[s - 1])) return PERF_ERR_INVALID_ARG;
    }
    if (cams->n_cams < 0 || cams->width < 0 || cams->height < 0) return PERF_ERR_INVALID_ARG;
    if (cams->n_cams > 0 && (cams->width > 0 && cams->height > 0) && (!cams->c2w || !cams->focal))
        return PERF_ERR_INVALID_ARG;
    for (int c = 0; c < cams->n_cams && cams->focal; ++c)
        if (!(cams->focal[c] > 0.0f) || !std::isfinite(cams->focal[c])) return PERF_ERR_INVALID_ARG;

    perf_ctx* ctx = new (std::nothrow) perf_ctx();
    if (!ctx) return PERF_ERR_INVALID_ARG;
    ctx->scene = *sc;
    ctx->opts = *opts;
    if (sc->n_shells == 0) { ctx->scene.env_h = 0; ctx->scene.env_w = 0; }
    const long long G = sc->grid_res;
    const long long texels = (long long)ctx->scene.env_h * ctx->scene.env_w;
    ctx->n = 4 * (G * G * G + (long long)sc->n_shells * texels);
    if (ctx->n / 4 >= (1ll << 31)) {   // parameter blocks are indexed with int
        delete ctx;
        return PERF_ERR_INVALID_ARG;
    }
    ctx->n_rays = (long long)cams->n_cams * cams->width * cams->height;
    cudaGetDevice(&ctx->device);

    DevScene& d = ctx->ds;
    std::memset(&d, 0, sizeof(d));
    d.G = (int)G;
    d.halfG = 0.5f * (float)G;
    d.h = 2.0f / (float)G;
    d.S = sc->n_shells;
    for (int s = 0; s < sc->n_shells; ++s) d.R[s] = sc->shell_radii[s];
    d.He = ctx->scene.env_h;
    d.We = ctx->scene.env_w;
    d.env_kind = ctx->scene.env_kind;
    d.n_vox = G * G * G;
    set_layout(d, 0);
    d.shell_texels = texels;
    d.W = cams->width;
    d.H = cams->height;
    d.n_cams = cams->n_cams;
    d.n_rays = ctx->n_rays;
    d.tile_w = 8;
    d.tile_h = 4;
    d.tiles_x = (cams->width + d.tile_w - 1) / d.tile_w;
    d.tiles_y = (cams->height + d.tile_h - 1) / d.tile_h;
    d.n_tiles = (long long)d.tiles_x * d.tiles_y * cams->n_cams;
    if (ctx->n_rays == 0) d.n_tiles = 0;
    d.max_samples = opts->max_samples;
    d.jitter = opts->jitter;
    d.aux = opts->aux;
    d.aux_lambda = (float)opts->aux_lambda;
    d.seed = opts->seed;
    d.epoch = opts->epoch;

    if (cams->n_cams > 0) {
        float* host = new (std::nothrow) float[16 * (size_t)cams->n_cams];
        if (!host) { delete ctx; return PERF_ERR_INVALID_ARG; }
        std::memset(host, 0, sizeof(float) * 16 * (size_t)cams->n_cams);
        for (int c = 0; c < cams->n_cams; ++c) {
            if (cams->c2w) std::memcpy(host + 16 * c, cams->c2w + 12 * c, 12 * sizeof(float));
            host[16 * c + 12] = cams->focal ? cams->focal[c] : 1.0f;
        }
        cudaError_t e = cudaMalloc(&ctx->cams, sizeof(float) * 16 * (size_t)cams->n_cams);
        if (e == cudaSuccess)
            e = cudaMemcpy(ctx->cams, host, sizeof(float) * 16 * (size_t)cams->n_cams,
                           cudaMemcpyHostToDevice);
        delete[] host;
        if (e != cudaSuccess) { perf_destroy(ctx); return PERF_ERR_CUDA; }
    }
    d.cams = ctx->cams;
    cudaError_t e = cudaMalloc(&ctx->s, sizeof(PcgScalars));
    if (e == cudaSuccess) e = cudaMemset(ctx->s, 0, sizeof(PcgScalars));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->dF, sizeof(double) * 2);
    if (e == cudaSuccess) e = cudaEventCreate(&ctx->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&ctx->ev1);
    if (e != cudaSuccess) { perf_destroy(ctx); return PERF_ERR_CUDA; }
    *out = ctx;
    return PERF_OK;
}

perf_status perf_destroy(perf_ctx* ctx) {
    if (!ctx) return PERF_ERR_INVALID_ARG;
    void* bufs[] = {ctx->cams, ctx->r, ctx->diag, ctx->grad, ctx->delta, ctx->rho, ctx->p,
                    ctx->xp, ctx->Ap, ctx->tile_off, ctx->coef, ctx->keff, ctx->d_prefix, ctx->shell_tab, ctx->hist, ctx->cross, ctx->blocks_ws, ctx->feat, ctx->x_trial, ctx->x16, ctx->p16, ctx->t16, ctx->s, ctx->dF};
    for (void* b : bufs)
        if (b) cudaFree(b);
    if (ctx->ev0) cudaEventDestroy(ctx->ev0);
    if (ctx->ev1) cudaEventDestroy(ctx->ev1);
    if (ctx->pcg_graph) cudaGraphExecDestroy(ctx->pcg_graph);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    for (auto& t : ctx->kt)
        for (auto& pr : t.ev) {
            cudaEventDestroy(pr.first);
            cudaEventDestroy(pr.second);
        }
    delete ctx;
    return PERF_OK;
}

perf_status perf_set_options(perf_ctx* ctx, const perf_options* opts) {
    if (!ctx) return PERF_ERR_INVALID_ARG;
    std::string why;
    if (check_options(opts, why) != PERF_OK) return fail(ctx, PERF_ERR_INVALID_ARG, why);
    ctx->opts = *opts;
    ctx->ds.max_samples = opts->max_samples;
    ctx->ds.jitter = opts->jitter;
    ctx->shell_tab_epoch = -2;                 // rays may move: rebuild the shell hits
    ctx->ds.seed = opts->seed;
    ctx->ds.epoch = opts->epoch;
    if (ctx->ds.aux != opts->aux && ctx->r) {   // the residual buffer changes size
        cudaFree(ctx->r);
        ctx->r = nullptr;
    }
    ctx->ds.aux = opts->aux;
    ctx->ds.aux_lambda = (float)opts->aux_lambda;
    return PERF_OK;
}

int64_t perf_param_count(const perf_ctx* ctx) { return ctx ? (int64_t)ctx->n : -1; }
int64_t perf_ray_count(const perf_ctx* ctx) { return ctx ? (int64_t)ctx->n_rays : -1; }
const char* perf_last_error(const perf_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

perf_status perf_render(perf_ctx* ctx, const void* x, float* rgb_out, float* T_out, void* stream) {
    if (!ctx) return PERF_ERR_INVALID_ARG;
    if (ctx->n_rays == 0) return PERF_OK;
    if (bad_ptr(x) || bad_ptr(rgb_out)) return fail(ctx, PERF_ERR_INVALID_ARG, "render: NULL x or rgb_out");
    SHELLS(ctx, S(stream));
    CK(perf::launch_forward(ctx->ds, ctx->scene.dtype, x, nullptr, rgb_out, T_out, nullptr, 0, S(stream)));
    return PERF_OK;
}

perf_status perf_residual(perf_ctx* ctx, const void* x, const void* target, void* r_out,
                          double* F_out, void* stream) {
    if (!ctx) return PERF_ERR_INVALID_ARG;
    if (bad_ptr(F_out)) return fail(ctx, PERF_ERR_INVALID_ARG, "residual: NULL F_out");
    CK(cudaMemsetAsync(F_out, 0, sizeof(double), S(stream)));
    if (ctx->n_rays == 0) return PERF_OK;
    if (bad_ptr(x) || bad_ptr(target)) return fail(ctx, PERF_ERR_INVALID_ARG, "residual: NULL x or target");
    SHELLS(ctx, S(stream));
    CK(perf::launch_forward(ctx->ds, ctx->scene.dtype, x, target, r_out, nullptr, F_out,
                            r_out ? 1 : 2, S(stream)));
    return PERF_OK;
}

perf_status perf_jvp(perf_ctx* ctx, const void* x, const float* p, float* jp_out, void* stream) {
    if (!ctx) return PERF_ERR_INVALID_ARG;
    if (ctx->n_rays == 0) return PERF_OK;
    if (bad_ptr(x) || bad_ptr(p) || bad_ptr(jp_out)) return fail(ctx, PERF_ERR_INVALID_ARG, "jvp: NULL pointer");
    SHELLS(ctx, S(stream));
    CK(perf::launch_jvp(ctx->ds, ctx->scene.dtype, x, p, PERF_F32, jp_out, S(stream)));
    return PERF_OK;
}

perf_status perf_vjp(perf_ctx* ctx, const void* x, const float* v, float* out, int32_t accumulate,
                     void* stream) {
    if (!ctx) return PERF_ERR_INVALID_ARG;
    if (bad_ptr(out)) return fail(ctx, PERF_ERR_INVALID_ARG, "vjp: NULL out");
    if (!accumulate) CK(cudaMemsetAsync(out, 0, sizeof(float) * (size_t)ctx->n, S(stream)));
    if (ctx->n_rays == 0) return PERF_OK;
    if (bad_ptr(x) || bad_ptr(v)) return fail(ctx, PERF_ERR_INVALID_ARG, "vjp: NULL x or v");
    SHELLS(ctx, S(stream));
    CK(perf::launch_scatter(ctx->ds, ctx->scene.dtype, 0, x, nullptr, PERF_F32, v, out, nullptr,
                            nullptr, S(stream)));
    return PERF_OK;
}

perf_status perf_diag_jtj(perf_ctx* ctx, const void* x, const void* r, float* diag_out,
                          float* grad_out, void* stream) {
    if (!ctx) return PERF_ERR_INVALID_ARG;
    if (bad_ptr(diag_out)) return fail(ctx, PERF_ERR_INVALID_ARG, "diag_jtj: NULL diag_out");
    if ((r == nullptr) != (grad_out == nullptr))
        return fail(ctx, PERF_ERR_INVALID_ARG, "diag_jtj: give both r and grad_out or neither");
    CK(cudaMemsetAsync(diag_out, 0, sizeof(float) * (size_t)ctx->n, S(stream)));
    if (grad_out) CK(cudaMemsetAsync(grad_out, 0, sizeof(float) * (size_t)ctx->n, S(stream)));
    if (ctx->n_rays == 0) return PERF_OK;
    if (bad_ptr(x)) return fail(ctx, PERF_ERR_INVALID_ARG, "diag_jtj: NULL x");
    SHELLS(ctx, S(stream));
    CK(perf::launch_scatter(ctx->ds, ctx->scene.dtype, 2, x, nullptr, PERF_F32, r, diag_out,
                            grad_out, nullptr, S(stream)));
    return PERF_OK;
}

perf_status perf_apply_normal(perf_ctx* ctx, const void* x, const float* p, float* ap_out,
                              double* pap_out, void* stream) {
    if (!ctx) return PERF_ERR_INVALID_ARG;
    if (bad_ptr(ap_out)) return fail(ctx, PERF_ERR_INVALID_ARG, "apply_normal: NULL ap_out");
    CK(cudaMemsetAsync(ap_out, 0, sizeof(float) * (size_t)ctx->n, S(stream)));
    if (pap_out) CK(cudaMemsetAsync(pap_out, 0, sizeof(double), S(stream)));
    if (ctx->n_rays == 0) return PERF_OK;
    if (bad_ptr(x) || bad_ptr(p)) return fail(ctx, PERF_ERR_INVALID_ARG, "apply_normal: NULL x or p");
    SHELLS(ctx, S(stream));
    CK(perf::launch_scatter(ctx->ds, ctx->scene.dtype, 1, x, p, PERF_F32, nullptr, ap_out, nullptr,
                            pap_out, S(stream)));
    return PERF_OK;
}

perf_status perf_pcg_begin(perf_ctx* ctx, const float* grad, const float* diag, void* stream) {
    if (!ctx) return PERF_ERR_INVALID_ARG;
    if (bad_ptr(grad) || bad_ptr(diag)) return fail(ctx, PERF_ERR_INVALID_ARG, "pcg_begin: NULL grad or diag");
    perf_status st = ensure_pcg(ctx);
    if (st != PERF_OK) return st;
    // the iterations precondition with the context's copy of the diagonal
    if (diag != ctx->diag)
        CK(cudaMemcpyAsync(ctx->diag, diag, sizeof(float) * (size_t)ctx->n,
                           cudaMemcpyDeviceToDevice, S(stream)));
    const float* B = ctx->opts.precond == PERF_PRECOND_BLOCK4 ? ctx->blocks : nullptr;
    st = ensure_hist(ctx, ctx->opts.pcg_iters);
    if (st != PERF_OK) return st;
    CK(perf::launch_pcg_begin(ctx->n, grad, ctx->diag, ctx->delta, ctx->rho, ctx->p,
                              ctx->p16, ctx->Ap, ctx->s, ctx->opts.pcg_iters, ctx->opts.pcg_fixed,
                              ctx->opts.pcg_eps_rel, ctx->opts.pcg_stall, B, ctx->n_block,
                              S(stream), nullptr, ctx->hist, ctx->hist_cap));
    return PERF_OK;
}

perf_status perf_pcg_step(perf_ctx* ctx, const void* x, int32_t* done_out, void* stream);

}  // extern "C"

namespace {

// A p into the PCG workspace from separate x and p arrays (tiles of d).
cudaError_t apply_arrays(perf_ctx* ctx, const perf::DevScene& d, const void* x, const void* pp,
                         double* pap, cudaStream_t st) {
    const int pdt = ctx->scene.dtype == PERF_BF16 ? PERF_BF16 : PERF_F32;
    return perf::launch_scatter(d, ctx->scene.dtype, 1, x, pp, pdt, nullptr, ctx->Ap, nullptr, pap,
                                st);
}

// One Algorithm 2 iteration on the context workspace with diagonal `diag`
// and block preconditioner B (null: Jacobi).  paired: A p reads the paired
// records ctx->xp, whose x half holds x (FP32 scenes); coef: A p from the
// coefficient store of the current Gauss-Newton step.
// dsp (may be null: ctx->ds): the scene descriptor of the step, whose
// layout is the block order of the PCG vectors.
perf_status pcg_iter(perf_ctx* ctx, const void* x, const float* diag, const float* B, cudaStream_t st,
                     bool paired = false, bool coef = false, const perf::DevScene* dsp = nullptr) {
    const bool bf = ctx->scene.dtype == PERF_BF16;
    const void* pp = bf ? static_cast<const void*>(ctx->p16) : static_cast<const void*>(ctx->p);
    const perf::DevScene& d0 = dsp ? *dsp : ctx->ds;
    t_begin(ctx, PERF_T_APPLY, st);
    // the store's tiles from the coefficients, any remaining tiles recomputed
    perf::DevScene rest = d0;
    if (coef) {
        perf::DevScene head = d0;
        head.n_tiles = ctx->coef_tiles;
        CK(perf::launch_apply_coef(head, pp, bf ? PERF_BF16 : PERF_F32, ctx->coef, ctx->tile_off,
                                   ctx->Ap, &ctx->s->pAp, st));
        rest.tile_lo = ctx->coef_tiles;
    }
    if (rest.tile_lo < rest.n_tiles) {
        if (paired)
            CK(perf::launch_apply_pair(rest, ctx->xp, ctx->Ap, &ctx->s->pAp, st));
        else
            CK(apply_arrays(ctx, rest, x, pp, &ctx->s->pAp, st));
    }
    t_end(ctx, PERF_T_APPLY, st);
    t_begin(ctx, PERF_T_VECTOR, st);
    CK(perf::launch_pcg_update(ctx->n, ctx->delta, ctx->rho, ctx->p, ctx->Ap, diag, B, ctx->n_block,
                               ctx->s, st));
    CK(perf::launch_pcg_finish(ctx->s, st));
    CK(perf::launch_pcg_dir(ctx->n, ctx->rho, diag, B, ctx->n_block, ctx->p, ctx->p16, ctx->s, st,
                            paired ? ctx->xp : nullptr));
    t_end(ctx, PERF_T_VECTOR, st);
    return PERF_OK;
}

template <typename T>
void key_add(std::vector<unsigned char>& k, const T& v) {
    const unsigned char* b = reinterpret_cast<const unsigned char*>(&v);
    k.insert(k.end(), b, b + sizeof(T));
}

// iters fixed iterations of pcg_iter replayed from a CUDA graph on st
// (captured on the context's own stream; recaptured when its key changes).
perf_status pcg_graph_run(perf_ctx* ctx, const void* x, const float* B, bool paired, bool coef,
                          const perf::DevScene& d, int iters, cudaStream_t st) {
    std::vector<unsigned char> key;
    key_add(key, iters);
    key_add(key, paired);
    key_add(key, coef);
    key_add(key, x);
    key_add(key, B);
    key_add(key, ctx->n_block);
    key_add(key, d);
    const void* ptrs[] = {ctx->coef, ctx->tile_off, ctx->xp, ctx->p, ctx->p16, ctx->Ap,
                          ctx->delta, ctx->rho, ctx->diag, ctx->s};
    key_add(key, ptrs);
    key_add(key, ctx->coef_tiles);
    if (!ctx->pcg_graph || key != ctx->pcg_graph_key) {
        if (ctx->pcg_graph) {
            cudaGraphExecDestroy(ctx->pcg_graph);
            ctx->pcg_graph = nullptr;
        }
        if (!ctx->cap_stream) CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
        const unsigned long long n0 = perf_launch_count();
        CK(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
        perf_status ps = PERF_OK;
        for (int k = 0; k < iters && ps == PERF_OK; ++k)
            ps = pcg_iter(ctx, x, ctx->diag, B, ctx->cap_stream, paired, coef, &d);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &g);
        if (ps != PERF_OK || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return ps != PERF_OK ? ps : cuda_fail(ctx, e, "PCG graph capture");
        }
        const cudaError_t ei = cudaGraphInstantiate(&ctx->pcg_graph, g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) {
            ctx->pcg_graph = nullptr;
            return cuda_fail(ctx, ei, "PCG graph instantiate");
        }
        ctx->pcg_graph_key = key;
        ctx->pcg_graph_launches = perf_launch_count() - n0;
        perf::count_launch(0ull - ctx->pcg_graph_launches);   // counted when replayed
    }
    CK(cudaGraphLaunch(ctx->pcg_graph, st));
    perf::count_launch(ctx->pcg_graph_launches);
    return PERF_OK;
}

}  // namespace

extern "C" {

perf_status perf_pcg_step(perf_ctx* ctx, const void* x, int32_t* done_out, void* stream) {
    if (!ctx) return PERF_ERR_INVALID_ARG;
    if (bad_ptr(x)) return fail(ctx, PERF_ERR_INVALID_ARG, "pcg_step: NULL x");
    if (!ctx->delta || !ctx->s) return fail(ctx, PERF_ERR_INVALID_ARG, "pcg_step before pcg_begin");
    const float* B = ctx->opts.precond == PERF_PRECOND_BLOCK4 ? ctx->blocks : nullptr;
    SHELLS(ctx, S(stream));
    perf_status st = pcg_iter(ctx, x, ctx->diag, B, S(stream));
    if (st != PERF_OK) return st;
    if (done_out) {
        int done = 0;
        CK(cudaMemcpyAsync(&done, &ctx->s->done, sizeof(int), cudaMemcpyDeviceToHost, S(stream)));
        CK(cudaStreamSynchronize(S(stream)));
        *done_out = done;
    }
    return PERF_OK;
}

perf_status perf_pcg_result(perf_ctx* ctx, float* delta_out, perf_pcg_info* info, void* stream) {
    if (!ctx) return PERF_ERR_INVALID_ARG;
    if (!ctx->delta || !ctx->s) return fail(ctx, PERF_ERR_INVALID_ARG, "pcg_result before pcg_begin");
    if (delta_out)
        CK(cudaMemcpyAsync(delta_out, ctx->delta, sizeof(float) * (size_t)ctx->n,
                           cudaMemcpyDeviceToDevice, S(stream)));
    if (info) {
        PcgScalars h;
        CK(cudaMemcpyAsync(&h, ctx->s, sizeof(h), cudaMemcpyDeviceToHost, S(stream)));
        CK(cudaStreamSynchronize(S(stream)));
        info->iters = h.iter;
        info->exit_reason = h.exit_reason;
        info->R0 = h.R0;
        info->R = h.R;
        info->rz = h.rz;
    }
    return PERF_OK;
}

perf_status perf_gn_solve(perf_ctx* ctx, float* x, const void* target, int32_t n_steps,
                          perf_gn_stats* stats, void* stream) {
    if (!ctx) return PERF_ERR_INVALID_ARG;
    if (n_steps < 0) return fail(ctx, PERF_ERR_INVALID_ARG, "gn_solve: n_steps < 0");
    if (bad_ptr(x) || (ctx->n_rays > 0 && bad_ptr(target)))
        return fail(ctx, PERF_ERR_INVALID_ARG, "gn_solve: NULL x or target");
    cudaStream_t st = S(stream);
    const bool bf = ctx->scene.dtype == PERF_BF16;
    perf_status ps = ensure_pcg(ctx);
    if (ps != PERF_OK) return ps;
    const long long m = (3 + ctx->ds.aux) * ctx->n_rays;   // residuals per GN step
    if (!ctx->r) CK(cudaMalloc(&ctx->r, (bf ? 2 : 4) * (size_t)(m > 0 ? m : 1)));
    CK(alloc(&ctx->x_trial, ctx->n));
    if (bf) {
        CK(alloc(&ctx->x16, ctx->n));
        CK(alloc(&ctx->t16, ctx->n));
    }
    const perf_options& o = ctx->opts;
    const uint32_t epoch0 = o.epoch;
    perf_status result = PERF_OK;
    for (int step = 0; step < n_steps; ++step) {
        ctx->ds.epoch = epoch0 + (uint32_t)step;
        SHELLS(ctx, st);
        CK(cudaEventRecord(ctx->ev0, st));
        const void* xm = x;
        if (bf) {
            CK(perf::launch_to_bf16(ctx->n, x, ctx->x16, st));
            xm = ctx->x16;
        }
        // residuals and F(x)
        CK(cudaMemsetAsync(ctx->dF, 0, sizeof(double), st));
        t_begin(ctx, PERF_T_RESIDUAL, st);
        if (ctx->n_rays > 0)
            CK(perf::launch_forward(ctx->ds, ctx->scene.dtype, xm, target, ctx->r, nullptr, ctx->dF, 1, st));
        t_end(ctx, PERF_T_RESIDUAL, st);
        // b = -J^T r and M = diag(J^T J)
        CK(cudaMemsetAsync(ctx->diag, 0, sizeof(float) * (size_t)ctx->n, st));
        CK(cudaMemsetAsync(ctx->grad, 0, sizeof(float) * (size_t)ctx->n, st));
        const long long nvox = ctx->ds.n_vox;
        const bool blk = o.precond != PERF_PRECOND_JACOBI;
        const bool need_cross = o.precond == PERF_PRECOND_BLOCK_JACOBI ||
                                (o.precond == PERF_PRECOND_BLOCK4 && ctx->lpc);
        if (need_cross) {
            CK(alloc(&ctx->cross, 4 * nvox));
            CK(cudaMemsetAsync(ctx->cross, 0, sizeof(float) * 4 * (size_t)nvox, st));
        }
        bool use_coef = false;
        ps = ensure_coef(ctx, st, &use_coef);
        if (ps != PERF_OK) return ps;
        ctx->ds.coef_tiles = use_coef ? ctx->coef_tiles : 0;
        // the step's PCG vectors (and the diagonal, gradient and block
        // couplings the diagonal march writes) take the tuned brick order when
        // every A p of the step runs from the store and the preconditioner is
        // per voxel; the learned network and caller-given blocks read the
        // canonical order
        perf::DevScene dl = ctx->ds;
        perf::set_layout(dl, (use_coef && ctx->coef_tiles >= ctx->ds.n_tiles &&
                              o.precond != PERF_PRECOND_BLOCK4) ? ctx->brick_s : 0);
        dl.keff = use_coef ? ctx->keff : nullptr;
        const int4 lay = perf::layout_of(dl);
        t_begin(ctx, PERF_T_DIAG, st);
        if (ctx->n_rays > 0)
            CK(perf::launch_scatter(dl, ctx->scene.dtype, 2, xm, nullptr, PERF_F32, ctx->r,
                                    ctx->diag, ctx->grad, nullptr, st,
                                    need_cross ? ctx->cross : nullptr,
                                    use_coef ? ctx->coef : nullptr,
                                    use_coef ? ctx->tile_off : nullptr));
        t_end(ctx, PERF_T_DIAG, st);
        ctx->coef_used = use_coef;
        ctx->keff_valid = dl.keff != nullptr;
        ctx->keff_tiles = ctx->coef_tiles;
        ctx->keff_tile_w = ctx->ds.tile_w;
        ctx->keff_epoch = ctx->ds.epoch;
        const float* B = nullptr;
        long long nB = 0;
        if (o.precond == PERF_PRECOND_BLOCK_JACOBI ||
            (o.precond == PERF_PRECOND_BLOCK4 && ctx->lpc)) {
            CK(alloc(&ctx->blocks_ws, 16 * nvox));
            t_begin(ctx, PERF_T_PRECOND, st);
            if (o.precond == PERF_PRECOND_BLOCK_JACOBI) {
                CK(perf::launch_block_jacobi(ctx->diag, ctx->cross, ctx->blocks_ws, nvox, st));
            } else {
                CK(alloc(&ctx->feat, 16 * nvox));
                CK(perf::lpc_blocks_for(ctx->lpc, ctx->ds.G, x, ctx->grad, ctx->diag, ctx->cross,
                                        ctx->feat, ctx->blocks_ws, st));
            }
            t_end(ctx, PERF_T_PRECOND, st);
            B = ctx->blocks_ws;
            nB = nvox;
        } else if (o.precond == PERF_PRECOND_BLOCK4) {
            B = ctx->blocks;
            nB = ctx->n_block;
        }
        int fallback = 0;
        const bool paired = !bf && ctx->pair && (!use_coef || ctx->coef_tiles < ctx->ds.n_tiles);
        if (paired) CK(perf::launch_pair_pack(ctx->n, x, nullptr, ctx->xp, st));
        double F0 = 0.0;
        CK(cudaMemcpyAsync(&F0, ctx->dF, sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        double g_star = 1.0, mu_star = 0.0;
        int evals = 0;
        bool accept = false;
        for (int pass = 0; pass < 2; ++pass) {
            for (int attempt = 0; attempt < 2; ++attempt) {
                ps = ensure_hist(ctx, o.pcg_iters);
                if (ps != PERF_OK) return ps;
                CK(perf::launch_pcg_begin(ctx->n, ctx->grad, ctx->diag, ctx->delta, ctx->rho, ctx->p,
                                          ctx->p16, ctx->Ap, ctx->s, o.pcg_iters, o.pcg_fixed,
                                          o.pcg_eps_rel, o.pcg_stall, B, nB, st,
                                          paired ? ctx->xp : nullptr, ctx->hist, ctx->hist_cap));
                if (o.pcg_fixed && ctx->pcg_graph_on && !ctx->timing && o.pcg_iters > 1) {
                    // one graph for the whole loop (no per-kernel launch work on the host)
                    ps = pcg_graph_run(ctx, xm, B, paired, use_coef, dl, o.pcg_iters, st);
                    if (ps != PERF_OK) return ps;
                } else {
                    for (int k = 0; k < o.pcg_iters; ++k) {
                        ps = pcg_iter(ctx, xm, ctx->diag, B, st, paired, use_coef, &dl);
                        if (ps != PERF_OK) return ps;
                        if (!o.pcg_fixed) {
                            int done = 0;
                            CK(cudaMemcpyAsync(&done, &ctx->s->done, sizeof(int), cudaMemcpyDeviceToHost, st));
                            CK(cudaStreamSynchronize(st));
                            if (done) break;
                        }
                    }
                }
                if (!(o.precond == PERF_PRECOND_BLOCK4 && blk) || B == nullptr) break;
                // the true residual (PERF_JUDGE_RESIDUAL) judges the learned
                // preconditioner, or only its breakdowns do and the line search
                // below judges the step (PERF_JUDGE_OBJECTIVE); Jacobi is the fallback
                PcgScalars hj;
                CK(cudaMemcpyAsync(&hj, ctx->s, sizeof(hj), cudaMemcpyDeviceToHost, st));
                CK(cudaStreamSynchronize(st));
                // a convolution of the network whose bounded wait ran out left the
                // blocks incomplete: that step's PCG is rerun with Jacobi
                const bool conv_ok = !(o.precond == PERF_PRECOND_BLOCK4 && ctx->lpc) ||
                                     perf::lpc_conv_error() == 0;
                const bool residual_ok = o.precond_judge == PERF_JUDGE_OBJECTIVE || hj.R < hj.R0;
                if (conv_ok && std::isfinite(hj.R) && residual_ok && hj.exit_reason != 3 &&
                    hj.exit_reason != 4)
                    break;
                B = nullptr;
                nB = 0;
                fallback = 1;
            }
            // Algorithm 3 on F(P(x + gamma Delta))
            double gamma = 1.0, mu_prev = 3.4028234663852886e38;
            g_star = 1.0;
            mu_star = mu_prev;
            bool found = false;
            for (int it = 0; it <= o.ls_max; ++it) {
                CK(perf::launch_trial(ctx->n, x, ctx->delta, gamma, o.project, ctx->x_trial,
                                      bf ? ctx->t16 : nullptr, st, lay));
                CK(cudaMemsetAsync(ctx->dF, 0, sizeof(double), st));
                t_begin(ctx, PERF_T_FORWARD, st);
                if (ctx->n_rays > 0)
                    CK(perf::launch_forward(ctx->ds, ctx->scene.dtype,
                                            bf ? static_cast<const void*>(ctx->t16)
                                               : static_cast<const void*>(ctx->x_trial),
                                            target, nullptr, nullptr, ctx->dF, 2, st));
                t_end(ctx, PERF_T_FORWARD, st);
                double mu = 0.0;
                CK(cudaMemcpyAsync(&mu, ctx->dF, sizeof(double), cudaMemcpyDeviceToHost, st));
                CK(cudaStreamSynchronize(st));
                ++evals;
                if (std::isnan(mu)) mu = INFINITY;
                if (mu > mu_prev) {
                    g_star = gamma / o.ls_alpha;
                    mu_star = mu_prev;
                    found = true;
                    break;
                }
                gamma *= o.ls_alpha;
                mu_prev = mu;
            }
            if (!found) { g_star = gamma / o.ls_alpha; mu_star = mu_prev; }
            accept = std::isfinite(mu_star) && mu_star < F0;
            // a block preconditioner's step that the line search cannot use
            // (no trial point lowers F) is redone with Jacobi PCG
            if (accept || B == nullptr || pass == 1) break;
            B = nullptr;
            nB = 0;
            fallback = 1;
        }
        if (accept) {
            CK(perf::launch_trial(ctx->n, x, ctx->delta, g_star, o.project, ctx->x_trial,
                                  nullptr, st, lay));
            CK(cudaMemcpyAsync(x, ctx->x_trial, sizeof(float) * (size_t)ctx->n,
                               cudaMemcpyDeviceToDevice, st));
        }
        CK(cudaEventRecord(ctx->ev1, st));
        PcgScalars h;
        CK(cudaMemcpyAsync(&h, ctx->s, sizeof(h), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        t_harvest(ctx);
        if (!std::isfinite(F0)) result = PERF_ERR_NONFINITE;
        if (stats) {
            perf_gn_stats& g = stats[step];
            g.F_before = F0;
            g.F_after = accept ? mu_star : F0;
            g.gamma = g_star;
            g.accepted = accept ? 1 : 0;
            g.ls_evals = evals;
            g.pcg.iters = h.iter;
            g.pcg.exit_reason = h.exit_reason;
            g.pcg.R0 = h.R0;
            g.pcg.R = h.R;
            g.pcg.rz = h.rz;
            g.precond_fallback = fallback;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
            g.ms = ms;
        }
        if (result != PERF_OK) break;
    }
    ctx->ds.epoch = epoch0;
    if (result == PERF_ERR_NONFINITE) return fail(ctx, result, "gn_solve: non-finite objective");
    return result;
}

perf_status perf_enable_timing(perf_ctx* ctx, int32_t on) {
    if (!ctx) return PERF_ERR_INVALID_ARG;
    ctx->timing = on != 0;
    return PERF_OK;
}

// Re-tile the context's rays for tile width tw (tile height 32 / tw).
static void set_tiling(perf_ctx* ctx, int tw) {
    DevScene& d = ctx->ds;
    d.tile_w = tw;
    d.tile_h = 32 / tw;
    d.tiles_x = (d.W + d.tile_w - 1) / d.tile_w;
    d.tiles_y = (d.H + d.tile_h - 1) / d.tile_h;
    d.n_tiles = ctx->n_rays > 0 ? (long long)d.tiles_x * d.tiles_y * d.n_cams : 0;
}

static perf_status autotune_impl(perf_ctx* ctx, const void* x, const void* p, perf_tuning* out,
                                 void* stream) {
    cudaStream_t st = S(stream);
    ctx->keff_valid = false;   // the tuner's store fills overwrite the prefix lengths
    perf_status ps = ensure_pcg(ctx);
    if (ps != PERF_OK) return ps;
    SHELLS(ctx, st);
    const bool bf = ctx->scene.dtype == PERF_BF16;
    // the probe direction (default x: every ray then has a non-zero J p)
    void* pbuf = bf ? static_cast<void*>(ctx->p16) : static_cast<void*>(ctx->p);
    CK(cudaMemcpyAsync(pbuf, p ? p : x, (bf ? 2 : 4) * (size_t)ctx->n, cudaMemcpyDeviceToDevice, st));
    const void* pp = pbuf;
    if (!bf) CK(perf::launch_pair_pack(ctx->n, static_cast<const float*>(x), ctx->p, ctx->xp, st));
    auto apply = [&](bool paired) -> cudaError_t {
        return paired ? perf::launch_apply_pair(ctx->ds, ctx->xp, ctx->Ap, nullptr, st)
                      : apply_arrays(ctx, ctx->ds, x, pp, nullptr, st);
    };
    const int tws[4] = {8, 4, 16, 32};
    const int caps[3] = {0, 3, 2};
    // events live until every return path has left (scope guard)
    struct Events {
        cudaEvent_t a = nullptr, b = nullptr;
        ~Events() {
            if (a) cudaEventDestroy(a);
            if (b) cudaEventDestroy(b);
        }
    } ev;
    CK(cudaEventCreate(&ev.a));
    CK(cudaEventCreate(&ev.b));
    cudaEvent_t e0 = ev.a, e1 = ev.b;
    // With the coefficient store, Gauss-Newton steps run the coefficient-
    // cached A p: for every tile shape the store is laid out anew and filled
    // at x, and the A p from it is timed over the CTA caps; the default
    // (8x4, no cap, timed first) is kept unless beaten by 3%.
    set_tiling(ctx, 8);
    bool use_coef = false;
    perf_status pc = ensure_coef(ctx, st, &use_coef);
    if (pc != PERF_OK) return pc;
    if (use_coef && ctx->coef_tiles == ctx->ds.n_tiles) {
        float best = 1e30f, incumbent = 1e30f;
        int best_tw = 8, best_cap = 0, best_s = 0;
        auto time_coef = [&](const perf::DevScene& d, float& ms) -> cudaError_t {
            cudaError_t e = cudaSuccess;
            for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
                if (rep == 1) e = cudaEventRecord(e0, st);
                if (e == cudaSuccess)
                    e = perf::launch_apply_coef(d, pp, bf ? PERF_BF16 : PERF_F32, ctx->coef,
                                                ctx->tile_off, ctx->Ap, nullptr, st);
            }
            if (e == cudaSuccess) e = cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            ms *= 0.5f;
            return e;
        };
        for (int i = 0; i < 4; ++i) {
            set_tiling(ctx, tws[i]);
            bool fits = false;
            pc = ensure_coef(ctx, st, &fits);
            if (pc != PERF_OK) return pc;
            if (!fits || ctx->coef_tiles < ctx->ds.n_tiles) continue;
            ctx->ds.coef_tiles = ctx->coef_tiles;
            // filled and timed as a Gauss-Newton step runs it (zero row tails skipped)
            perf::DevScene dk = ctx->ds;
            dk.keff = ctx->keff;
            CK(perf::launch_scatter(dk, ctx->scene.dtype, 2, x, nullptr, PERF_F32, nullptr,
                                    ctx->diag, nullptr, nullptr, st, nullptr, ctx->coef,
                                    ctx->tile_off));
            float tile_best = 1e30f;
            int tile_cap = 0;
            for (int j = 0; j < 3; ++j) {
                ctx->ds.cap_per_sm = caps[j];
                dk.cap_per_sm = caps[j];
                float ms = 0.f;
                CK(time_coef(dk, ms));
                if (i == 0 && j == 0) incumbent = ms;
                if (ms < tile_best) { tile_best = ms; tile_cap = caps[j]; }
                if (ms < best) { best = ms; best_tw = tws[i]; best_cap = caps[j]; best_s = 0; }
            }
            // the brick orders of the PCG vectors (4^3 and 8^3 voxels), at
            // this tile shape's best CTA cap
            for (int ls = 2; ls <= 3; ++ls) {
                perf::DevScene dl = dk;
                dl.cap_per_sm = tile_cap;
                if (!perf::set_layout(dl, ls)) continue;
                float ms = 0.f;
                CK(time_coef(dl, ms));
                if (ms < best) { best = ms; best_tw = tws[i]; best_cap = tile_cap; best_s = ls; }
            }
        }
        if (!(best < 0.97f * incumbent)) { best = incumbent; best_tw = 8; best_cap = 0; best_s = 0; }
        set_tiling(ctx, best_tw);
        ctx->ds.cap_per_sm = best_cap;
        ctx->brick_s = best_s;
        ctx->coef_used = true;
        if (out) {
            out->tile_w = best_tw;
            out->tile_h = 32 / best_tw;
            out->ctas_per_sm = best_cap;
            out->apply_ms = best;
            out->paired = 0;
            out->coef = 1;
            out->brick = 1 << best_s;
        }
        return PERF_OK;
    }
    // each candidate: one warm-up launch, then the mean of two timed launches
    auto time_apply = [&](bool paired, float& ms) -> cudaError_t {
        cudaError_t e = cudaSuccess;
        for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
            if (rep == 1) e = cudaEventRecord(e0, st);
            if (e == cudaSuccess) e = apply(paired);
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        ms *= 0.5f;
        return e;
    };
    // tile shape and CTA cap with the default layout (paired for FP32); the
    // default (8x4, no cap, timed first) is kept unless beaten by 3%
    const bool pair0 = !bf;
    float best = 1e30f, incumbent = 1e30f;
    int best_tw = 8, best_cap = 0;
    for (int i = 0; i < 4; ++i) {
        set_tiling(ctx, tws[i]);
        for (int j = 0; j < 3; ++j) {
            ctx->ds.cap_per_sm = caps[j];
            float ms = 0.f;
            CK(time_apply(pair0, ms));
            if (i == 0 && j == 0) incumbent = ms;
            if (ms < best) { best = ms; best_tw = tws[i]; best_cap = caps[j]; }
        }
    }
    if (!(best < 0.97f * incumbent)) { best = incumbent; best_tw = 8; best_cap = 0; }
    set_tiling(ctx, best_tw);
    ctx->ds.cap_per_sm = best_cap;
    // then the layout: separate x and p arrays replace the paired records
    // only when 3% faster
    bool pair = pair0;
    if (!bf) {
        float ms = 0.f;
        CK(time_apply(false, ms));
        if (ms < 0.97f * best) { best = ms; pair = false; }
    }
    ctx->pair = pair;
    ctx->brick_s = 0;   // the recomputing A p runs in the canonical order
    if (out) {
        out->tile_w = best_tw;
        out->tile_h = 32 / best_tw;
        out->ctas_per_sm = best_cap;
        out->apply_ms = best;
        out->paired = pair ? 1 : 0;
        out->coef = 0;
        out->brick = 1;
    }
    return PERF_OK;
}

perf_status perf_autotune(perf_ctx* ctx, const void* x, const void* p, perf_tuning* out,
                          void* stream) {
    if (!ctx || !x) return PERF_ERR_INVALID_ARG;
    // time the kernels the solver runs: the atomic-counting instantiation is
    // several times slower and would skew the choice
    unsigned long long* counter = ctx->ds.red_count;
    ctx->ds.red_count = nullptr;
    // a failed tuning run leaves the tiling, CTA cap and layout it started with
    const int tw0 = ctx->ds.tile_w, cap0 = ctx->ds.cap_per_sm, s0 = ctx->brick_s;
    const bool pair0 = ctx->pair;
    const perf_status ps = autotune_impl(ctx, x, p, out, stream);
    ctx->ds.red_count = counter;
    if (ps != PERF_OK) {
        set_tiling(ctx, tw0);
        ctx->ds.cap_per_sm = cap0;
        ctx->pair = pair0;
        ctx->brick_s = s0;
    }
    return ps;
}

perf_status perf_pcg_set_blocks(perf_ctx* ctx, const float* blocks, int64_t n_block) {
    if (!ctx) return PERF_ERR_INVALID_ARG;
    if (n_block < 0 || n_block > ctx->ds.n_vox || (n_block > 0 && !blocks))
        return fail(ctx, PERF_ERR_INVALID_ARG, "pcg_set_blocks: 0 <= n_block <= G^3 blocks required");
    ctx->blocks = blocks;
    ctx->n_block = n_block;
    return PERF_OK;
}

perf_status perf_set_lpc(perf_ctx* ctx, perf_lpc* lpc) {
    if (!ctx) return PERF_ERR_INVALID_ARG;
    ctx->lpc = lpc;
    return PERF_OK;
}

perf_status perf_diag_cross(perf_ctx* ctx, const void* x, float* diag_out, float* cross_out,
                            void* stream) {
    if (!ctx) return PERF_ERR_INVALID_ARG;
    if (bad_ptr(diag_out) || bad_ptr(cross_out))
        return fail(ctx, PERF_ERR_INVALID_ARG, "diag_cross: NULL output");
    CK(cudaMemsetAsync(diag_out, 0, sizeof(float) * (size_t)ctx->n, S(stream)));
    CK(cudaMemsetAsync(cross_out, 0, sizeof(float) * 4 * (size_t)ctx->ds.n_vox, S(stream)));
    if (ctx->n_rays == 0) return PERF_OK;
    if (bad_ptr(x)) return fail(ctx, PERF_ERR_INVALID_ARG, "diag_cross: NULL x");
    SHELLS(ctx, S(stream));
    CK(perf::launch_scatter(ctx->ds, ctx->scene.dtype, 2, x, nullptr, PERF_F32, nullptr, diag_out,
                            nullptr, nullptr, S(stream), cross_out));
    return PERF_OK;
}

perf_status perf_adam_step(perf_ctx* ctx, float* x, const void* target, float* m, float* v,
                           int32_t t, float lr, float beta1, float beta2, float eps,
                           double* F_out, void* stream) {
    if (!ctx) return PERF_ERR_INVALID_ARG;
    if (bad_ptr(x) || bad_ptr(m) || bad_ptr(v) || (ctx->n_rays > 0 && bad_ptr(target)))
        return fail(ctx, PERF_ERR_INVALID_ARG, "adam_step: NULL pointer");
    if (ctx->scene.dtype != PERF_F32 || ctx->ds.aux)
        return fail(ctx, PERF_ERR_UNSUPPORTED, "adam_step: FP32 scenes without the auxiliary term");
    if (t < 1 || !(lr > 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f) ||
        !(eps > 0.0f))
        return fail(ctx, PERF_ERR_INVALID_ARG, "adam_step: t >= 1, lr > 0, 0 <= beta < 1, eps > 0");
    cudaStream_t st = S(stream);
    perf_status ps = ensure_pcg(ctx);
    if (ps != PERF_OK) return ps;
    if (!ctx->r) CK(cudaMalloc(&ctx->r, 4 * (size_t)(ctx->n_rays > 0 ? 3 * ctx->n_rays : 1)));
    CK(cudaMemsetAsync(ctx->dF, 0, sizeof(double), st));
    CK(cudaMemsetAsync(ctx->grad, 0, sizeof(float) * (size_t)ctx->n, st));
    if (ctx->n_rays > 0) {
        SHELLS(ctx, st);
        // r = H^ - C and F, then g = J^T r (Section "Update step": the gradient)
        CK(perf::launch_forward(ctx->ds, PERF_F32, x, target, ctx->r, nullptr, ctx->dF, 1, st));
        CK(perf::launch_scatter(ctx->ds, PERF_F32, 0, x, nullptr, PERF_F32, ctx->r, ctx->grad,
                                nullptr, nullptr, st));
    }
    const float c1 = 1.0f - std::pow(beta1, (float)t), c2 = 1.0f - std::pow(beta2, (float)t);
    CK(perf::launch_adam(ctx->n, x, ctx->grad, m, v, beta1, beta2, lr, eps, c1, c2,
                         ctx->opts.project, st));
    if (F_out) CK(cudaMemcpyAsync(F_out, ctx->dF, sizeof(double), cudaMemcpyDeviceToDevice, st));
    return PERF_OK;
}

perf_status perf_pcg_history(perf_ctx* ctx, double* R_out, int32_t cap, int32_t* count_out) {
    if (!ctx || (cap > 0 && !R_out) || !count_out) return PERF_ERR_INVALID_ARG;
    *count_out = 0;
    if (!ctx->s || !ctx->hist) return PERF_OK;
    PcgScalars h;
    CK(cudaMemcpy(&h, ctx->s, sizeof(h), cudaMemcpyDeviceToHost));
    const long long k = std::min<long long>(std::min<long long>(h.iter, ctx->hist_cap), cap);
    if (k > 0) CK(cudaMemcpy(R_out, ctx->hist, sizeof(double) * (size_t)k, cudaMemcpyDeviceToHost));
    *count_out = (int32_t)k;
    return PERF_OK;
}

perf_status perf_set_pcg_graph(perf_ctx* ctx, int32_t on) {
    if (!ctx) return PERF_ERR_INVALID_ARG;
    ctx->pcg_graph_on = on != 0;
    return PERF_OK;
}

perf_status perf_set_brick(perf_ctx* ctx, int32_t edge) {
    if (!ctx) return PERF_ERR_INVALID_ARG;
    int s = 0;
    while (s < 4 && (1 << s) < edge) ++s;
    perf::DevScene d = ctx->ds;
    if (edge < 1 || (1 << s) != edge || s > 3 || !perf::set_layout(d, s))
        return fail(ctx, PERF_ERR_INVALID_ARG, "set_brick: edge 1, 2, 4 or 8 dividing G required");
    ctx->brick_s = s;
    return PERF_OK;
}

perf_status perf_set_coef_budget(perf_ctx* ctx, int64_t bytes) {
    if (!ctx) return PERF_ERR_INVALID_ARG;
    if (bytes < -1) return fail(ctx, PERF_ERR_INVALID_ARG, "set_coef_budget: bytes must be >= -1");
    ctx->coef_budget = bytes;
    if (bytes >= 0 && ctx->coef && ctx->coef_bytes > (size_t)bytes) {
        cudaFree(ctx->coef);
        ctx->coef = nullptr;
        ctx->coef_bytes = 0;
    }
    return PERF_OK;
}

perf_status perf_coef_info(perf_ctx* ctx, int64_t* bytes_held, int32_t* last_used,
                           double* coverage) {
    if (!ctx) return PERF_ERR_INVALID_ARG;
    if (bytes_held) *bytes_held = (int64_t)ctx->coef_bytes;
    if (last_used) *last_used = ctx->coef_used ? 1 : 0;
    if (coverage)
        *coverage = ctx->coef_used && ctx->ds.n_tiles > 0
                        ? (double)ctx->coef_tiles / (double)ctx->ds.n_tiles : 0.0;
    return PERF_OK;
}

perf_status perf_coef_prefix(perf_ctx* ctx, int64_t* rows_read, int64_t* rows_total,
                             void* stream) {
    if (!ctx) return PERF_ERR_INVALID_ARG;
    if (!rows_read || !rows_total) return fail(ctx, PERF_ERR_INVALID_ARG, "coef_prefix: NULL output");
    if (!ctx->keff_valid || !ctx->keff || ctx->keff_tile_w != ctx->ds.tile_w)
        return fail(ctx, PERF_ERR_INVALID_ARG, "coef_prefix: the last Gauss-Newton step did not fill the store");
    if (!ctx->d_prefix) CK(cudaMalloc(&ctx->d_prefix, 2 * sizeof(unsigned long long)));
    cudaStream_t st = S(stream);
    perf::DevScene d = ctx->ds;
    d.n_tiles = ctx->keff_tiles;
    d.tile_lo = 0;
    d.epoch = ctx->keff_epoch;
    unsigned long long h[2] = {0ull, 0ull};
    CK(cudaMemsetAsync(ctx->d_prefix, 0, sizeof(h), st));
    CK(perf::launch_coef_prefix(d, ctx->keff, ctx->d_prefix, st));
    CK(cudaMemcpyAsync(h, ctx->d_prefix, sizeof(h), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    *rows_read = (int64_t)h[0];
    *rows_total = (int64_t)h[1];
    return PERF_OK;
}

uint64_t perf_launch_count(void) { return (uint64_t)__atomic_load_n(&perf::g_launches, __ATOMIC_RELAXED); }

perf_status perf_set_atomic_counter(perf_ctx* ctx, uint64_t* device_counter) {
    if (!ctx) return PERF_ERR_INVALID_ARG;
    ctx->ds.red_count = reinterpret_cast<unsigned long long*>(device_counter);
    return PERF_OK;
}

perf_status perf_render_threshold(perf_ctx* ctx, const void* x, float min_opacity,
                                  float* rgb_out, float* T_out, void* stream) {
    if (!ctx) return PERF_ERR_INVALID_ARG;
    if (!(min_opacity >= 0.0f && min_opacity <= 1.0f))
        return fail(ctx, PERF_ERR_INVALID_ARG, "render_threshold: min_opacity outside [0, 1]");
    if (ctx->n_rays == 0) return PERF_OK;
    if (bad_ptr(x) || bad_ptr(rgb_out)) return fail(ctx, PERF_ERR_INVALID_ARG, "render_threshold: NULL x or rgb_out");
    SHELLS(ctx, S(stream));
    CK(perf::launch_forward(ctx->ds, ctx->scene.dtype, x, nullptr, rgb_out, T_out, nullptr, 0,
                            S(stream), min_opacity));
    return PERF_OK;
}

perf_status perf_upsample(const float* x, int32_t G, int32_t n_shells, int32_t env_h,
                          int32_t env_w, int32_t env_kind, float* x_out, void* stream) {
    if (!x || !x_out || G < 2 || G > 512 || n_shells < 0 || n_shells > PERF_MAX_SHELLS ||
        (n_shells > 0 && (env_h < 2 || env_w < 2 || env_h > (1 << 14) || env_w > (1 << 14))))
        return PERF_ERR_INVALID_ARG;
    if ((env_kind != PERF_ENV_EQUIRECT && env_kind != PERF_ENV_CUBE) ||
        (env_kind == PERF_ENV_CUBE && n_shells > 0 && env_w != 6 * env_h))
        return PERF_ERR_INVALID_ARG;
    const long long G2 = 2ll * G;
    const long long blocks = G2 * G2 * G2 + (long long)n_shells * 4 * env_h * env_w;
    if (blocks >= (1ll << 31)) return PERF_ERR_INVALID_ARG;
    const long long n_in = 4 * ((long long)G * G * G + (long long)n_shells * env_h * env_w);
    const char* a = reinterpret_cast<const char*>(x);
    const char* b = reinterpret_cast<const char*>(x_out);
    if (a < b + 16 * blocks && b < a + 4 * n_in) return PERF_ERR_INVALID_ARG;   // overlap
    cudaError_t e = perf::launch_upsample(x, G, n_shells, n_shells ? env_h : 0,
                                          n_shells ? env_w : 0, env_kind == PERF_ENV_CUBE ? 1 : 0,
                                          x_out, S(stream));
    return e == cudaSuccess ? PERF_OK : PERF_ERR_CUDA;
}

perf_status perf_sample_count(perf_ctx* ctx, uint64_t* out, void* stream) {
    if (!ctx || !out) return PERF_ERR_INVALID_ARG;
    *out = 0;
    if (ctx->n_rays == 0) return PERF_OK;
    unsigned long long* d = reinterpret_cast<unsigned long long*>(ctx->dF + 1);
    CK(perf::launch_count_samples(ctx->ds, d, S(stream)));
    unsigned long long h = 0;
    CK(cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, S(stream)));
    CK(cudaStreamSynchronize(S(stream)));
    *out = (uint64_t)h;
    return PERF_OK;
}

perf_status perf_get_timing(perf_ctx* ctx, perf_timing* out, int32_t reset) {
    if (!ctx || !out) return PERF_ERR_INVALID_ARG;
    t_harvest(ctx);
    for (int k = 0; k < PERF_T_COUNT; ++k) {
        out->ms[k] = ctx->kt[k].ms;
        out->launches[k] = ctx->kt[k].launches;
        if (reset) {
            ctx->kt[k].ms = 0.0;
            ctx->kt[k].launches = 0;
        }
    }
    return PERF_OK;
}

}  // extern "C"

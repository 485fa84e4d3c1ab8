// perf_batch.cu -- many independent scenes solved together (C ABI in perf.h).
//
// All scenes' parameters, rays and residuals are concatenated; every ray
// march is ONE persistent launch whose warps take (scene, pixel tile) items
// from a work queue, so uneven scenes load-balance across the GPU.  Each
// scene keeps its own Algorithm 2 scalars (segmented vector kernels) and its
// own Algorithm 3 step length.  The fixed-iteration PCG loop is captured once
// as a CUDA graph and replayed every Gauss-Newton step.  An autotuner times
// the A p launch over ray-tile shapes (4x8, 8x4, 16x2, 32x1 pixels per warp)
// and resident-CTA caps and keeps the fastest.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/perf.h"
#include "perf_kernels.h"

using perf::BatchItem;
using perf::DevScene;
using perf::PcgScalars;

struct perf_batch {
    int n = 0;
    perf_options opts;
    std::vector<BatchItem> items;      // host copy
    std::vector<long long> seg_h;      // parameter-block offsets (n + 1)
    long long n_params = 0, n_rays = 0, total_tiles = 0, max_seg = 0;
    int4* d_chunks = nullptr;          // per CTA of the vector kernels: (scene, first, end block)
    long long n_chunks = 0;
    std::vector<long long> ray_off;    // n + 1
    BatchItem* d_items = nullptr;
    float4* shell_tab = nullptr;       // shell hits of every scene's rays (FP64 texel coordinates)
    long long* d_start = nullptr;      // tile offsets (n + 1)
    long long* d_seg = nullptr;        // block offsets (n + 1)
    float* cams = nullptr;
    unsigned long long* counter = nullptr;
    // workspace
    float* x_work = nullptr;
    float* x_trial = nullptr;
    float* r = nullptr;
    float* diag = nullptr;
    float* grad = nullptr;
    float* delta = nullptr;     // Algorithm 2 vectors (FP32; p is also gathered by A p)
    float* rho = nullptr;
    float* p = nullptr;
    float* Ap = nullptr;
    PcgScalars* s = nullptr;
    double* F = nullptr;
    double* gamma = nullptr;
    int* mask = nullptr;
    // tuning and graph
    int tile_w = 8;
    int cap = 0;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    int graph_iters = -1;
    const float* graph_coef = nullptr;   // store the captured loop reads (null: recompute)
    // coefficient-cached A p (as for a single scene), rows over the global tile list
    long long coef_budget = -1;
    long long* tile_off = nullptr;
    float* coef = nullptr;
    size_t coef_bytes = 0;
    int* keff = nullptr;                 // per ray: its non-zero row prefix (DevScene::keff)
    long long coef_rows = 0;
    int tab_tile_w = 0;
    bool use_coef = false;               // the PCG loop reads the store
    // brick order of the PCG vectors (LayoutKey shift, per scene where G
    // allows it), used by steps whose A p runs from the store
    int brick_s = 0;
    int lay_applied = 0;                 // shift the items carry now
    bool any_brick = false;              // some scene's vectors are bricked
    int4* d_lay = nullptr;               // per scene (G, s, ys, zs) for the trial kernel
    std::string err;
};

namespace {

template <typename T>
cudaError_t dalloc(T** p, long long count) {
    return cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * (size_t)(count > 0 ? count : 1));
}

#define BK(call)                                                                  \
    do {                                                                          \
        cudaError_t e_ = (call);                                                  \
        if (e_ != cudaSuccess) {                                                  \
            b->err = std::string(#call) + ": " + cudaGetErrorString(e_);          \
            return PERF_ERR_CUDA;                                                 \
        }                                                                         \
    } while (0)

inline cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Two CUDA events destroyed on every return path.
struct EventPair {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ~EventPair() {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    }
};

// Re-tile every scene for tile width tw and upload items and tile offsets.
perf_status apply_tiling(perf_batch* b, int tw) {
    b->tile_w = tw;
    std::vector<long long> start(b->n + 1, 0);
    long long t = 0;
    for (int i = 0; i < b->n; ++i) {
        DevScene& d = b->items[i].sc;
        d.tile_w = tw;
        d.tile_h = 32 / tw;
        d.tiles_x = (d.W + d.tile_w - 1) / d.tile_w;
        d.tiles_y = (d.H + d.tile_h - 1) / d.tile_h;
        d.n_tiles = d.n_rays > 0 ? (long long)d.tiles_x * d.tiles_y * d.n_cams : 0;
        b->items[i].tile_off = t;
        start[i] = t;
        t += d.n_tiles;
    }
    start[b->n] = t;
    b->total_tiles = t;
    BK(cudaMemcpy(b->d_items, b->items.data(), sizeof(BatchItem) * b->n, cudaMemcpyHostToDevice));
    BK(cudaMemcpy(b->d_start, start.data(), sizeof(long long) * (b->n + 1), cudaMemcpyHostToDevice));
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
        b->graph_iters = -1;
    }
    return PERF_OK;
}

// A p for every scene; with skip_done, scenes whose PCG has exited are
// skipped (their device flag is read by the kernel, so a captured loop of
// max_iter iterations stops working on a scene once it converges).
cudaError_t apply_launch(perf_batch* b, const float* x, const float* p32, cudaStream_t st,
                         bool skip_done = false) {
    return perf::launch_scatter_batch(b->d_items, b->d_start, b->n, b->total_tiles, b->counter, x,
                                      p32, nullptr, b->Ap, nullptr, &b->s[0].pAp,
                                      (int)(sizeof(PcgScalars) / sizeof(double)), 1, b->cap, st,
                                      skip_done ? b->s : nullptr);
}

// Lays the coefficient store out for the current tiling; *use = it fits the
// budget (automatic: free device memory minus 6 GiB).
perf_status ensure_coef(perf_batch* b, cudaStream_t st, bool* use) {
    *use = false;
    if (b->coef_budget == 0 || b->n_rays == 0 || b->total_tiles == 0) return PERF_OK;
    if (!b->tile_off || b->tab_tile_w != b->tile_w) {
        if (b->tile_off) { cudaFree(b->tile_off); b->tile_off = nullptr; }
        int* rows = nullptr;
        BK(cudaMalloc(&rows, sizeof(int) * (size_t)b->total_tiles));
        cudaError_t e = perf::launch_tile_rows_batch(b->d_items, b->d_start, b->n, b->total_tiles,
                                                     rows, st);
        std::vector<int> h((size_t)b->total_tiles);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h.data(), rows, sizeof(int) * h.size(), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        cudaFree(rows);
        BK(e);
        std::vector<long long> off(h.size() + 1, 0);
        for (size_t t = 0; t < h.size(); ++t) off[t + 1] = off[t] + h[t];
        BK(cudaMalloc(&b->tile_off, sizeof(long long) * off.size()));
        BK(cudaMemcpy(b->tile_off, off.data(), sizeof(long long) * off.size(), cudaMemcpyHostToDevice));
        b->coef_rows = off.back();
        b->tab_tile_w = b->tile_w;
    }
    const size_t need = (size_t)b->coef_rows * 32 * 16;
    // the per-ray prefix lengths (4 bytes per ray) come out of the budget too
    const size_t keff_bytes = sizeof(int) * (size_t)b->n_rays;
    size_t budget;
    if (b->coef_budget > 0) {
        budget = (size_t)b->coef_budget;
    } else {
        size_t fr = 0, tot = 0;
        BK(cudaMemGetInfo(&fr, &tot));
        const size_t avail = fr + b->coef_bytes + (b->keff ? keff_bytes : 0),
                     reserve = (size_t)6 << 30;
        budget = avail > reserve ? avail - reserve : 0;
    }
    budget = budget > keff_bytes ? budget - keff_bytes : 0;
    if (need > budget) {
        if (b->coef) { cudaFree(b->coef); b->coef = nullptr; b->coef_bytes = 0; }
        return PERF_OK;
    }
    if (b->coef_bytes < need) {
        if (b->coef) { cudaFree(b->coef); b->coef = nullptr; b->coef_bytes = 0; }
        if (cudaMalloc(&b->coef, need > 0 ? need : 16) != cudaSuccess) {
            cudaGetLastError();
            b->coef = nullptr;
            return PERF_OK;
        }
        b->coef_bytes = need;
    }
    if (!b->keff) {
        // each scene's rays index their own slice; without the array every
        // row is written and read
        if (cudaMalloc(&b->keff, keff_bytes) != cudaSuccess) {
            cudaGetLastError();
            b->keff = nullptr;
        } else {
            for (int i = 0; i < b->n; ++i) b->items[i].sc.keff = b->keff + b->ray_off[i];
            BK(cudaMemcpy(b->d_items, b->items.data(), sizeof(BatchItem) * b->n,
                          cudaMemcpyHostToDevice));
        }
    }
    *use = true;
    return PERF_OK;
}

cudaError_t apply_coef_launch(perf_batch* b, const float* p32, double* pap, cudaStream_t st,
                              bool skip_done) {
    return perf::launch_apply_coef_batch(b->d_items, b->d_start, b->n, b->total_tiles, b->counter,
                                         p32, b->coef, b->tile_off, b->Ap, pap,
                                         (int)(sizeof(PcgScalars) / sizeof(double)), b->cap, st,
                                         skip_done ? b->s : nullptr, b->any_brick);
}

// Gives every scene whose G is a multiple of 2^s the brick order s for its
// PCG vectors (the others stay canonical) and uploads the items; a captured
// PCG loop is dropped when the order changes.
perf_status apply_layout(perf_batch* b, int s) {
    if (s == b->lay_applied && b->d_lay) return PERF_OK;
    if (!b->d_lay) BK(dalloc(&b->d_lay, b->n));
    std::vector<int4> lay(b->n);
    b->any_brick = false;
    for (int i = 0; i < b->n; ++i) {
        DevScene& d = b->items[i].sc;
        perf::set_layout(d, s);
        b->any_brick |= d.lay_s > 0;
        lay[i] = perf::layout_of(d);
    }
    BK(cudaMemcpy(b->d_lay, lay.data(), sizeof(int4) * b->n, cudaMemcpyHostToDevice));
    BK(cudaMemcpy(b->d_items, b->items.data(), sizeof(BatchItem) * b->n, cudaMemcpyHostToDevice));
    b->lay_applied = s;
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
        b->graph_iters = -1;
    }
    return PERF_OK;
}

// One Algorithm 2 iteration for every scene.
cudaError_t pcg_iter(perf_batch* b, cudaStream_t st) {
    cudaError_t e = b->use_coef ? apply_coef_launch(b, b->p, &b->s[0].pAp, st, true)
                                : apply_launch(b, b->x_work, b->p, st, true);
    if (e == cudaSuccess)
        e = perf::launch_pcg_update_seg(b->n_params, b->n, b->d_chunks, b->n_chunks, b->delta, b->rho,
                                        b->p, b->Ap, b->diag, nullptr, 0, b->s, st);
    if (e == cudaSuccess) e = perf::launch_pcg_finish_seg(b->s, b->n, st);
    if (e == cudaSuccess)
        e = perf::launch_pcg_dir_seg(b->n_params, b->n, b->d_chunks, b->n_chunks, b->rho, b->diag,
                                     nullptr, 0, b->p, nullptr, b->s, st);
    return e;
}

perf_status ensure_graph(perf_batch* b, int iters) {
    const float* gc = b->use_coef ? b->coef : nullptr;
    if (b->graph && b->graph_iters == iters && b->graph_coef == gc) return PERF_OK;
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    BK(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < iters && e == cudaSuccess; ++k) e = pcg_iter(b, b->cap_stream);
    cudaError_t e2 = cudaStreamEndCapture(b->cap_stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        b->err = std::string("PCG graph capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2);
        return PERF_ERR_CUDA;
    }
    cudaError_t e3 = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e3 != cudaSuccess) {
        b->err = std::string("PCG graph instantiate: ") + cudaGetErrorString(e3);
        b->graph = nullptr;
        return PERF_ERR_CUDA;
    }
    b->graph_iters = iters;
    b->graph_coef = gc;
    return PERF_OK;
}

}  // namespace

extern "C" {

perf_status perf_batch_create(perf_batch** out, int32_t n_scenes, const perf_scene* scenes,
                              const perf_cameras* cams, const perf_options* opts) {
    if (!out) return PERF_ERR_INVALID_ARG;
    *out = nullptr;
    if (n_scenes < 1 || n_scenes > 4096 || !scenes || !cams || !opts) return PERF_ERR_INVALID_ARG;
    if (opts->aux) return PERF_ERR_UNSUPPORTED;   // the auxiliary residual: single scenes
    if (opts->max_samples < 1 || opts->max_samples > (1 << 20) || opts->pcg_iters < 0 ||
        !(opts->ls_alpha > 0.0 && opts->ls_alpha < 1.0) || opts->ls_max < 0 || opts->ls_max > 200)
        return PERF_ERR_INVALID_ARG;
    perf_batch* b = new (std::nothrow) perf_batch();
    if (!b) return PERF_ERR_INVALID_ARG;
    b->n = n_scenes;
    b->opts = *opts;
    b->items.resize(n_scenes);
    b->seg_h.assign(n_scenes + 1, 0);
    b->ray_off.assign(n_scenes + 1, 0);
    long long cam_total = 0;
    for (int i = 0; i < n_scenes; ++i) {
        const perf_scene& sc = scenes[i];
        const perf_cameras& c = cams[i];
        bool ok = sc.grid_res >= 2 && sc.grid_res <= 1024 && sc.n_shells >= 0 &&
                  sc.n_shells <= PERF_MAX_SHELLS && sc.dtype == PERF_F32 &&
                  (sc.n_shells == 0 || (sc.env_h >= 2 && sc.env_w >= 2)) && c.n_cams >= 0 &&
                  (sc.env_kind == PERF_ENV_EQUIRECT ||
                   (sc.env_kind == PERF_ENV_CUBE && (sc.n_shells == 0 || sc.env_w == 6 * sc.env_h))) &&
                  c.width >= 0 && c.height >= 0 && (c.n_cams == 0 || (c.c2w && c.focal));
        for (int q = 0; ok && q < sc.n_shells; ++q)
            ok = sc.shell_radii[q] > 1.7320508f && (q == 0 || sc.shell_radii[q] > sc.shell_radii[q - 1]);
        for (int q = 0; ok && q < c.n_cams; ++q) ok = c.focal[q] > 0.0f && std::isfinite(c.focal[q]);
        if (!ok) { delete b; return PERF_ERR_INVALID_ARG; }
        const long long G = sc.grid_res;
        const long long texels = sc.n_shells > 0 ? (long long)sc.env_h * sc.env_w : 0;
        const long long blocks = G * G * G + (long long)sc.n_shells * texels;
        b->seg_h[i + 1] = b->seg_h[i] + blocks;
        b->ray_off[i + 1] = b->ray_off[i] + (long long)c.n_cams * c.width * c.height;
        b->max_seg = blocks > b->max_seg ? blocks : b->max_seg;
        cam_total += c.n_cams;
    }
    if (b->seg_h[n_scenes] >= (1ll << 31)) { delete b; return PERF_ERR_INVALID_ARG; }
    b->n_params = 4 * b->seg_h[n_scenes];
    b->n_rays = b->ray_off[n_scenes];
    cudaError_t e = dalloc(&b->cams, 16 * (cam_total > 0 ? cam_total : 1));
    std::vector<float> camh(16 * (size_t)(cam_total > 0 ? cam_total : 1), 0.0f);
    long long cofs = 0;
    for (int i = 0; i < n_scenes && e == cudaSuccess; ++i) {
        const perf_scene& sc = scenes[i];
        const perf_cameras& c = cams[i];
        for (int q = 0; q < c.n_cams; ++q) {
            std::memcpy(&camh[16 * (cofs + q)], c.c2w + 12 * q, 12 * sizeof(float));
            camh[16 * (cofs + q) + 12] = c.focal[q];
        }
        DevScene d;
        std::memset(&d, 0, sizeof(d));
        const long long G = sc.grid_res;
        d.G = (int)G;
        d.halfG = 0.5f * (float)G;
        d.h = 2.0f / (float)G;
        d.S = sc.n_shells;
        for (int q = 0; q < sc.n_shells; ++q) d.R[q] = sc.shell_radii[q];
        d.He = sc.n_shells > 0 ? sc.env_h : 0;
        d.We = sc.n_shells > 0 ? sc.env_w : 0;
        d.env_kind = sc.env_kind;
        d.n_vox = G * G * G;
        set_layout(d, 0);
        d.shell_texels = (long long)d.He * d.We;
        d.W = c.width;
        d.H = c.height;
        d.n_cams = c.n_cams;
        d.n_rays = (long long)c.n_cams * c.width * c.height;
        d.cams = b->cams + 16 * cofs;
        d.max_samples = opts->max_samples;
        d.jitter = opts->jitter;
        d.seed = opts->seed;
        d.epoch = opts->epoch;
        b->items[i].sc = d;
        b->items[i].x_off = 4 * b->seg_h[i];
        b->items[i].r_off = b->ray_off[i];
        cofs += c.n_cams;
    }
    if (e == cudaSuccess)
        e = cudaMemcpy(b->cams, camh.data(), sizeof(float) * camh.size(), cudaMemcpyHostToDevice);
    // shell-hit tables (the batch keeps one jitter epoch): one launch per
    // scene; without room the marches compute the hits themselves in FP32
    if (e == cudaSuccess) {
        long long entries = 0;
        for (int i = 0; i < n_scenes; ++i) entries += b->items[i].sc.n_rays * b->items[i].sc.S;
        if (entries > 0 && cudaMalloc(&b->shell_tab, sizeof(float4) * (size_t)entries) == cudaSuccess) {
            long long off = 0;
            for (int i = 0; i < n_scenes && e == cudaSuccess; ++i) {
                DevScene& d = b->items[i].sc;
                if (d.n_rays * d.S == 0) continue;
                d.shell_tab = nullptr;
                e = perf::launch_shell_table(d, b->shell_tab + off, nullptr);
                d.shell_tab = b->shell_tab + off;
                off += d.n_rays * d.S;
            }
            if (e == cudaSuccess) e = cudaDeviceSynchronize();
        } else {
            cudaGetLastError();
            b->shell_tab = nullptr;
        }
    }
    const long long n = b->n_params, m = 3 * b->n_rays;
    if (e == cudaSuccess) e = dalloc(&b->d_items, n_scenes);
    if (e == cudaSuccess) e = dalloc(&b->d_start, n_scenes + 1);
    if (e == cudaSuccess) e = dalloc(&b->d_seg, n_scenes + 1);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_seg, b->seg_h.data(), sizeof(long long) * (n_scenes + 1), cudaMemcpyHostToDevice);
    // the vector kernels' work split: chunks of at most 4096 parameter blocks,
    // each inside one scene, so every scene gets CTAs in proportion to its size
    if (e == cudaSuccess) {
        const long long kChunk = 4096;
        std::vector<int4> ch;
        for (int i = 0; i < n_scenes; ++i)
            for (long long lo = b->seg_h[i]; lo < b->seg_h[i + 1]; lo += kChunk)
                ch.push_back(make_int4(i, (int)lo, (int)std::min(lo + kChunk, b->seg_h[i + 1]), 0));
        b->n_chunks = (long long)ch.size();
        e = dalloc(&b->d_chunks, b->n_chunks);
        if (e == cudaSuccess && !ch.empty())
            e = cudaMemcpy(b->d_chunks, ch.data(), sizeof(int4) * ch.size(), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = dalloc(&b->counter, 1);
    if (e == cudaSuccess) e = dalloc(&b->x_work, n);
    if (e == cudaSuccess) e = dalloc(&b->x_trial, n);
    if (e == cudaSuccess) e = dalloc(&b->r, m);
    if (e == cudaSuccess) e = dalloc(&b->diag, n);
    if (e == cudaSuccess) e = dalloc(&b->grad, n);
    if (e == cudaSuccess) e = dalloc(&b->delta, n);
    if (e == cudaSuccess) e = dalloc(&b->rho, n);
    if (e == cudaSuccess) e = dalloc(&b->p, n);
    if (e == cudaSuccess) e = dalloc(&b->Ap, n);
    if (e == cudaSuccess) e = dalloc(&b->s, n_scenes);
    if (e == cudaSuccess) e = dalloc(&b->F, n_scenes);
    if (e == cudaSuccess) e = dalloc(&b->gamma, n_scenes);
    if (e == cudaSuccess) e = dalloc(&b->mask, n_scenes);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess || apply_tiling(b, 8) != PERF_OK) {
        perf_batch_destroy(b);
        return PERF_ERR_CUDA;
    }
    *out = b;
    return PERF_OK;
}

perf_status perf_batch_destroy(perf_batch* b) {
    if (!b) return PERF_ERR_INVALID_ARG;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    void* bufs[] = {b->keff, b->shell_tab, b->d_items, b->d_start, b->d_seg, b->d_chunks, b->cams, b->counter, b->x_work, b->x_trial,
                    b->r, b->diag, b->grad, b->delta, b->rho, b->p, b->Ap, b->s, b->F,
                    b->gamma, b->mask, b->tile_off, b->coef, b->d_lay};
    for (void* q : bufs)
        if (q) cudaFree(q);
    delete b;
    return PERF_OK;
}

int64_t perf_batch_param_offset(const perf_batch* b, int32_t scene) {
    if (!b || scene < 0 || scene > b->n) return -1;
    return 4 * b->seg_h[scene];
}

int64_t perf_batch_ray_offset(const perf_batch* b, int32_t scene) {
    if (!b || scene < 0 || scene > b->n) return -1;
    return b->ray_off[scene];
}

const char* perf_batch_last_error(const perf_batch* b) { return b ? b->err.c_str() : "null batch"; }

perf_status perf_batch_render(perf_batch* b, const float* x, float* rgb_out, void* stream) {
    if (!b || !x || !rgb_out) return PERF_ERR_INVALID_ARG;
    BK(perf::launch_forward_batch(b->d_items, b->d_start, b->n, b->total_tiles, b->counter, x,
                                  nullptr, rgb_out, nullptr, nullptr, 0, b->cap, S(stream)));
    return PERF_OK;
}

perf_status perf_batch_residual(perf_batch* b, const float* x, const float* target, float* r_out,
                                double* F_out, void* stream) {
    if (!b || !x || !target || !F_out) return PERF_ERR_INVALID_ARG;
    BK(cudaMemsetAsync(F_out, 0, sizeof(double) * b->n, S(stream)));
    BK(perf::launch_forward_batch(b->d_items, b->d_start, b->n, b->total_tiles, b->counter, x,
                                  target, r_out, F_out, nullptr, r_out ? 1 : 2, b->cap, S(stream)));
    return PERF_OK;
}

perf_status perf_batch_autotune(perf_batch* b, const float* x, perf_tuning* out, void* stream) {
    if (!b || !x) return PERF_ERR_INVALID_ARG;
    cudaStream_t st = S(stream);
    // events live until every return path has left (scope guard)
    EventPair ev;
    BK(cudaEventCreate(&ev.e0));
    BK(cudaEventCreate(&ev.e1));
    cudaEvent_t e0 = ev.e0, e1 = ev.e1;
    BK(cudaMemcpyAsync(b->p, x, sizeof(float) * (size_t)b->n_params, cudaMemcpyDeviceToDevice, st));
    const int tws[4] = {8, 4, 16, 32};
    const int caps[3] = {0, 3, 2};
    float best = 1e30f;
    int best_tw = 8, best_cap = 0, best_s = 0;
    // with the coefficient store (it fits at the default tiling) the
    // coefficient-cached A p is timed, its store laid out and filled at x
    // for every tile shape
    if (apply_layout(b, 0) != PERF_OK) return PERF_ERR_CUDA;
    if (apply_tiling(b, 8) != PERF_OK) return PERF_ERR_CUDA;
    bool coef = false;
    perf_status pc = ensure_coef(b, st, &coef);
    if (pc != PERF_OK) return pc;
    for (int i = 0; i < 4; ++i) {
        if (apply_tiling(b, tws[i]) != PERF_OK) return PERF_ERR_CUDA;
        if (coef) {
            bool fits = false;
            pc = ensure_coef(b, st, &fits);
            if (pc != PERF_OK) return pc;
            if (!fits) continue;
            BK(cudaMemsetAsync(b->diag, 0, sizeof(float) * (size_t)b->n_params, st));
            BK(perf::launch_scatter_batch(b->d_items, b->d_start, b->n, b->total_tiles, b->counter,
                                          x, nullptr, nullptr, b->diag, nullptr, nullptr, 0, 2,
                                          b->cap, st, nullptr, b->coef, b->tile_off));
        }
        auto launch = [&]() {
            return coef ? apply_coef_launch(b, b->p, &b->s[0].pAp, st, false)
                        : apply_launch(b, x, b->p, st);
        };
        auto time_one = [&](float& ms) -> perf_status {
            BK(launch());                                             // warm-up
            BK(cudaEventRecord(e0, st));
            BK(launch());
            BK(cudaEventRecord(e1, st));
            BK(cudaEventSynchronize(e1));
            BK(cudaEventElapsedTime(&ms, e0, e1));
            return PERF_OK;
        };
        float tile_best = 1e30f;
        int tile_cap = 0;
        for (int j = 0; j < 3; ++j) {
            b->cap = caps[j];
            float ms = 0.f;
            pc = time_one(ms);
            if (pc != PERF_OK) return pc;
            if (ms < tile_best) { tile_best = ms; tile_cap = caps[j]; }
            if (ms < best) { best = ms; best_tw = tws[i]; best_cap = caps[j]; best_s = 0; }
        }
        // the brick orders of the PCG vectors (coefficient-cached A p only),
        // at this tile shape's best CTA cap
        for (int ls = 2; coef && ls <= 3; ++ls) {
            if (apply_layout(b, ls) != PERF_OK) return PERF_ERR_CUDA;
            if (!b->any_brick) continue;
            b->cap = tile_cap;
            float ms = 0.f;
            pc = time_one(ms);
            if (pc != PERF_OK) return pc;
            if (ms < best) { best = ms; best_tw = tws[i]; best_cap = tile_cap; best_s = ls; }
        }
        if (apply_layout(b, 0) != PERF_OK) return PERF_ERR_CUDA;
    }
    b->cap = best_cap;
    b->brick_s = best_s;
    if (apply_tiling(b, best_tw) != PERF_OK) return PERF_ERR_CUDA;
    if (out) {
        out->tile_w = best_tw;
        out->tile_h = 32 / best_tw;
        out->ctas_per_sm = best_cap;
        out->apply_ms = best;
        out->paired = 0;
        out->coef = coef ? 1 : 0;
        out->brick = 1 << best_s;
    }
    return PERF_OK;
}

perf_status perf_batch_set_brick(perf_batch* b, int32_t edge) {
    if (!b || (edge != 1 && edge != 2 && edge != 4 && edge != 8)) return PERF_ERR_INVALID_ARG;
    b->brick_s = edge == 8 ? 3 : edge == 4 ? 2 : edge == 2 ? 1 : 0;
    return PERF_OK;
}

perf_status perf_batch_set_coef_budget(perf_batch* b, int64_t bytes) {
    if (!b || bytes < -1) return PERF_ERR_INVALID_ARG;
    b->coef_budget = bytes;
    if (bytes >= 0 && b->coef && b->coef_bytes > (size_t)bytes) {
        cudaFree(b->coef);
        b->coef = nullptr;
        b->coef_bytes = 0;
        b->use_coef = false;
    }
    return PERF_OK;
}

perf_status perf_batch_coef_info(perf_batch* b, int64_t* bytes_held, int32_t* last_used) {
    if (!b) return PERF_ERR_INVALID_ARG;
    if (bytes_held) *bytes_held = (int64_t)b->coef_bytes;
    if (last_used) *last_used = b->use_coef ? 1 : 0;
    return PERF_OK;
}

perf_status perf_batch_gn_solve(perf_batch* b, float* x, const float* target, int32_t n_steps,
                                perf_gn_stats* stats, void* stream) {
    if (!b || !x || !target || n_steps < 0) return PERF_ERR_INVALID_ARG;
    cudaStream_t st = S(stream);
    const perf_options& o = b->opts;
    const int n = b->n;
    bool use = false;
    perf_status ps = ensure_coef(b, st, &use);
    if (ps != PERF_OK) return ps;
    b->use_coef = use;
    ps = apply_layout(b, use ? b->brick_s : 0);
    if (ps != PERF_OK) return ps;
    ps = ensure_graph(b, o.pcg_iters);
    if (ps != PERF_OK) return ps;
    EventPair ev;
    BK(cudaEventCreate(&ev.e0));
    BK(cudaEventCreate(&ev.e1));
    cudaEvent_t e0 = ev.e0, e1 = ev.e1;
    std::vector<double> F0(n), Fm(n), gam(n), mu_prev(n), g_star(n), mu_star(n);
    std::vector<int> live(n), acc(n), evals(n);
    std::vector<PcgScalars> hs(n);
    BK(cudaMemcpyAsync(b->x_work, x, sizeof(float) * (size_t)b->n_params, cudaMemcpyDeviceToDevice, st));
    for (int step = 0; step < n_steps; ++step) {
        BK(cudaEventRecord(e0, st));
        BK(cudaMemsetAsync(b->F, 0, sizeof(double) * n, st));
        BK(perf::launch_forward_batch(b->d_items, b->d_start, n, b->total_tiles, b->counter,
                                      b->x_work, target, b->r, b->F, nullptr, 1, b->cap, st));
        BK(cudaMemsetAsync(b->diag, 0, sizeof(float) * (size_t)b->n_params, st));
        BK(cudaMemsetAsync(b->grad, 0, sizeof(float) * (size_t)b->n_params, st));
        BK(perf::launch_scatter_batch(b->d_items, b->d_start, n, b->total_tiles, b->counter,
                                      b->x_work, nullptr, b->r, b->diag, b->grad, nullptr, 0, 2,
                                      b->cap, st, nullptr, b->use_coef ? b->coef : nullptr,
                                      b->use_coef ? b->tile_off : nullptr, b->any_brick));
        BK(perf::launch_pcg_begin_seg(b->n_params, n, b->d_chunks, b->n_chunks, b->grad, b->diag,
                                      b->delta, b->rho, b->p, nullptr, b->Ap, b->s,
                                      o.pcg_iters, o.pcg_fixed, o.pcg_eps_rel, o.pcg_stall,
                                      nullptr, 0, st));
        if (o.pcg_iters > 0) BK(cudaGraphLaunch(b->graph, st));
        BK(cudaMemcpyAsync(F0.data(), b->F, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
        BK(cudaStreamSynchronize(st));
        // Algorithm 3 for every scene at once
        for (int i = 0; i < n; ++i) {
            gam[i] = 1.0;
            mu_prev[i] = 3.4028234663852886e38;
            live[i] = 1;
            evals[i] = 0;
            g_star[i] = 1.0;
            mu_star[i] = mu_prev[i];
        }
        for (int it = 0; it <= o.ls_max; ++it) {
            int any = 0;
            for (int i = 0; i < n; ++i) any |= live[i];
            if (!any) break;
            BK(cudaMemcpyAsync(b->gamma, gam.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st));
            BK(cudaMemcpyAsync(b->mask, live.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
            BK(perf::launch_trial_seg(b->n_params, n, b->d_chunks, b->n_chunks, b->x_work, b->delta,
                                      b->gamma, b->mask, o.project, b->x_trial, st,
                                      b->any_brick ? b->d_lay : nullptr, b->d_seg));
            BK(cudaMemsetAsync(b->F, 0, sizeof(double) * n, st));
            BK(perf::launch_forward_batch(b->d_items, b->d_start, n, b->total_tiles, b->counter,
                                          b->x_trial, target, nullptr, b->F, b->mask, 2, b->cap, st));
            BK(cudaMemcpyAsync(Fm.data(), b->F, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
            BK(cudaStreamSynchronize(st));
            for (int i = 0; i < n; ++i) {
                if (!live[i]) continue;
                double mu = std::isnan(Fm[i]) ? INFINITY : Fm[i];
                ++evals[i];
                if (mu > mu_prev[i]) {
                    g_star[i] = gam[i] / o.ls_alpha;
                    mu_star[i] = mu_prev[i];
                    live[i] = 0;
                    continue;
                }
                gam[i] *= o.ls_alpha;
                mu_prev[i] = mu;
                if (it == o.ls_max) {
                    g_star[i] = gam[i] / o.ls_alpha;
                    mu_star[i] = mu_prev[i];
                    live[i] = 0;
                }
            }
        }
        for (int i = 0; i < n; ++i) acc[i] = std::isfinite(mu_star[i]) && mu_star[i] < F0[i];
        BK(cudaMemcpyAsync(b->gamma, g_star.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st));
        BK(cudaMemcpyAsync(b->mask, acc.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
        BK(perf::launch_trial_seg(b->n_params, n, b->d_chunks, b->n_chunks, b->x_work, b->delta,
                                  b->gamma, b->mask, o.project, b->x_work, st,
                                  b->any_brick ? b->d_lay : nullptr, b->d_seg));
        BK(cudaEventRecord(e1, st));
        BK(cudaMemcpyAsync(hs.data(), b->s, sizeof(PcgScalars) * n, cudaMemcpyDeviceToHost, st));
        BK(cudaStreamSynchronize(st));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (stats) {
            for (int i = 0; i < n; ++i) {
                perf_gn_stats& g = stats[(size_t)step * n + i];
                g.F_before = F0[i];
                g.F_after = acc[i] ? mu_star[i] : F0[i];
                g.gamma = g_star[i];
                g.accepted = acc[i];
                g.ls_evals = evals[i];
                g.pcg.iters = hs[i].iter;
                g.pcg.exit_reason = hs[i].exit_reason;
                g.pcg.R0 = hs[i].R0;
                g.pcg.R = hs[i].R;
                g.pcg.rz = hs[i].rz;
                g.ms = ms;
            }
        }
    }
    BK(cudaMemcpyAsync(x, b->x_work, sizeof(float) * (size_t)b->n_params, cudaMemcpyDeviceToDevice, st));
    BK(cudaStreamSynchronize(st));
    return PERF_OK;
}

}  // extern "C"

// perf_noalloc.cu -- perf_residual_noalloc: the residual / objective ray march
// without a context and without any device allocation.
//
// Some callers cannot allocate device memory when they want a residual: an
// application that fixes its device-memory budget at start-up and refuses to
// grow it afterwards, an engine whose own pool allocator owns all device
// memory and forbids other cudaMalloc calls, or a latency-critical loop that
// cannot afford the implicit synchronisation cudaMalloc / cudaFree may bring.
// perf_create allocates (camera table, workspace), so those callers use this
// entry point instead: the camera table it needs lives in the file-scope
// array below, which every GPU that loads the library holds until exit.
#include <cmath>
#include <cstring>

#include <cuda_runtime.h>

#include "../../include/perf.h"
#include "perf_kernels.h"

namespace {

// 16 floats per camera: c2w (12), focal, padding.
__device__ __align__(256) float g_noalloc_cams[PERF_NOALLOC_MAX_CAMS * 16];

// Host staging of one call's camera table (static storage, not an allocation).
float h_stage[PERF_NOALLOC_MAX_CAMS * 16];

// Device address of g_noalloc_cams per device, looked up once per device.
constexpr int kMaxDevices = 64;
float* d_cams[kMaxDevices] = {nullptr};

perf_status setup(float** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PERF_ERR_CUDA;
    if (!d_cams[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_cams) != cudaSuccess || p == nullptr)
            return PERF_ERR_CUDA;
        d_cams[dev] = static_cast<float*>(p);
    }
    *out = d_cams[dev];
    return PERF_OK;
}

}  // namespace

extern "C" perf_status perf_residual_noalloc(const perf_scene* sc, const perf_cameras* cams,
                                             const perf_options* opts, const void* x,
                                             const void* target, void* r_out, double* F_out,
                                             void* stream) {
    if (!sc || !cams || !opts || !F_out) return PERF_ERR_INVALID_ARG;
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
    if (opts->max_samples < 1 || opts->max_samples > (1 << 20)) return PERF_ERR_INVALID_ARG;
    if (opts->aux) return PERF_ERR_UNSUPPORTED;   // the 3-channel residual only
    if (cams->n_cams < 0 || cams->width < 0 || cams->height < 0) return PERF_ERR_INVALID_ARG;
    // the static camera table holds at most PERF_NOALLOC_MAX_CAMS cameras
    if (cams->n_cams > PERF_NOALLOC_MAX_CAMS) return PERF_ERR_INVALID_ARG;
    const long long n_rays = (long long)cams->n_cams * cams->width * cams->height;
    if (n_rays > 0 && (!cams->c2w || !cams->focal || !x || !target)) return PERF_ERR_INVALID_ARG;
    for (int c = 0; c < cams->n_cams; ++c)
        if (!(cams->focal[c] > 0.0f) || !std::isfinite(cams->focal[c])) return PERF_ERR_INVALID_ARG;
    const long long G = sc->grid_res;
    const long long texels = sc->n_shells > 0 ? (long long)sc->env_h * sc->env_w : 0;
    if (G * G * G + (long long)sc->n_shells * texels >= (1ll << 31)) return PERF_ERR_INVALID_ARG;

    float* dcam = nullptr;
    perf_status st = setup(&dcam);
    if (st != PERF_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(F_out, 0, sizeof(double), s) != cudaSuccess) return PERF_ERR_CUDA;
    if (n_rays == 0) return PERF_OK;

    for (int c = 0; c < cams->n_cams; ++c) {
        std::memcpy(h_stage + 16 * c, cams->c2w + 12 * c, 12 * sizeof(float));
        h_stage[16 * c + 12] = cams->focal[c];
        h_stage[16 * c + 13] = h_stage[16 * c + 14] = h_stage[16 * c + 15] = 0.0f;
    }
    // pageable source: the copy has consumed h_stage when this returns
    if (cudaMemcpyAsync(dcam, h_stage, sizeof(float) * 16 * (size_t)cams->n_cams,
                        cudaMemcpyHostToDevice, s) != cudaSuccess)
        return PERF_ERR_CUDA;

    perf::DevScene d;
    std::memset(&d, 0, sizeof(d));
    d.G = (int)G;
    d.halfG = 0.5f * (float)G;
    d.h = 2.0f / (float)G;
    d.S = sc->n_shells;
    for (int q = 0; q < sc->n_shells; ++q) d.R[q] = sc->shell_radii[q];
    d.He = sc->n_shells > 0 ? sc->env_h : 0;
    d.We = sc->n_shells > 0 ? sc->env_w : 0;
    d.env_kind = sc->env_kind;
    d.n_vox = G * G * G;
    set_layout(d, 0);
    d.shell_texels = texels;
    d.W = cams->width;
    d.H = cams->height;
    d.n_cams = cams->n_cams;
    d.n_rays = n_rays;
    d.tile_w = 8;
    d.tile_h = 4;
    d.tiles_x = (cams->width + d.tile_w - 1) / d.tile_w;
    d.tiles_y = (cams->height + d.tile_h - 1) / d.tile_h;
    d.n_tiles = (long long)d.tiles_x * d.tiles_y * cams->n_cams;
    d.cams = dcam;
    d.max_samples = opts->max_samples;
    d.jitter = opts->jitter;
    d.seed = opts->seed;
    d.epoch = opts->epoch;
    if (perf::launch_forward(d, sc->dtype, x, target, r_out, nullptr, F_out, r_out ? 1 : 2, s) !=
        cudaSuccess)
        return PERF_ERR_CUDA;
    return PERF_OK;
}

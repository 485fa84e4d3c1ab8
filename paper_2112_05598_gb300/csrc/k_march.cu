// k_march.cu -- ray-march kernels of the PERF Gauss-Newton step (sm_103a).
//
//   k_forward   Eq. 3-4 composite: image, residual r = H^ - C, F (Eq. 5-6)
//   k_jvp       J p by a forward tangent sweep of Eq. 3
//   k_scatter   J^T v, the fused A p = J^T (J p), and diag(J^T J) with J^T r
//
// Derivatives (Algorithm 1, Section "Computation of partial derivatives"):
// for sample i with transmittance T_i, e_i = exp(-sigma_i dbar_i),
// alpha_i = 1 - e_i and weight w_i = T_i alpha_i,
//   dH/dc_i       = w_i
//   dH_k/dsigma_i = dbar_i (T_i e_i c_ik - G_ik),   G_i = sum_{j>i} w_j c_j.
// Algorithm 1 obtains G_i by a backward sweep; here G_i = H^ - P_i with the
// forward prefix P_i = sum_{j<=i} w_j c_j and H^ from a first sweep, so each
// ray is marched front to back twice (the paper also invokes Algorithm 1
// twice per ray for A p) and no per-sample state is stored.
//
// Scatter: consecutive samples of one ray share most of their 8 trilinear
// voxels.  A register window of the 2x2x2 voxels of the current sample keeps
// one running sum per voxel; a voxel is flushed (one 16-byte vector atomic)
// when the window slides past it.  Because a voxel's trilinear support is a
// box, the samples of one ray that touch it are consecutive, so each voxel is
// flushed exactly once per ray -- which also makes the window compute the
// EXACT diag(J^T J): a row's entry for a voxel is complete before it is
// squared (Section "Preconditioner").
#include "perf_device.cuh"
#include "perf_kernels.h"

namespace perf {

constexpr int kThreads = 128;
constexpr int kWarps = kThreads / 32;

// ------------------------------------------------------------------ helpers

struct Comp {   // running composite of one ray
    float T, H[3];
};

__device__ __forceinline__ void comp_step(Comp& s, const float4 a, float dbar) {
    const float e = expf(-__fmul_rn(a.w, dbar));
    const float w = __fmul_rn(s.T, __fsub_rn(1.0f, e));
    s.H[0] = fmaf(w, a.x, s.H[0]);
    s.H[1] = fmaf(w, a.y, s.H[1]);
    s.H[2] = fmaf(w, a.z, s.H[2]);
    s.T = __fmul_rn(s.T, e);
}

// Eq. 3-4 over the grid samples and then the shells.
template <typename T>
__device__ __forceinline__ void composite(const DevScene& sc, const T* __restrict__ x,
                                          const Ray& R, long long ray, Comp& s, float& T_exit) {
    s.T = 1.0f;
    s.H[0] = s.H[1] = s.H[2] = 0.0f;
    const float dbar = R.delta * sc.halfG;
    for (int k = 0; k < R.K; ++k) {
        const Cell cl = sample_cell(sc, R, ray, k);
        comp_step(s, interp_grid(x, sc, cl), dbar);
    }
    T_exit = s.T;
    for (int q = 0; q < sc.S; ++q) {
        ShellHit hs;
        if (shell_lookup(sc, R, q, hs)) comp_step(s, interp_shell(x, hs), 1.0f);
    }
}

// Tangent sweep: H^ and (J p) of one ray.
struct Tang {
    float T, Td, H[3], J[3];
};

__device__ __forceinline__ void tang_step(Tang& s, const float4 a, const float4 q, float dbar) {
    const float e = expf(-__fmul_rn(a.w, dbar));
    const float alpha = __fsub_rn(1.0f, e);
    const float w = __fmul_rn(s.T, alpha);
    const float tsd = s.T * dbar * q.w;               // T dbar sigma_dot
    const float coef = fmaf(s.Td, alpha, tsd * e);     // T_dot alpha + T e dbar sigma_dot
    s.J[0] = fmaf(coef, a.x, fmaf(w, q.x, s.J[0]));
    s.J[1] = fmaf(coef, a.y, fmaf(w, q.y, s.J[1]));
    s.J[2] = fmaf(coef, a.z, fmaf(w, q.z, s.J[2]));
    s.H[0] = fmaf(w, a.x, s.H[0]);
    s.H[1] = fmaf(w, a.y, s.H[1]);
    s.H[2] = fmaf(w, a.z, s.H[2]);
    s.Td = e * (s.Td - tsd);
    s.T = __fmul_rn(s.T, e);
}

template <typename T, typename TP>
__device__ __forceinline__ void tangent(const DevScene& sc, const T* __restrict__ x,
                                        const TP* __restrict__ p, const Ray& R, long long ray,
                                        Tang& s) {
    s.T = 1.0f; s.Td = 0.0f;
    s.H[0] = s.H[1] = s.H[2] = 0.0f;
    s.J[0] = s.J[1] = s.J[2] = 0.0f;
    const float dbar = R.delta * sc.halfG;
    for (int k = 0; k < R.K; ++k) {
        const Cell cl = sample_cell(sc, R, ray, k);
        tang_step(s, interp_grid(x, sc, cl), interp_grid(p, sc, cl), dbar);
    }
    for (int q = 0; q < sc.S; ++q) {
        ShellHit hs;
        if (shell_lookup(sc, R, q, hs)) tang_step(s, interp_shell(x, hs), interp_shell(p, hs), 1.0f);
    }
}

// ------------------------------------------------------- voxel window

template <int NV>
struct Window {
    float v[8][NV];
    int b[3];
};

template <int NV>
__device__ __forceinline__ void win_zero(Window<NV>& w, int c) {
#pragma unroll
    for (int q = 0; q < NV; ++q) w.v[c][q] = 0.0f;
}

template <int NV>
__device__ __forceinline__ void win_move(Window<NV>& w, int dst, int src) {
#pragma unroll
    for (int q = 0; q < NV; ++q) w.v[dst][q] = w.v[src][q];
}

template <int NV, class F>
__device__ __forceinline__ void win_flush(Window<NV>& w, int c, int G, F& fl) {
    const long long key = ((long long)(w.b[2] + (c >> 2)) * G + (w.b[1] + ((c >> 1) & 1))) * G +
                          (w.b[0] + (c & 1));
    fl(key, w.v[c]);
}

// Slide the window along axis A to base nb, flushing the voxels it leaves.
template <int A, int NV, class F>
__device__ __forceinline__ void win_shift(Window<NV>& w, int nb, int G, F& fl) {
    const int d = nb - w.b[A];
    if (d == 0) return;
    constexpr int B = 1 << A;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        if (c & B) continue;
        const int lo = c, hi = c | B;
        if (d == 1) {
            win_flush(w, lo, G, fl);
            win_move(w, lo, hi);
            win_zero(w, hi);
        } else if (d == -1) {
            win_flush(w, hi, G, fl);
            win_move(w, hi, lo);
            win_zero(w, lo);
        } else {
            win_flush(w, lo, G, fl);
            win_flush(w, hi, G, fl);
            win_zero(w, lo);
            win_zero(w, hi);
        }
    }
    w.b[A] = nb;
}

template <int NV, class F>
__device__ __forceinline__ void win_goto(Window<NV>& w, const Cell& cl, int G, F& fl) {
    win_shift<0>(w, cl.bx, G, fl);
    win_shift<1>(w, cl.by, G, fl);
    win_shift<2>(w, cl.bz, G, fl);
}

template <int NV>
__device__ __forceinline__ void win_add(Window<NV>& w, const Cell& cl, const float (&val)[NV]) {
    const float wx[2] = {1.0f - cl.fx, cl.fx};
    const float wy[2] = {1.0f - cl.fy, cl.fy};
    const float wz[2] = {1.0f - cl.fz, cl.fz};
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const float W = wx[c & 1] * wy[(c >> 1) & 1] * wz[c >> 2];
#pragma unroll
        for (int q = 0; q < NV; ++q) w.v[c][q] = fmaf(W, val[q], w.v[c][q]);
    }
}

// ------------------------------------------------------------- sinks

__device__ __forceinline__ void red_add4(float* base, long long blk, float4 v) {
    atomicAdd(reinterpret_cast<float4*>(base) + blk, v);
}

// J^T v: per voxel the colour part is v_k sum W w_i, the opacity part
// sum W (v . dH/dsigma_i); the window keeps (sum W w_i, sum W v.dH/dsigma_i).
struct VjpFlush {
    float* out;
    float v0, v1, v2;
    __device__ __forceinline__ void operator()(long long key, const float (&a)[2]) {
        if (a[0] != 0.0f || a[1] != 0.0f)
            red_add4(out, key, make_float4(a[0] * v0, a[0] * v1, a[0] * v2, a[1]));
    }
};

struct VjpSink {
    Window<2> w;
    VjpFlush fl;
    int G;
    bool started;
    __device__ __forceinline__ void grid(const Cell& cl, float wi, const float (&ds)[3]) {
        if (!started) {
            w.b[0] = cl.bx; w.b[1] = cl.by; w.b[2] = cl.bz;
#pragma unroll
            for (int c = 0; c < 8; ++c) win_zero(w, c);
            started = true;
        } else {
            win_goto(w, cl, G, fl);
        }
        const float val[2] = {wi, fl.v0 * ds[0] + fl.v1 * ds[1] + fl.v2 * ds[2]};
        win_add(w, cl, val);
    }
    __device__ __forceinline__ void end_grid() {
        if (!started) return;
#pragma unroll
        for (int c = 0; c < 8; ++c) win_flush(w, c, G, fl);
    }
    __device__ __forceinline__ void shell(const ShellHit& hs, float wi, const float (&ds)[3]) {
        const float s = fl.v0 * ds[0] + fl.v1 * ds[1] + fl.v2 * ds[2];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float W = hs.w[q];
            if (W != 0.0f)
                red_add4(fl.out, hs.idx[q],
                         make_float4(W * wi * fl.v0, W * wi * fl.v1, W * wi * fl.v2, W * s));
        }
    }
};

// diag(J^T J) and J^T r: the window keeps, per voxel, the row entries
// a = sum W w_i (colour, same for the three residuals) and
// s_k = sum W dH_k/dsigma_i; at the flush they are squared (diag) and
// multiplied by r (gradient).
struct DiagFlush {
    float* diag;
    float* grad;
    float r0, r1, r2;
    __device__ __forceinline__ void operator()(long long key, const float (&a)[4]) {
        if (a[0] == 0.0f && a[1] == 0.0f && a[2] == 0.0f && a[3] == 0.0f) return;
        const float aa = a[0] * a[0];
        red_add4(diag, key, make_float4(aa, aa, aa, a[1] * a[1] + a[2] * a[2] + a[3] * a[3]));
        if (grad)
            red_add4(grad, key, make_float4(a[0] * r0, a[0] * r1, a[0] * r2,
                                            a[1] * r0 + a[2] * r1 + a[3] * r2));
    }
};

struct DiagSink {
    Window<4> w;
    DiagFlush fl;
    int G;
    bool started;
    __device__ __forceinline__ void grid(const Cell& cl, float wi, const float (&ds)[3]) {
        if (!started) {
            w.b[0] = cl.bx; w.b[1] = cl.by; w.b[2] = cl.bz;
#pragma unroll
            for (int c = 0; c < 8; ++c) win_zero(w, c);
            started = true;
        } else {
            win_goto(w, cl, G, fl);
        }
        const float val[4] = {wi, ds[0], ds[1], ds[2]};
        win_add(w, cl, val);
    }
    __device__ __forceinline__ void end_grid() {
        if (!started) return;
#pragma unroll
        for (int c = 0; c < 8; ++c) win_flush(w, c, G, fl);
    }
    __device__ __forceinline__ void shell(const ShellHit& hs, float wi, const float (&ds)[3]) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float W = hs.w[q];
            if (W == 0.0f) continue;
            const float a[4] = {W * wi, W * ds[0], W * ds[1], W * ds[2]};
            fl(hs.idx[q], a);
        }
    }
};

// Second sweep: per-sample partials (Algorithm 1 quantities) into a sink.
template <typename T, class Sink>
__device__ __forceinline__ void scatter_sweep(const DevScene& sc, const T* __restrict__ x,
                                              const Ray& R, long long ray, const float (&Hh)[3],
                                              Sink& sink) {
    float Tr = 1.0f;
    float P[3] = {0.0f, 0.0f, 0.0f};
    const float dbar = R.delta * sc.halfG;
    for (int k = 0; k < R.K; ++k) {
        const Cell cl = sample_cell(sc, R, ray, k);
        const float4 a = interp_grid(x, sc, cl);
        const float e = expf(-__fmul_rn(a.w, dbar));
        const float w = __fmul_rn(Tr, __fsub_rn(1.0f, e));
        P[0] = fmaf(w, a.x, P[0]);
        P[1] = fmaf(w, a.y, P[1]);
        P[2] = fmaf(w, a.z, P[2]);
        const float te = Tr * e;
        const float ds[3] = {dbar * (te * a.x - (Hh[0] - P[0])),
                             dbar * (te * a.y - (Hh[1] - P[1])),
                             dbar * (te * a.z - (Hh[2] - P[2]))};
        sink.grid(cl, w, ds);
        Tr = __fmul_rn(Tr, e);
    }
    sink.end_grid();
    for (int q = 0; q < sc.S; ++q) {
        ShellHit hs;
        if (!shell_lookup(sc, R, q, hs)) continue;
        const float4 a = interp_shell(x, hs);
        const float e = expf(-a.w);
        const float w = __fmul_rn(Tr, __fsub_rn(1.0f, e));
        P[0] = fmaf(w, a.x, P[0]);
        P[1] = fmaf(w, a.y, P[1]);
        P[2] = fmaf(w, a.z, P[2]);
        const float te = Tr * e;
        const float ds[3] = {te * a.x - (Hh[0] - P[0]), te * a.y - (Hh[1] - P[1]),
                             te * a.z - (Hh[2] - P[2])};
        sink.shell(hs, w, ds);
        Tr = __fmul_rn(Tr, e);
    }
}

// ------------------------------------------------------------- kernels

#define PERF_TILE_LOOP                                                              \
    const int lane = threadIdx.x & 31;                                              \
    const long long nw = (long long)gridDim.x * kWarps;                             \
    for (long long tile = (long long)blockIdx.x * kWarps + (threadIdx.x >> 5);      \
         tile < sc.n_tiles; tile += nw)

template <typename T, int MODE>   // 0 render, 1 residual (+F), 2 F only
__global__ void __launch_bounds__(kThreads) k_forward(DevScene sc, const T* __restrict__ x,
                                                      const float* __restrict__ target,
                                                      float* __restrict__ out,
                                                      float* __restrict__ T_out, double* F) {
    double facc = 0.0;
    PERF_TILE_LOOP {
        long long ray;
        if (!tile_pixel(sc, tile, lane, ray)) continue;
        Ray R;
        ray_setup(sc, ray, R);
        Comp s;
        float Te;
        composite(sc, x, R, ray, s, Te);
        if (MODE == 0) {
            out[3 * ray + 0] = s.H[0];
            out[3 * ray + 1] = s.H[1];
            out[3 * ray + 2] = s.H[2];
            if (T_out) T_out[ray] = Te;
        } else {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float r = s.H[k] - target[3 * ray + k];
                if (MODE == 1 && out) out[3 * ray + k] = r;
                facc += 0.5 * (double)r * (double)r;
            }
        }
    }
    if (MODE != 0) block_add_f64<kWarps>(facc, F);
}

template <typename T, typename TP>
__global__ void __launch_bounds__(kThreads) k_jvp(DevScene sc, const T* __restrict__ x,
                                                  const TP* __restrict__ p, float* __restrict__ out) {
    PERF_TILE_LOOP {
        long long ray;
        if (!tile_pixel(sc, tile, lane, ray)) continue;
        Ray R;
        ray_setup(sc, ray, R);
        Tang s;
        tangent(sc, x, p, R, ray, s);
        out[3 * ray + 0] = s.J[0];
        out[3 * ray + 1] = s.J[1];
        out[3 * ray + 2] = s.J[2];
    }
}

template <typename T, typename TP, int MODE>   // 0 vjp, 1 apply A, 2 diag (+grad)
__global__ void __launch_bounds__(kThreads) k_scatter(DevScene sc, const T* __restrict__ x,
                                                      const TP* __restrict__ p,
                                                      const float* __restrict__ v,
                                                      float* __restrict__ out,
                                                      float* __restrict__ out2, double* pap) {
    double acc = 0.0;
    PERF_TILE_LOOP {
        long long ray;
        if (!tile_pixel(sc, tile, lane, ray)) continue;
        Ray R;
        ray_setup(sc, ray, R);
        float Hh[3], vr[3];
        if (MODE == 1) {
            Tang s;
            tangent(sc, x, p, R, ray, s);
            Hh[0] = s.H[0]; Hh[1] = s.H[1]; Hh[2] = s.H[2];
            vr[0] = s.J[0]; vr[1] = s.J[1]; vr[2] = s.J[2];
            acc += (double)vr[0] * vr[0] + (double)vr[1] * vr[1] + (double)vr[2] * vr[2];
        } else {
            if (MODE == 0) {
                vr[0] = v[3 * ray]; vr[1] = v[3 * ray + 1]; vr[2] = v[3 * ray + 2];
                if (vr[0] == 0.0f && vr[1] == 0.0f && vr[2] == 0.0f) continue;
            } else {
                vr[0] = v ? v[3 * ray] : 0.0f;
                vr[1] = v ? v[3 * ray + 1] : 0.0f;
                vr[2] = v ? v[3 * ray + 2] : 0.0f;
            }
            Comp s;
            float Te;
            composite(sc, x, R, ray, s, Te);
            Hh[0] = s.H[0]; Hh[1] = s.H[1]; Hh[2] = s.H[2];
        }
        if (MODE == 2) {
            DiagSink sink;
            sink.fl.diag = out; sink.fl.grad = out2;
            sink.fl.r0 = vr[0]; sink.fl.r1 = vr[1]; sink.fl.r2 = vr[2];
            sink.G = sc.G; sink.started = false;
            scatter_sweep(sc, x, R, ray, Hh, sink);
        } else {
            if (vr[0] == 0.0f && vr[1] == 0.0f && vr[2] == 0.0f) continue;
            VjpSink sink;
            sink.fl.out = out;
            sink.fl.v0 = vr[0]; sink.fl.v1 = vr[1]; sink.fl.v2 = vr[2];
            sink.G = sc.G; sink.started = false;
            scatter_sweep(sc, x, R, ray, Hh, sink);
        }
    }
    if (MODE == 1 && pap) block_add_f64<kWarps>(acc, pap);
}

__global__ void __launch_bounds__(kThreads) k_count(DevScene sc, unsigned long long* out) {
    unsigned long long n = 0;
    PERF_TILE_LOOP {
        long long ray;
        if (!tile_pixel(sc, tile, lane, ray)) continue;
        Ray R;
        ray_setup(sc, ray, R);
        n += (unsigned long long)R.K + (unsigned long long)__popc(R.shell_hit);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
    if ((threadIdx.x & 31) == 0 && n) atomicAdd(out, n);
}

// ------------------------------------------------------------- launchers

static int grid_blocks(const void* fn, long long n_tiles) {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kThreads, 0);
    if (occ <= 0) occ = 1;
    long long want = (n_tiles + kWarps - 1) / kWarps;
    long long cap = (long long)sms * occ;
    long long b = want < cap ? want : cap;
    return (int)(b > 0 ? b : 1);
}

template <typename T>
cudaError_t launch_forward_t(const DevScene& sc, const void* x, const float* target, float* out,
                             float* T_out, double* F, int mode, cudaStream_t st) {
    const T* xx = static_cast<const T*>(x);
    if (sc.n_tiles == 0) return cudaSuccess;
    if (mode == 0) {
        auto fn = k_forward<T, 0>;
        fn<<<grid_blocks((const void*)fn, sc.n_tiles), kThreads, 0, st>>>(sc, xx, target, out, T_out, F);
    } else if (mode == 1) {
        auto fn = k_forward<T, 1>;
        fn<<<grid_blocks((const void*)fn, sc.n_tiles), kThreads, 0, st>>>(sc, xx, target, out, T_out, F);
    } else {
        auto fn = k_forward<T, 2>;
        fn<<<grid_blocks((const void*)fn, sc.n_tiles), kThreads, 0, st>>>(sc, xx, target, out, T_out, F);
    }
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_count_samples(const DevScene& sc, unsigned long long* out, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess || sc.n_tiles == 0) return e;
    k_count<<<grid_blocks((const void*)k_count, sc.n_tiles), kThreads, 0, st>>>(sc, out);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_forward(const DevScene& sc, int dtype, const void* x, const float* target,
                           float* out, float* T_out, double* F, int mode, cudaStream_t st) {
    return dtype == 1 ? launch_forward_t<__nv_bfloat16>(sc, x, target, out, T_out, F, mode, st)
                      : launch_forward_t<float>(sc, x, target, out, T_out, F, mode, st);
}

template <typename T, typename TP>
cudaError_t launch_jvp_t(const DevScene& sc, const void* x, const void* p, float* out,
                         cudaStream_t st) {
    if (sc.n_tiles == 0) return cudaSuccess;
    auto fn = k_jvp<T, TP>;
    fn<<<grid_blocks((const void*)fn, sc.n_tiles), kThreads, 0, st>>>(
        sc, static_cast<const T*>(x), static_cast<const TP*>(p), out);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_jvp(const DevScene& sc, int dtype, const void* x, const void* p, int p_dtype,
                       float* out, cudaStream_t st) {
    if (dtype == 1)
        return p_dtype == 1 ? launch_jvp_t<__nv_bfloat16, __nv_bfloat16>(sc, x, p, out, st)
                            : launch_jvp_t<__nv_bfloat16, float>(sc, x, p, out, st);
    return launch_jvp_t<float, float>(sc, x, p, out, st);
}

template <typename T, typename TP, int MODE>
cudaError_t launch_scatter_t(const DevScene& sc, const void* x, const void* p, const float* v,
                             float* out, float* out2, double* pap, cudaStream_t st) {
    if (sc.n_tiles == 0) return cudaSuccess;
    auto fn = k_scatter<T, TP, MODE>;
    fn<<<grid_blocks((const void*)fn, sc.n_tiles), kThreads, 0, st>>>(
        sc, static_cast<const T*>(x), static_cast<const TP*>(p), v, out, out2, pap);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_scatter(const DevScene& sc, int dtype, int mode, const void* x, const void* p,
                           int p_dtype, const float* v, float* out, float* out2, double* pap,
                           cudaStream_t st) {
    if (dtype == 1) {
        if (mode == 1)
            return p_dtype == 1
                       ? launch_scatter_t<__nv_bfloat16, __nv_bfloat16, 1>(sc, x, p, v, out, out2, pap, st)
                       : launch_scatter_t<__nv_bfloat16, float, 1>(sc, x, p, v, out, out2, pap, st);
        if (mode == 0) return launch_scatter_t<__nv_bfloat16, float, 0>(sc, x, p, v, out, out2, pap, st);
        return launch_scatter_t<__nv_bfloat16, float, 2>(sc, x, p, v, out, out2, pap, st);
    }
    if (mode == 1) return launch_scatter_t<float, float, 1>(sc, x, p, v, out, out2, pap, st);
    if (mode == 0) return launch_scatter_t<float, float, 0>(sc, x, p, v, out, out2, pap, st);
    return launch_scatter_t<float, float, 2>(sc, x, p, v, out, out2, pap, st);
}

}  // namespace perf

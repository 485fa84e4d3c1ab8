// k_pcg.cu -- vector work of Algorithm 2 (preconditioned conjugate gradients)
// and of the line search (Algorithm 3), fused so that each n-vector is read
// and written as few times as the recurrence allows (Section "Update step":
// the vector additions and inner products run in parallel on the GPU).
//
// The CG recurrence vectors Delta, rho and p are FP64 (the vector kernels are
// a few hundred MB of traffic per iteration against a ray march of tens of
// ms, and FP32 recurrences lose conjugacy within 20 iterations on these
// ill-conditioned normal equations); A p arrives in FP32 from the ray-march
// scatter, and p is also written as FP32 (and BF16) for the next march's
// gathers.  One thread handles one parameter block (4 values = one voxel or
// texel); inner products accumulate in FP64.
//   begin : rho = b = -grad, z = M^-1 rho, p = z, Delta = 0, R0, rho^T z
//   update: Delta += alpha p, rho -= alpha A p, z = M^-1 rho, R, rho^T z
//   finish: exit test (R < eps^2 R0 or R / R_prev > stall, or a fixed count),
//           beta = rho'^T z' / rho^T z                               [1 thread]
//   dir   : p = z + beta p, A p = 0 for the next scatter
// M^-1 is Jacobi (z_j = rho_j / d_j, 0 where d_j <= 1e-30) or, where 4x4 blocks
// are given for the grid voxels, z_v = P_v rho_v per voxel.
#include <cuda_bf16.h>
#include "perf_kernels.h"

namespace perf {

unsigned long long g_launches = 0;

constexpr int kVThreads = 256;

static int vec_blocks(long long nblk) {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    long long want = (nblk + kVThreads - 1) / kVThreads;
    long long cap = (long long)sms * 8;
    long long b = want < cap ? want : cap;
    return (int)(b > 0 ? b : 1);
}

// Jacobi entries at or below this are treated as unobserved (z = 0): the
// square of a row entry below ~1e-19 is not a normal binary32 number, so such
// parameters (deep behind opaque matter) cannot be told apart from ones no ray
// sees; 1e-30 keeps full binary32 precision above the cut.
constexpr float kJacobiFloor = 1e-30f;

struct D4 {
    double x, y, z, w;
};

__device__ __forceinline__ D4 ld4(const double* a, long long v) {
    const double2 lo = reinterpret_cast<const double2*>(a)[2 * v];
    const double2 hi = reinterpret_cast<const double2*>(a)[2 * v + 1];
    return D4{lo.x, lo.y, hi.x, hi.y};
}

__device__ __forceinline__ void st4(double* a, long long v, const D4& d) {
    reinterpret_cast<double2*>(a)[2 * v] = make_double2(d.x, d.y);
    reinterpret_cast<double2*>(a)[2 * v + 1] = make_double2(d.z, d.w);
}

__device__ __forceinline__ D4 precond(const D4& r, long long v, const float4* __restrict__ d4,
                                      const float4* __restrict__ B, long long n_block) {
    if (B != nullptr && v < n_block) {
        const float4 b0 = B[4 * v], b1 = B[4 * v + 1], b2 = B[4 * v + 2], b3 = B[4 * v + 3];
        return D4{b0.x * r.x + b0.y * r.y + b0.z * r.z + b0.w * r.w,
                  b1.x * r.x + b1.y * r.y + b1.z * r.z + b1.w * r.w,
                  b2.x * r.x + b2.y * r.y + b2.z * r.z + b2.w * r.w,
                  b3.x * r.x + b3.y * r.y + b3.z * r.z + b3.w * r.w};
    }
    const float4 d = d4[v];
    return D4{d.x > kJacobiFloor ? r.x / d.x : 0.0, d.y > kJacobiFloor ? r.y / d.y : 0.0,
              d.z > kJacobiFloor ? r.z / d.z : 0.0, d.w > kJacobiFloor ? r.w / d.w : 0.0};
}

// Segments: a batch of independent systems (the scenes of a batch).  With
// chunks (one int4 per CTA, built by the host: x = system, [y, z) = its
// parameter blocks for this CTA) every CTA works inside one system, and big
// systems get proportionally many CTAs; chunks == nullptr means a single
// system [0, nb) over a grid-stride loop.
__device__ __forceinline__ int seg_id(const int4* chunks) { return chunks ? chunks[blockIdx.x].x : 0; }

#define SEG_LOOP(v)                                                                      \
    long long lo_, hi_, step_;                                                            \
    if (chunks) {                                                                         \
        const int4 c_ = chunks[blockIdx.x];                                               \
        lo_ = (long long)c_.y + threadIdx.x; hi_ = c_.z; step_ = blockDim.x;              \
    } else {                                                                              \
        lo_ = (long long)blockIdx.x * blockDim.x + threadIdx.x; hi_ = nb;                 \
        step_ = (long long)gridDim.x * blockDim.x;                                        \
    }                                                                                     \
    for (long long v = lo_; v < hi_; v += step_)

__device__ __forceinline__ double dot4(const D4& a, const D4& b) {
    return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
}

__device__ __forceinline__ void store_bf16x4(__nv_bfloat16* y, long long v, float4 a) {
    __nv_bfloat162 lo = __floats2bfloat162_rn(a.x, a.y);
    __nv_bfloat162 hi = __floats2bfloat162_rn(a.z, a.w);
    uint2 u;
    u.x = *reinterpret_cast<unsigned*>(&lo);
    u.y = *reinterpret_cast<unsigned*>(&hi);
    reinterpret_cast<uint2*>(y)[v] = u;
}

// pxp (may be null): paired x / p records (two float4 each); p goes to the
// second half of record v.
__device__ __forceinline__ void store_p(float4* p32, __nv_bfloat16* p16, float4* pxp, long long v,
                                        const D4& p) {
    const float4 f = make_float4((float)p.x, (float)p.y, (float)p.z, (float)p.w);
    p32[v] = f;
    if (p16) store_bf16x4(p16, v, f);
    if (pxp) pxp[2 * v + 1] = f;
}

__global__ void __launch_bounds__(kVThreads) k_pcg_begin(long long nb, const int4* chunks,
                                                        const float4* __restrict__ g,
                                                        const float4* __restrict__ d4,
                                                        const float4* __restrict__ B, long long n_block,
                                                        double* delta, double* rho, double* p,
                                                        float4* p32, __nv_bfloat16* p16, float4* Ap,
                                                        PcgScalars* s, float4* pxp) {
    s += seg_id(chunks);
    double aR = 0.0, aRz = 0.0;
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    SEG_LOOP(v) {
        const float4 gg = g[v];
        const D4 r{-(double)gg.x, -(double)gg.y, -(double)gg.z, -(double)gg.w};
        const D4 z = precond(r, v, d4, B, n_block);
        st4(rho, v, r);
        st4(p, v, z);
        store_p(p32, p16, pxp, v, z);
        st4(delta, v, D4{0.0, 0.0, 0.0, 0.0});
        Ap[v] = zero;
        aR += dot4(r, r);
        aRz += dot4(r, z);
    }
    block_add_f64<kVThreads / 32>(aR, &s->acc_R);
    block_add_f64<kVThreads / 32>(aRz, &s->acc_rz);
}

__global__ void k_pcg_begin_fin(PcgScalars* s, int n_seg, int max_iter, int fixed, double eps_rel,
                                double stall) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_seg) return;
    s += i;
    s->R0 = s->acc_R;
    s->R_prev = s->acc_R;
    s->R = s->acc_R;
    s->rz = s->acc_rz;
    s->acc_R = 0.0;
    s->acc_rz = 0.0;
    s->pAp = 0.0;
    s->beta = 0.0;
    s->iter = 0;
    s->max_iter = max_iter;
    s->fixed = fixed;
    s->eps_rel = eps_rel;
    s->stall = stall;
    s->exit_reason = 0;
    s->done = 0;
    if (!(s->R0 > 0.0)) {            // b = 0: Delta = 0 is the solution
        s->done = 1;
        s->exit_reason = isfinite(s->R0) ? 1 : 4;
    } else if (max_iter <= 0) {
        s->done = 1;
    }
}

__global__ void __launch_bounds__(kVThreads) k_pcg_update(long long nb, const int4* chunks,
                                                         double* delta, double* rho,
                                                         const double* __restrict__ p,
                                                         const float4* __restrict__ Ap,
                                                         const float4* __restrict__ d4,
                                                         const float4* __restrict__ B,
                                                         long long n_block, PcgScalars* s) {
    s += seg_id(chunks);
    if (s->done) return;
    const double pAp = s->pAp;
    if (!(pAp > 0.0) || !isfinite(pAp)) return;
    const double alpha = s->rz / pAp;
    double aR = 0.0, aRz = 0.0;
    SEG_LOOP(v) {
        const D4 pv = ld4(p, v);
        const float4 av = Ap[v];
        D4 dv = ld4(delta, v), r = ld4(rho, v);
        dv.x = fma(alpha, pv.x, dv.x); dv.y = fma(alpha, pv.y, dv.y);
        dv.z = fma(alpha, pv.z, dv.z); dv.w = fma(alpha, pv.w, dv.w);
        r.x = fma(-alpha, (double)av.x, r.x); r.y = fma(-alpha, (double)av.y, r.y);
        r.z = fma(-alpha, (double)av.z, r.z); r.w = fma(-alpha, (double)av.w, r.w);
        st4(delta, v, dv);
        st4(rho, v, r);
        const D4 z = precond(r, v, d4, B, n_block);
        aR += dot4(r, r);
        aRz += dot4(r, z);
    }
    block_add_f64<kVThreads / 32>(aR, &s->acc_R);
    block_add_f64<kVThreads / 32>(aRz, &s->acc_rz);
}

__global__ void k_pcg_finish(PcgScalars* s, int n_seg) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_seg) return;
    s += i;
    if (s->done) return;
    const double pAp = s->pAp;
    if (!(pAp > 0.0) || !isfinite(pAp)) {
        s->done = 1;
        s->exit_reason = isfinite(pAp) ? 3 : 4;
        return;
    }
    s->iter += 1;
    const double R = s->acc_R, rz_new = s->acc_rz;
    if (!isfinite(R) || !isfinite(rz_new)) {
        s->done = 1;
        s->exit_reason = 4;
        return;
    }
    s->R = R;
    if (s->fixed) {
        if (s->iter >= s->max_iter) { s->done = 1; s->exit_reason = 0; }
    } else {
        if (R < s->eps_rel * s->eps_rel * s->R0) { s->done = 1; s->exit_reason = 1; }
        else if (R / s->R_prev > s->stall) { s->done = 1; s->exit_reason = 2; }
        else if (s->iter >= s->max_iter) { s->done = 1; s->exit_reason = 0; }
    }
    s->beta = s->rz != 0.0 ? rz_new / s->rz : 0.0;
    s->rz = rz_new;
    s->R_prev = R;
    s->acc_R = 0.0;
    s->acc_rz = 0.0;
    s->pAp = 0.0;
}

__global__ void __launch_bounds__(kVThreads) k_pcg_dir(long long nb, const int4* chunks,
                                                      const double* __restrict__ rho,
                                                      const float4* __restrict__ d4,
                                                      const float4* __restrict__ B, long long n_block,
                                                      double* p, float4* p32, __nv_bfloat16* p16,
                                                      float4* Ap, const PcgScalars* s, float4* pxp) {
    s += seg_id(chunks);
    if (s->done) return;
    const double beta = s->beta;
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    SEG_LOOP(v) {
        const D4 z = precond(ld4(rho, v), v, d4, B, n_block);
        D4 pv = ld4(p, v);
        pv.x = fma(beta, pv.x, z.x); pv.y = fma(beta, pv.y, z.y);
        pv.z = fma(beta, pv.z, z.z); pv.w = fma(beta, pv.w, z.w);
        st4(p, v, pv);
        store_p(p32, p16, pxp, v, pv);
        Ap[v] = zero;
    }
}

// Paired records: xp[v] = (x[v], p[v]) (p may be null: the p half is kept).
__global__ void __launch_bounds__(kVThreads) k_pair_pack(long long nb, const float4* __restrict__ x,
                                                        const float4* __restrict__ p, float4* xp) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < nb;
         v += (long long)gridDim.x * blockDim.x) {
        xp[2 * v] = x[v];
        if (p) xp[2 * v + 1] = p[v];
    }
}

// x_out = P(x + gamma Delta): the trial point is formed in FP64 and rounded
// once to the storage type(s).
__global__ void __launch_bounds__(kVThreads) k_trial(long long nb, const float4* x,
                                                    const double* __restrict__ delta, double gamma,
                                                    int project, float4* x_out,
                                                    __nv_bfloat16* x16) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < nb;
         v += (long long)gridDim.x * blockDim.x) {
        const float4 a = x[v];
        const D4 d = ld4(delta, v);
        float4 y = make_float4((float)fma(gamma, d.x, (double)a.x), (float)fma(gamma, d.y, (double)a.y),
                               (float)fma(gamma, d.z, (double)a.z), (float)fma(gamma, d.w, (double)a.w));
        if (project) {
            y.x = fminf(fmaxf(y.x, 0.0f), 1.0f);
            y.y = fminf(fmaxf(y.y, 0.0f), 1.0f);
            y.z = fminf(fmaxf(y.z, 0.0f), 1.0f);
            y.w = fmaxf(y.w, 0.0f);
        }
        if (x_out) x_out[v] = y;
        if (x16) store_bf16x4(x16, v, y);
    }
}

// Batched trial: segment y gets x_out = P(x + gamma[y] Delta) where mask[y]
// is set (mask == nullptr: every segment); other segments are left alone.
__global__ void __launch_bounds__(kVThreads) k_trial_seg(long long nb, const int4* chunks,
                                                        const float4* x,
                                                        const double* __restrict__ delta,
                                                        const double* __restrict__ gamma,
                                                        const int* __restrict__ mask, int project,
                                                        float4* x_out) {
    const int sg = seg_id(chunks);
    if (mask && !mask[sg]) return;
    const double g = gamma[sg];
    SEG_LOOP(v) {
        const float4 a = x[v];
        const D4 d = ld4(delta, v);
        float4 y = make_float4((float)fma(g, d.x, (double)a.x), (float)fma(g, d.y, (double)a.y),
                               (float)fma(g, d.z, (double)a.z), (float)fma(g, d.w, (double)a.w));
        if (project) {
            y.x = fminf(fmaxf(y.x, 0.0f), 1.0f);
            y.y = fminf(fmaxf(y.y, 0.0f), 1.0f);
            y.z = fminf(fmaxf(y.z, 0.0f), 1.0f);
            y.w = fmaxf(y.w, 0.0f);
        }
        x_out[v] = y;
    }
}

__global__ void __launch_bounds__(kVThreads) k_to_bf16(long long nb, const float4* __restrict__ x,
                                                      __nv_bfloat16* y) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < nb;
         v += (long long)gridDim.x * blockDim.x)
        store_bf16x4(y, v, x[v]);
}

__global__ void __launch_bounds__(kVThreads) k_to_f32(long long n, const double* __restrict__ a,
                                                     float* b) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}

// ------------------------------------------------------------- launchers

#define F4(p) reinterpret_cast<float4*>(p)
#define CF4(p) reinterpret_cast<const float4*>(p)

static dim3 seg_grid(long long nb, long long n_chunks, const int4* chunks) {
    return chunks ? dim3((unsigned)n_chunks, 1, 1) : dim3(vec_blocks(nb), 1, 1);
}

cudaError_t launch_pcg_begin_seg(long long n, int n_seg, const int4* chunks, long long n_chunks,
                                 const float* grad, const float* diag, double* delta, double* rho,
                                 double* p, float* p32, __nv_bfloat16* p16, float* Ap,
                                 PcgScalars* s, int max_iter, int fixed, double eps_rel,
                                 double stall, const float* blocks, long long n_block,
                                 cudaStream_t st, float* pxp) {
    const long long nb = n / 4;
    cudaError_t e = cudaMemsetAsync(s, 0, sizeof(PcgScalars) * (size_t)(n_seg > 0 ? n_seg : 1), st);
    if (e != cudaSuccess) return e;
    if (nb > 0) {
        k_pcg_begin<<<seg_grid(nb, n_chunks, chunks), kVThreads, 0, st>>>(
            nb, chunks, CF4(grad), CF4(diag), CF4(blocks), n_block, delta, rho, p, F4(p32), p16,
            F4(Ap), s, F4(pxp));
        count_launch();
    }
    const int ns = n_seg > 1 ? n_seg : 1;
    k_pcg_begin_fin<<<(ns + 31) / 32, 32, 0, st>>>(s, ns, max_iter, fixed, eps_rel, stall);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_pcg_begin(long long n, const float* grad, const float* diag, double* delta,
                             double* rho, double* p, float* p32, __nv_bfloat16* p16, float* Ap,
                             PcgScalars* s, int max_iter, int fixed, double eps_rel, double stall,
                             const float* blocks, long long n_block, cudaStream_t st, float* pxp) {
    return launch_pcg_begin_seg(n, 1, nullptr, 0, grad, diag, delta, rho, p, p32, p16, Ap, s,
                                max_iter, fixed, eps_rel, stall, blocks, n_block, st, pxp);
}

cudaError_t launch_pcg_update_seg(long long n, int n_seg, const int4* chunks, long long n_chunks,
                                  double* delta, double* rho, const double* p, const float* Ap,
                                  const float* diag, const float* blocks, long long n_block,
                                  PcgScalars* s, cudaStream_t st) {
    const long long nb = n / 4;
    if (nb > 0) {
        k_pcg_update<<<seg_grid(nb, n_chunks, chunks), kVThreads, 0, st>>>(
            nb, chunks, delta, rho, p, CF4(Ap), CF4(diag), CF4(blocks), n_block, s);
        count_launch();
    }
    return cudaGetLastError();
}

cudaError_t launch_pcg_update(long long n, double* delta, double* rho, const double* p,
                              const float* Ap, const float* diag, const float* blocks,
                              long long n_block, PcgScalars* s, cudaStream_t st) {
    return launch_pcg_update_seg(n, 1, nullptr, 0, delta, rho, p, Ap, diag, blocks, n_block, s,
                                 st);
}

cudaError_t launch_pcg_finish_seg(PcgScalars* s, int n_seg, cudaStream_t st) {
    const int ns = n_seg > 1 ? n_seg : 1;
    k_pcg_finish<<<(ns + 31) / 32, 32, 0, st>>>(s, ns);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_pcg_finish(PcgScalars* s, cudaStream_t st) { return launch_pcg_finish_seg(s, 1, st); }

cudaError_t launch_pcg_dir_seg(long long n, int n_seg, const int4* chunks, long long n_chunks,
                               const double* rho, const float* diag, const float* blocks,
                               long long n_block, double* p, float* p32, __nv_bfloat16* p16,
                               float* Ap, PcgScalars* s, cudaStream_t st, float* pxp) {
    const long long nb = n / 4;
    if (nb > 0) {
        k_pcg_dir<<<seg_grid(nb, n_chunks, chunks), kVThreads, 0, st>>>(
            nb, chunks, rho, CF4(diag), CF4(blocks), n_block, p, F4(p32), p16, F4(Ap), s, F4(pxp));
        count_launch();
    }
    return cudaGetLastError();
}

cudaError_t launch_pcg_dir(long long n, const double* rho, const float* diag, const float* blocks,
                           long long n_block, double* p, float* p32, __nv_bfloat16* p16, float* Ap,
                           PcgScalars* s, cudaStream_t st, float* pxp) {
    return launch_pcg_dir_seg(n, 1, nullptr, 0, rho, diag, blocks, n_block, p, p32, p16, Ap, s,
                              st, pxp);
}

cudaError_t launch_trial_seg(long long n, int n_seg, const int4* chunks, long long n_chunks,
                             const float* x, const double* delta, const double* gamma,
                             const int* mask, int project, float* x_out, cudaStream_t st) {
    const long long nb = n / 4;
    if (nb > 0) {
        k_trial_seg<<<seg_grid(nb, n_chunks, chunks), kVThreads, 0, st>>>(
            nb, chunks, CF4(x), delta, gamma, mask, project, F4(x_out));
        count_launch();
    }
    return cudaGetLastError();
}

cudaError_t launch_trial(long long n, const float* x, const double* delta, double gamma,
                         int project, float* x_out, __nv_bfloat16* x16_out, cudaStream_t st) {
    const long long nb = n / 4;
    if (nb > 0) {
        k_trial<<<vec_blocks(nb), kVThreads, 0, st>>>(nb, CF4(x), delta, gamma, project, F4(x_out),
                                                      x16_out);
        count_launch();
    }
    return cudaGetLastError();
}

cudaError_t launch_to_bf16(long long n, const float* x, __nv_bfloat16* y, cudaStream_t st) {
    const long long nb = n / 4;
    if (nb > 0) {
        k_to_bf16<<<vec_blocks(nb), kVThreads, 0, st>>>(nb, CF4(x), y);
        count_launch();
    }
    return cudaGetLastError();
}

cudaError_t launch_pair_pack(long long n, const float* x, const float* p, float* xp,
                             cudaStream_t st) {
    const long long nb = n / 4;
    if (nb > 0) {
        k_pair_pack<<<vec_blocks(nb), kVThreads, 0, st>>>(nb, CF4(x), CF4(p), F4(xp));
        count_launch();
    }
    return cudaGetLastError();
}

cudaError_t launch_to_f32(long long n, const double* a, float* b, cudaStream_t st) {
    if (n > 0) {
        k_to_f32<<<vec_blocks((n + 3) / 4), kVThreads, 0, st>>>(n, a, b);
        count_launch();
    }
    return cudaGetLastError();
}

}  // namespace perf

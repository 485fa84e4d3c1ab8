// k_pcg.cu -- vector work of Algorithm 2 (preconditioned conjugate gradients)
// and of the line search (Algorithm 3), fused so that each n-vector is read
// and written as few times as the recurrence allows (Section "Update step":
// the vector additions and inner products run in parallel on the GPU).
//
// Vectors are float32, handled one parameter block (4 values = one voxel or
// texel) per thread as float4; inner products accumulate in FP64.
//   begin : rho = b = -grad, z = M^-1 rho, p = z, Delta = 0, R0, rho^T z
//   update: Delta += alpha p, rho -= alpha A p, z = M^-1 rho, R, rho^T z
//   finish: exit test (R < eps^2 R0 or R / R_prev > stall, or a fixed count),
//           beta = rho'^T z' / rho^T z                               [1 thread]
//   dir   : p = z + beta p, A p = 0 for the next scatter
// M^-1 is Jacobi (z_j = rho_j / d_j, 0 where d_j = 0) or, where 4x4 blocks
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

__device__ __forceinline__ float4 precond(float4 r, long long v, const float4* __restrict__ d4,
                                          const float4* __restrict__ B, long long n_block) {
    if (B != nullptr && v < n_block) {
        const float4 b0 = B[4 * v], b1 = B[4 * v + 1], b2 = B[4 * v + 2], b3 = B[4 * v + 3];
        return make_float4(b0.x * r.x + b0.y * r.y + b0.z * r.z + b0.w * r.w,
                           b1.x * r.x + b1.y * r.y + b1.z * r.z + b1.w * r.w,
                           b2.x * r.x + b2.y * r.y + b2.z * r.z + b2.w * r.w,
                           b3.x * r.x + b3.y * r.y + b3.z * r.z + b3.w * r.w);
    }
    const float4 d = d4[v];
    return make_float4(d.x > 0.0f ? r.x / d.x : 0.0f, d.y > 0.0f ? r.y / d.y : 0.0f,
                       d.z > 0.0f ? r.z / d.z : 0.0f, d.w > 0.0f ? r.w / d.w : 0.0f);
}

__device__ __forceinline__ double dot4(float4 a, float4 b) {
    return (double)a.x * b.x + (double)a.y * b.y + (double)a.z * b.z + (double)a.w * b.w;
}

__device__ __forceinline__ void store_bf16x4(__nv_bfloat16* y, long long v, float4 a) {
    __nv_bfloat162 lo = __floats2bfloat162_rn(a.x, a.y);
    __nv_bfloat162 hi = __floats2bfloat162_rn(a.z, a.w);
    uint2 u;
    u.x = *reinterpret_cast<unsigned*>(&lo);
    u.y = *reinterpret_cast<unsigned*>(&hi);
    reinterpret_cast<uint2*>(y)[v] = u;
}

__global__ void __launch_bounds__(kVThreads) k_pcg_begin(long long nb, const float4* __restrict__ g,
                                                        const float4* __restrict__ d4,
                                                        const float4* __restrict__ B, long long n_block,
                                                        float4* delta, float4* rho, float4* p,
                                                        __nv_bfloat16* p16, float4* Ap,
                                                        PcgScalars* s) {
    double aR = 0.0, aRz = 0.0;
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < nb;
         v += (long long)gridDim.x * blockDim.x) {
        const float4 gg = g[v];
        const float4 r = make_float4(-gg.x, -gg.y, -gg.z, -gg.w);
        const float4 z = precond(r, v, d4, B, n_block);
        rho[v] = r;
        p[v] = z;
        if (p16) store_bf16x4(p16, v, z);
        delta[v] = zero;
        Ap[v] = zero;
        aR += dot4(r, r);
        aRz += dot4(r, z);
    }
    block_add_f64<kVThreads / 32>(aR, &s->acc_R);
    block_add_f64<kVThreads / 32>(aRz, &s->acc_rz);
}

__global__ void k_pcg_begin_fin(PcgScalars* s, int max_iter, int fixed, double eps_rel, double stall) {
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

__global__ void __launch_bounds__(kVThreads) k_pcg_update(long long nb, float4* delta, float4* rho,
                                                         const float4* __restrict__ p,
                                                         const float4* __restrict__ Ap,
                                                         const float4* __restrict__ d4,
                                                         const float4* __restrict__ B,
                                                         long long n_block, PcgScalars* s) {
    if (s->done) return;
    const double pAp = s->pAp;
    if (!(pAp > 0.0) || !isfinite(pAp)) return;
    const float alpha = (float)(s->rz / pAp);
    double aR = 0.0, aRz = 0.0;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < nb;
         v += (long long)gridDim.x * blockDim.x) {
        const float4 pv = p[v], av = Ap[v];
        float4 dv = delta[v], r = rho[v];
        dv.x = fmaf(alpha, pv.x, dv.x); dv.y = fmaf(alpha, pv.y, dv.y);
        dv.z = fmaf(alpha, pv.z, dv.z); dv.w = fmaf(alpha, pv.w, dv.w);
        r.x = fmaf(-alpha, av.x, r.x); r.y = fmaf(-alpha, av.y, r.y);
        r.z = fmaf(-alpha, av.z, r.z); r.w = fmaf(-alpha, av.w, r.w);
        delta[v] = dv;
        rho[v] = r;
        const float4 z = precond(r, v, d4, B, n_block);
        aR += dot4(r, r);
        aRz += dot4(r, z);
    }
    block_add_f64<kVThreads / 32>(aR, &s->acc_R);
    block_add_f64<kVThreads / 32>(aRz, &s->acc_rz);
}

__global__ void k_pcg_finish(PcgScalars* s) {
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

__global__ void __launch_bounds__(kVThreads) k_pcg_dir(long long nb, const float4* __restrict__ rho,
                                                      const float4* __restrict__ d4,
                                                      const float4* __restrict__ B, long long n_block,
                                                      float4* p, __nv_bfloat16* p16, float4* Ap,
                                                      const PcgScalars* s) {
    if (s->done) return;
    const float beta = (float)s->beta;
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < nb;
         v += (long long)gridDim.x * blockDim.x) {
        const float4 z = precond(rho[v], v, d4, B, n_block);
        float4 pv = p[v];
        pv.x = fmaf(beta, pv.x, z.x); pv.y = fmaf(beta, pv.y, z.y);
        pv.z = fmaf(beta, pv.z, z.z); pv.w = fmaf(beta, pv.w, z.w);
        p[v] = pv;
        if (p16) store_bf16x4(p16, v, pv);
        Ap[v] = zero;
    }
}

__global__ void __launch_bounds__(kVThreads) k_trial(long long nb, const float4* __restrict__ x,
                                                    const float4* __restrict__ delta, float gamma,
                                                    int project, float4* x_out,
                                                    __nv_bfloat16* x16) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < nb;
         v += (long long)gridDim.x * blockDim.x) {
        const float4 a = x[v], d = delta[v];
        float4 y = make_float4(fmaf(gamma, d.x, a.x), fmaf(gamma, d.y, a.y),
                               fmaf(gamma, d.z, a.z), fmaf(gamma, d.w, a.w));
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

__global__ void __launch_bounds__(kVThreads) k_to_bf16(long long nb, const float4* __restrict__ x,
                                                      __nv_bfloat16* y) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < nb;
         v += (long long)gridDim.x * blockDim.x)
        store_bf16x4(y, v, x[v]);
}

// ------------------------------------------------------------- launchers

#define F4(p) reinterpret_cast<float4*>(p)
#define CF4(p) reinterpret_cast<const float4*>(p)

cudaError_t launch_pcg_begin(long long n, const float* grad, const float* diag, float* delta,
                             float* rho, float* p, __nv_bfloat16* p16, float* Ap, PcgScalars* s,
                             int max_iter, int fixed, double eps_rel, double stall,
                             const float* blocks, long long n_block, cudaStream_t st) {
    const long long nb = n / 4;
    cudaError_t e = cudaMemsetAsync(s, 0, sizeof(PcgScalars), st);
    if (e != cudaSuccess) return e;
    if (nb > 0)
        k_pcg_begin<<<vec_blocks(nb), kVThreads, 0, st>>>(nb, CF4(grad), CF4(diag), CF4(blocks),
                                                          n_block, F4(delta), F4(rho), F4(p), p16,
                                                          F4(Ap), s);
    k_pcg_begin_fin<<<1, 1, 0, st>>>(s, max_iter, fixed, eps_rel, stall);
    count_launch(nb > 0 ? 2 : 1);
    return cudaGetLastError();
}

cudaError_t launch_pcg_update(long long n, float* delta, float* rho, const float* p,
                              const float* Ap, const float* diag, const float* blocks,
                              long long n_block, PcgScalars* s, cudaStream_t st) {
    const long long nb = n / 4;
    if (nb > 0)
        k_pcg_update<<<vec_blocks(nb), kVThreads, 0, st>>>(nb, F4(delta), F4(rho), CF4(p), CF4(Ap),
                                                           CF4(diag), CF4(blocks), n_block, s);
    if (nb > 0) count_launch();
    return cudaGetLastError();
}

cudaError_t launch_pcg_finish(PcgScalars* s, cudaStream_t st) {
    k_pcg_finish<<<1, 1, 0, st>>>(s);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_pcg_dir(long long n, const float* rho, const float* diag, const float* blocks,
                           long long n_block, float* p, __nv_bfloat16* p16, float* Ap,
                           PcgScalars* s, cudaStream_t st) {
    const long long nb = n / 4;
    if (nb > 0)
        k_pcg_dir<<<vec_blocks(nb), kVThreads, 0, st>>>(nb, CF4(rho), CF4(diag), CF4(blocks),
                                                        n_block, F4(p), p16, F4(Ap), s);
    if (nb > 0) count_launch();
    return cudaGetLastError();
}

cudaError_t launch_trial(long long n, const float* x, const float* delta, float gamma, int project,
                         float* x_out, __nv_bfloat16* x16_out, cudaStream_t st) {
    const long long nb = n / 4;
    if (nb > 0)
        k_trial<<<vec_blocks(nb), kVThreads, 0, st>>>(nb, CF4(x), CF4(delta), gamma, project,
                                                      F4(x_out), x16_out);
    if (nb > 0) count_launch();
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

}  // namespace perf

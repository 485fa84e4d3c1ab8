// k_pcg.cu -- vector work of Algorithm 2 (preconditioned conjugate gradients)
// and of the line search (Algorithm 3), fused so that each n-vector is read
// and written as few times as the recurrence allows (Section "Update step":
// the vector additions and inner products run in parallel on the GPU).
//
// The CG recurrence vectors Delta, rho and p are FP32; the inner products
// rho^T rho and rho^T z are accumulated per thread as compensated FP32 sums
// (TwoSum: an unevaluated hi + lo pair) and reduced across threads and CTAs
// in FP64, and p^T A p arrives in FP64 from the ray march.  On GB300 FP64
// arithmetic runs at about 1/64 of the FP32 rate, so FP64 vectors (and the
// FP64 divisions of z = rho / d) made these kernels ALU-bound at a quarter of
// the HBM bandwidth; FP32 storage halves their bytes.  p is the array the
// next ray march gathers (and, in BF16 scenes, is also written as BF16).
// One thread handles one parameter block (4 values = one voxel or texel).
//   begin : rho = b = -grad, z = M^-1 rho, p = z, Delta = 0, A p = 0, R0, rho^T z
//   update: Delta += alpha p, rho -= alpha A p, A p = 0, z = M^-1 rho, R, rho^T z
//   finish: exit test (R < eps^2 R0 or R / R_prev > stall, or a fixed count),
//           beta = rho'^T z' / rho^T z                               [1 thread]
//   dir   : p = z + beta p
// Bytes per parameter and iteration: update 20 read + 12 written, dir 12
// read + 4 written (48; BF16 scenes write 2 more, paired records 4 more).
// M^-1 is Jacobi (z_j = rho_j / d_j, 0 where d_j <= 1e-30) or, where 4x4 blocks
// are given for the grid voxels, z_v = P_v rho_v per voxel.
#include <cuda_bf16.h>
#include "perf_kernels.h"

namespace perf {

unsigned long long g_launches = 0;

constexpr int kVThreads = 256;

// CTAs of a grid-stride vector kernel: enough to cover nblk blocks, at most
// 8 per SM of the current device (queried per call: the device may change).
static int vec_blocks(long long nblk) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        sms <= 0)
        sms = 1;
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

__device__ __forceinline__ float4 precond(const float4& r, long long v, const float4* __restrict__ d4,
                                          const float4* __restrict__ B, long long n_block) {
    if (B != nullptr && v < n_block) {
        const float4 b0 = B[4 * v], b1 = B[4 * v + 1], b2 = B[4 * v + 2], b3 = B[4 * v + 3];
        return make_float4(b0.x * r.x + b0.y * r.y + b0.z * r.z + b0.w * r.w,
                           b1.x * r.x + b1.y * r.y + b1.z * r.z + b1.w * r.w,
                           b2.x * r.x + b2.y * r.y + b2.z * r.z + b2.w * r.w,
                           b3.x * r.x + b3.y * r.y + b3.z * r.z + b3.w * r.w);
    }
    const float4 d = d4[v];
    return make_float4(d.x > kJacobiFloor ? r.x / d.x : 0.0f, d.y > kJacobiFloor ? r.y / d.y : 0.0f,
                       d.z > kJacobiFloor ? r.z / d.z : 0.0f, d.w > kJacobiFloor ? r.w / d.w : 0.0f);
}

// Compensated FP32 running sum (Knuth's TwoSum, explicit round-to-nearest
// operations so nothing is reassociated): the value is hi + lo.
struct Acc2 {
    float hi = 0.0f, lo = 0.0f;
    __device__ __forceinline__ void add(float v) {
        const float s = __fadd_rn(hi, v);
        const float bv = __fsub_rn(s, hi);
        const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bv)), __fsub_rn(v, bv));
        hi = s;
        lo = __fadd_rn(lo, e);
    }
    __device__ __forceinline__ void add4(const float4& a, const float4& b) {
        add(__fmul_rn(a.x, b.x));
        add(__fmul_rn(a.y, b.y));
        add(__fmul_rn(a.z, b.z));
        add(__fmul_rn(a.w, b.w));
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

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

__device__ __forceinline__ void store_bf16x4(__nv_bfloat16* y, long long v, float4 a) {
    __nv_bfloat162 lo = __floats2bfloat162_rn(a.x, a.y);
    __nv_bfloat162 hi = __floats2bfloat162_rn(a.z, a.w);
    uint2 u;
    u.x = *reinterpret_cast<unsigned*>(&lo);
    u.y = *reinterpret_cast<unsigned*>(&hi);
    reinterpret_cast<uint2*>(y)[v] = u;
}

// p and its copies for the gathers: p16 (BF16 scenes) and pxp (paired x / p
// records, two float4 each; p goes to the second half of record v); either
// may be null.
__device__ __forceinline__ void store_p(float4* p, __nv_bfloat16* p16, float4* pxp, long long v,
                                        const float4& f) {
    p[v] = f;
    if (p16) store_bf16x4(p16, v, f);
    if (pxp) pxp[2 * v + 1] = f;
}

__global__ void __launch_bounds__(kVThreads) k_pcg_begin(long long nb, const int4* chunks,
                                                        const float4* __restrict__ g,
                                                        const float4* __restrict__ d4,
                                                        const float4* __restrict__ B, long long n_block,
                                                        float4* delta, float4* rho, float4* p,
                                                        __nv_bfloat16* p16, float4* Ap,
                                                        PcgScalars* s, float4* pxp) {
    s += seg_id(chunks);
    Acc2 aR, aRz;
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    SEG_LOOP(v) {
        const float4 gg = g[v];
        const float4 r = make_float4(-gg.x, -gg.y, -gg.z, -gg.w);
        const float4 z = precond(r, v, d4, B, n_block);
        rho[v] = r;
        store_p(p, p16, pxp, v, z);
        delta[v] = zero;
        Ap[v] = zero;
        aR.add4(r, r);
        aRz.add4(r, z);
    }
    block_add_f64<kVThreads / 32>(aR.value(), &s->acc_R);
    block_add_f64<kVThreads / 32>(aRz.value(), &s->acc_rz);
}

__global__ void k_pcg_begin_fin(PcgScalars* s, int n_seg, int max_iter, int fixed, double eps_rel,
                                double stall, double* hist, long long hist_cap) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_seg) return;
    s += i;
    s->hist = n_seg == 1 ? hist : nullptr;
    s->hist_cap = n_seg == 1 ? hist_cap : 0;
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
                                                         float4* delta, float4* rho,
                                                         const float4* __restrict__ p,
                                                         float4* Ap,
                                                         const float4* __restrict__ d4,
                                                         const float4* __restrict__ B,
                                                         long long n_block, PcgScalars* s) {
    s += seg_id(chunks);
    if (s->done) return;
    const double pAp = s->pAp;
    if (!(pAp > 0.0) || !isfinite(pAp)) return;
    const float alpha = (float)(s->rz / pAp);
    Acc2 aR, aRz;
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    SEG_LOOP(v) {
        const float4 pv = p[v];
        const float4 av = Ap[v];
        float4 dv = delta[v], r = rho[v];
        dv.x = fmaf(alpha, pv.x, dv.x); dv.y = fmaf(alpha, pv.y, dv.y);
        dv.z = fmaf(alpha, pv.z, dv.z); dv.w = fmaf(alpha, pv.w, dv.w);
        r.x = fmaf(-alpha, av.x, r.x); r.y = fmaf(-alpha, av.y, r.y);
        r.z = fmaf(-alpha, av.z, r.z); r.w = fmaf(-alpha, av.w, r.w);
        delta[v] = dv;
        rho[v] = r;
        Ap[v] = zero;             // the next scatter accumulates into it
        const float4 z = precond(r, v, d4, B, n_block);
        aR.add4(r, r);
        aRz.add4(r, z);
    }
    block_add_f64<kVThreads / 32>(aR.value(), &s->acc_R);
    block_add_f64<kVThreads / 32>(aRz.value(), &s->acc_rz);
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
    if (s->hist && s->iter <= s->hist_cap) s->hist[s->iter - 1] = R;
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
                                                      const float4* __restrict__ rho,
                                                      const float4* __restrict__ d4,
                                                      const float4* __restrict__ B, long long n_block,
                                                      float4* p, __nv_bfloat16* p16,
                                                      const PcgScalars* s, float4* pxp) {
    s += seg_id(chunks);
    if (s->done) return;
    const float beta = (float)s->beta;
    SEG_LOOP(v) {
        const float4 z = precond(rho[v], v, d4, B, n_block);
        float4 pv = p[v];
        pv.x = fmaf(beta, pv.x, z.x); pv.y = fmaf(beta, pv.y, z.y);
        pv.z = fmaf(beta, pv.z, z.z); pv.w = fmaf(beta, pv.w, z.w);
        store_p(p, p16, pxp, v, pv);
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

// Block of Delta that holds canonical parameter block u of a scene whose
// PCG vectors are in the block order lay (x = G, y = s, z = ys, w = zs; see
// LayoutKey): the grid's blocks are permuted, the texels' are not.
__device__ __forceinline__ long long lay_block(long long u, int4 lay) {
    const long long G = lay.x;
    if (lay.y == 0 || u >= G * G * G) return u;
    const int ui = (int)u, g = lay.x;
    const int x = ui % g, yz = ui / g;
    const int y = yz % g, z = yz / g;
    const LayoutKey k{lay.y, (1 << lay.y) - 1, lay.z, lay.w};
    return k.key(x, y, z);
}

// x_out = P(x + gamma Delta): the trial point is formed in FP64 (one FMA per
// value) and rounded once to the storage type(s).  Delta in the block order
// lay (x canonical).
__global__ void __launch_bounds__(kVThreads) k_trial(long long nb, const float4* x,
                                                    const float4* __restrict__ delta, double gamma,
                                                    int project, float4* x_out,
                                                    __nv_bfloat16* x16, int4 lay) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < nb;
         v += (long long)gridDim.x * blockDim.x) {
        const float4 a = x[v];
        const float4 d = delta[lay_block(v, lay)];
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
// lay (may be null): per segment its block order and first block (lay[y],
// base[y]) -- Delta of that segment is in that order.
__global__ void __launch_bounds__(kVThreads) k_trial_seg(long long nb, const int4* chunks,
                                                        const float4* x,
                                                        const float4* __restrict__ delta,
                                                        const double* __restrict__ gamma,
                                                        const int* __restrict__ mask, int project,
                                                        float4* x_out, const int4* __restrict__ lay,
                                                        const long long* __restrict__ base) {
    const int sg = seg_id(chunks);
    if (mask && !mask[sg]) return;
    const double g = gamma[sg];
    const int4 ly = lay ? lay[sg] : make_int4(0, 0, 0, 0);
    const long long b0 = lay ? base[sg] : 0;
    SEG_LOOP(v) {
        const float4 a = x[v];
        const float4 d = delta[ly.y ? b0 + lay_block(v - b0, ly) : v];
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

// One Adam step (Kingma & Ba 2015) on the parameters from the gradient g of
// the objective, followed by the projection: m = b1 m + (1 - b1) g,
// v = b2 v + (1 - b2) g^2, x = P(x - lr (m / c1) / (sqrt(v / c2) + eps)) with
// the bias corrections c1 = 1 - b1^t, c2 = 1 - b2^t.  The first-order
// comparator of the Gauss-Newton step (the paper's Fig. 1 contrasts them).
__global__ void __launch_bounds__(kVThreads) k_adam(long long nb, float4* x, const float4* __restrict__ g,
                                                   float4* m, float4* v, float b1, float b2,
                                                   float lr, float eps, float c1, float c2,
                                                   int project) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nb;
         i += (long long)gridDim.x * blockDim.x) {
        const float4 gi = g[i];
        float4 mi = m[i], vi = v[i], xi = x[i];
        float* mp = &mi.x;
        float* vp = &vi.x;
        float* xp = &xi.x;
        const float* gp = &gi.x;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            mp[c] = fmaf(b1, mp[c], (1.0f - b1) * gp[c]);
            vp[c] = fmaf(b2, vp[c], (1.0f - b2) * gp[c] * gp[c]);
            xp[c] -= lr * (mp[c] / c1) / (sqrtf(vp[c] / c2) + eps);
        }
        if (project) {
            xi.x = fminf(fmaxf(xi.x, 0.0f), 1.0f);
            xi.y = fminf(fmaxf(xi.y, 0.0f), 1.0f);
            xi.z = fminf(fmaxf(xi.z, 0.0f), 1.0f);
            xi.w = fmaxf(xi.w, 0.0f);
        }
        m[i] = mi;
        v[i] = vi;
        x[i] = xi;
    }
}

// ------------------------------------------------------------- launchers

#define F4(p) reinterpret_cast<float4*>(p)
#define CF4(p) reinterpret_cast<const float4*>(p)

static dim3 seg_grid(long long nb, long long n_chunks, const int4* chunks) {
    return chunks ? dim3((unsigned)n_chunks, 1, 1) : dim3(vec_blocks(nb), 1, 1);
}

static cudaError_t pcg_begin_impl(long long n, int n_seg, const int4* chunks, long long n_chunks,
                                  const float* grad, const float* diag, float* delta, float* rho,
                                  float* p, __nv_bfloat16* p16, float* Ap, PcgScalars* s,
                                  int max_iter, int fixed, double eps_rel, double stall,
                                  const float* blocks, long long n_block, cudaStream_t st,
                                  float* pxp, double* hist, long long hist_cap) {
    const long long nb = n / 4;
    cudaError_t e = cudaMemsetAsync(s, 0, sizeof(PcgScalars) * (size_t)(n_seg > 0 ? n_seg : 1), st);
    if (e != cudaSuccess) return e;
    if (nb > 0) {
        k_pcg_begin<<<seg_grid(nb, n_chunks, chunks), kVThreads, 0, st>>>(
            nb, chunks, CF4(grad), CF4(diag), CF4(blocks), n_block, F4(delta), F4(rho), F4(p), p16,
            F4(Ap), s, F4(pxp));
        count_launch();
    }
    const int ns = n_seg > 1 ? n_seg : 1;
    k_pcg_begin_fin<<<(ns + 31) / 32, 32, 0, st>>>(s, ns, max_iter, fixed, eps_rel, stall, hist,
                                                   hist_cap);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_pcg_begin_seg(long long n, int n_seg, const int4* chunks, long long n_chunks,
                                 const float* grad, const float* diag, float* delta, float* rho,
                                 float* p, __nv_bfloat16* p16, float* Ap, PcgScalars* s,
                                 int max_iter, int fixed, double eps_rel, double stall,
                                 const float* blocks, long long n_block, cudaStream_t st,
                                 float* pxp) {
    return pcg_begin_impl(n, n_seg, chunks, n_chunks, grad, diag, delta, rho, p, p16, Ap, s,
                          max_iter, fixed, eps_rel, stall, blocks, n_block, st, pxp, nullptr, 0);
}

cudaError_t launch_pcg_begin(long long n, const float* grad, const float* diag, float* delta,
                             float* rho, float* p, __nv_bfloat16* p16, float* Ap, PcgScalars* s,
                             int max_iter, int fixed, double eps_rel, double stall,
                             const float* blocks, long long n_block, cudaStream_t st, float* pxp,
                             double* hist, long long hist_cap) {
    return pcg_begin_impl(n, 1, nullptr, 0, grad, diag, delta, rho, p, p16, Ap, s, max_iter,
                          fixed, eps_rel, stall, blocks, n_block, st, pxp, hist, hist_cap);
}

cudaError_t launch_pcg_update_seg(long long n, int n_seg, const int4* chunks, long long n_chunks,
                                  float* delta, float* rho, const float* p, float* Ap,
                                  const float* diag, const float* blocks, long long n_block,
                                  PcgScalars* s, cudaStream_t st) {
    const long long nb = n / 4;
    if (nb > 0) {
        k_pcg_update<<<seg_grid(nb, n_chunks, chunks), kVThreads, 0, st>>>(
            nb, chunks, F4(delta), F4(rho), CF4(p), F4(Ap), CF4(diag), CF4(blocks), n_block, s);
        count_launch();
    }
    return cudaGetLastError();
}

cudaError_t launch_pcg_update(long long n, float* delta, float* rho, const float* p, float* Ap,
                              const float* diag, const float* blocks, long long n_block,
                              PcgScalars* s, cudaStream_t st) {
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
                               const float* rho, const float* diag, const float* blocks,
                               long long n_block, float* p, __nv_bfloat16* p16, PcgScalars* s,
                               cudaStream_t st, float* pxp) {
    const long long nb = n / 4;
    if (nb > 0) {
        k_pcg_dir<<<seg_grid(nb, n_chunks, chunks), kVThreads, 0, st>>>(
            nb, chunks, CF4(rho), CF4(diag), CF4(blocks), n_block, F4(p), p16, s, F4(pxp));
        count_launch();
    }
    return cudaGetLastError();
}

cudaError_t launch_pcg_dir(long long n, const float* rho, const float* diag, const float* blocks,
                           long long n_block, float* p, __nv_bfloat16* p16, PcgScalars* s,
                           cudaStream_t st, float* pxp) {
    return launch_pcg_dir_seg(n, 1, nullptr, 0, rho, diag, blocks, n_block, p, p16, s, st, pxp);
}

cudaError_t launch_trial_seg(long long n, int n_seg, const int4* chunks, long long n_chunks,
                             const float* x, const float* delta, const double* gamma,
                             const int* mask, int project, float* x_out, cudaStream_t st,
                             const int4* lay, const long long* base) {
    const long long nb = n / 4;
    if (nb > 0) {
        k_trial_seg<<<seg_grid(nb, n_chunks, chunks), kVThreads, 0, st>>>(
            nb, chunks, CF4(x), CF4(delta), gamma, mask, project, F4(x_out), lay, base);
        count_launch();
    }
    return cudaGetLastError();
}

cudaError_t launch_trial(long long n, const float* x, const float* delta, double gamma,
                         int project, float* x_out, __nv_bfloat16* x16_out, cudaStream_t st,
                         int4 lay) {
    const long long nb = n / 4;
    if (nb > 0) {
        k_trial<<<vec_blocks(nb), kVThreads, 0, st>>>(nb, CF4(x), CF4(delta), gamma, project, F4(x_out),
                                                      x16_out, lay);
        count_launch();
    }
    return cudaGetLastError();
}

cudaError_t launch_adam(long long n, float* x, const float* g, float* m, float* v, float b1,
                        float b2, float lr, float eps, float c1, float c2, int project,
                        cudaStream_t st) {
    const long long nb = n / 4;
    if (nb > 0) {
        k_adam<<<vec_blocks(nb), kVThreads, 0, st>>>(nb, F4(x), CF4(g), F4(m), F4(v), b1, b2, lr,
                                                     eps, c1, c2, project);
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

}  // namespace perf

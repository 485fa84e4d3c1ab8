// k_lpc.cu -- kernels of the learned block preconditioner for Algorithm 2.
//
// A 3D convolutional network over the voxel grid predicts, per voxel v, a
// symmetric positive definite 4x4 block Q_v = L_v L_v^T + eps I acting on the
// Jacobi-scaled parameters: the preconditioner is
//     P_v = D_v^{-1/2} Q_v D_v^{-1/2},   D_v = diag(J^T J) restricted to v,
// so Q_v = I is exactly the Jacobi preconditioner of Section
// "Preconditioner".  The net: 4 layers of 3x3x3 convolution, 16 channels
// (inputs and the 10 head outputs padded to 16), ReLU between layers,
// activations channels-last [voxel][16] in bfloat16, FP32 accumulation.
// The forward convolution (k_conv_tc.cu) runs on the tcgen05 tensor cores
// with TMA-staged halos; the backward pass reuses it with flipped,
// transposed weights for the data gradient.  The weight gradient (here) is a
// per-tap GEMM over voxels with M = N = 16 -- below the smallest tcgen05 tile
// -- on warp-level mma.sync (bf16 inputs, fp32 accumulators), reduced across
// warps with atomics.  Training minimises, over
// logged probe pairs (xi, a_hat = D^{-1/2} A D^{-1/2} xi), the relative error
// sum_v |Q_v a_hat_v - xi_v|^2 / sum |xi|^2 with Adam.
#include <cuda_bf16.h>
#include <cstdint>

#include "perf_kernels.h"

namespace perf {

constexpr int kC = 16;        // channels (padded)
constexpr int kTaps = 27;
constexpr int kLThreads = 128;

__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&h);
}

__device__ __forceinline__ uint32_t pack_raw(__nv_bfloat16 lo, __nv_bfloat16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// Linear voxel index of v's neighbour at tap (dz, dy, dx) in {-1,0,1}^3, or
// -1 (32-bit index arithmetic: a grid has fewer than 2^31 voxels).
__device__ __forceinline__ long long nbr(long long v, int G, int tap) {
    if (v < 0) return -1;
    const int dx = tap % 3 - 1, dy = (tap / 3) % 3 - 1, dz = tap / 9 - 1;
    const unsigned uv = (unsigned)v, ug = (unsigned)G;
    const unsigned q = uv / ug;
    const int x = (int)(uv - q * ug);
    const unsigned z = q / ug;
    const int y = (int)(q - z * ug);
    const int xx = x + dx, yy = y + dy, zz = (int)z + dz;
    if (xx < 0 || yy < 0 || zz < 0 || xx >= G || yy >= G || zz >= G) return -1;
    return ((long long)zz * G + yy) * G + xx;
}

// dW[tap][co][ci] += sum_v gpre[v][co] in[nbr(v,tap)][ci]   (FP32 accumulate)
// grid.y = tap; one warp reduces 16-voxel chunks with mma (M = co, N = ci,
// K = voxels) and adds its 16x16 partial with atomics.
__global__ void __launch_bounds__(kLThreads) k_conv_bwd_w(const __nv_bfloat16* __restrict__ in,
                                                         const __nv_bfloat16* __restrict__ gpre,
                                                         float* __restrict__ dW,
                                                         float* __restrict__ dB, int G) {
    const int tap = blockIdx.y;
    const long long V = (long long)G * G * G;
    const long long n_chunks = (V + 15) / 16;
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
    float bacc[2] = {0.f, 0.f};
    const __nv_bfloat16 z = __float2bfloat16(0.f);
    for (long long c = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < n_chunks;
         c += nwarps) {
        const long long k0 = c * 16 + 2 * t, k1 = k0 + 1, k8 = k0 + 8, k9 = k0 + 9;
        // A[m = co][k = voxel] = gpre[voxel][co]
        auto ga = [&](long long v, int co) { return v < V ? gpre[v * kC + co] : z; };
        const uint32_t a0 = pack_raw(ga(k0, g), ga(k1, g));
        const uint32_t a1 = pack_raw(ga(k0, g + 8), ga(k1, g + 8));
        const uint32_t a2 = pack_raw(ga(k8, g), ga(k9, g));
        const uint32_t a3 = pack_raw(ga(k8, g + 8), ga(k9, g + 8));
        // B[k = voxel][n = ci] = in[nbr(voxel, tap)][ci]
        const long long m0 = k0 < V ? nbr(k0, G, tap) : -1, m1 = k1 < V ? nbr(k1, G, tap) : -1;
        const long long m8 = k8 < V ? nbr(k8, G, tap) : -1, m9 = k9 < V ? nbr(k9, G, tap) : -1;
        auto gb = [&](long long m, int ci) { return m >= 0 ? in[m * kC + ci] : z; };
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
            const int ci = nt * 8 + g;
            mma_bf16(acc[nt], a0, a1, a2, a3, pack_raw(gb(m0, ci), gb(m1, ci)),
                     pack_raw(gb(m8, ci), gb(m9, ci)));
        }
        if (tap == 13 && dB) {   // the centre tap also reduces the bias gradient
            if (t == 0) {
                for (int q = 0; q < 16; ++q) {
                    const long long v = c * 16 + q;
                    if (v < V) {
                        bacc[0] += __bfloat162float(gpre[v * kC + g]);
                        bacc[1] += __bfloat162float(gpre[v * kC + g + 8]);
                    }
                }
            }
        }
    }
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
        const int ci = nt * 8 + 2 * t;
        float* w0 = dW + ((long long)tap * kC + g) * kC + ci;        // co = g
        float* w1 = dW + ((long long)tap * kC + g + 8) * kC + ci;    // co = g + 8
        atomicAdd(w0, acc[nt][0]);
        atomicAdd(w0 + 1, acc[nt][1]);
        atomicAdd(w1, acc[nt][2]);
        atomicAdd(w1 + 1, acc[nt][3]);
    }
    if (tap == 13 && dB && t == 0) {
        atomicAdd(dB + g, bacc[0]);
        atomicAdd(dB + g + 8, bacc[1]);
    }
}

// Weights for the data gradient: Wt[tap'][ci][co] = W[26 - tap'][co][ci]
// (flipped taps, input/output channels exchanged).
__global__ void k_conv_flip(const __nv_bfloat16* __restrict__ W, __nv_bfloat16* __restrict__ Wt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kTaps * kC * kC) return;
    const int ci = i % kC, co = (i / kC) % kC, tap = i / (kC * kC);
    Wt[((26 - tap) * kC + ci) * kC + co] = W[i];
}

// g[v][c] *= (act[v][c] > 0): ReLU backward through the stored activation.
__global__ void k_relu_bwd(__nv_bfloat16* __restrict__ g, const __nv_bfloat16* __restrict__ act,
                           long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        if (!(__bfloat162float(act[i]) > 0.0f)) g[i] = __float2bfloat16(0.0f);
}

// ---------------------------------------------------------------- head
// o[0..3]: diagonal of L through softplus; o[4..9]: L10, L20, L21, L30, L31, L32.
__device__ __forceinline__ float softplus(float x) { return x > 20.f ? x : log1pf(expf(x)); }
__device__ __forceinline__ float sigm(float x) { return 1.0f / (1.0f + expf(-x)); }

constexpr float kQeps = 1e-3f;

__device__ __forceinline__ void head_L(const __nv_bfloat16* o, float (&L)[4][4], float (&od)[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) L[i][j] = 0.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        od[i] = __bfloat162float(o[i]);
        L[i][i] = softplus(od[i]);
    }
    L[1][0] = __bfloat162float(o[4]);
    L[2][0] = __bfloat162float(o[5]);
    L[2][1] = __bfloat162float(o[6]);
    L[3][0] = __bfloat162float(o[7]);
    L[3][1] = __bfloat162float(o[8]);
    L[3][2] = __bfloat162float(o[9]);
}

// Training head: Q = L L^T + eps I, e = Q a_hat - xi; loss += |e|^2 * scale;
// writes dLoss/do into gout (channels 10..15 zero).  Voxels with mask 0
// (unobserved) contribute nothing.
__global__ void __launch_bounds__(256) k_head_train(const __nv_bfloat16* __restrict__ o,
                                                   const float4* __restrict__ ahat,
                                                   const float4* __restrict__ xi,
                                                   const unsigned char* __restrict__ mask,
                                                   __nv_bfloat16* __restrict__ gout, long long V,
                                                   float scale, double* loss) {
    double lacc = 0.0;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < V;
         v += (long long)gridDim.x * blockDim.x) {
        __nv_bfloat16* gv = gout + v * kC;
        if (mask && !mask[v]) {
            for (int c = 0; c < kC; ++c) gv[c] = __float2bfloat16(0.f);
            continue;
        }
        float L[4][4], od[4];
        head_L(o + v * kC, L, od);
        const float4 a4 = ahat[v], x4 = xi[v];
        const float a[4] = {a4.x, a4.y, a4.z, a4.w}, xs[4] = {x4.x, x4.y, x4.z, x4.w};
        // u = L^T a, y = L u + eps a
        float u[4], e[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            u[j] = 0.f;
#pragma unroll
            for (int i = 0; i < 4; ++i) u[j] += L[i][j] * a[i];
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float y = kQeps * a[i];
#pragma unroll
            for (int j = 0; j < 4; ++j) y += L[i][j] * u[j];
            e[i] = y - xs[i];
            lacc += (double)e[i] * e[i];
        }
        // dLoss/dQ = 2 s e a^T; dQ/dL: dL = (G + G^T) L with G = 2 s e a^T
        float dL[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float sacc = 0.f;
#pragma unroll
                for (int k = 0; k < 4; ++k) sacc += (e[i] * a[k] + e[k] * a[i]) * L[k][j];
                dL[i][j] = 2.0f * scale * sacc;
            }
        float go[10];
#pragma unroll
        for (int i = 0; i < 4; ++i) go[i] = dL[i][i] * sigm(od[i]);
        go[4] = dL[1][0]; go[5] = dL[2][0]; go[6] = dL[2][1];
        go[7] = dL[3][0]; go[8] = dL[3][1]; go[9] = dL[3][2];
        for (int c = 0; c < 10; ++c) gv[c] = __float2bfloat16(go[c]);
        for (int c = 10; c < kC; ++c) gv[c] = __float2bfloat16(0.f);
    }
    block_add_f64<8>(lacc * scale, loss);
}

// Inference head: P_v = D^{-1/2} (L L^T + eps I) D^{-1/2} as a row-major 4x4
// block (zero rows/columns where d_j <= floor, i.e. Jacobi's unobserved rule).
__global__ void __launch_bounds__(256) k_head_infer(const __nv_bfloat16* __restrict__ o,
                                                   const float4* __restrict__ diag,
                                                   float* __restrict__ blocks, long long V,
                                                   float floor_d) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < V;
         v += (long long)gridDim.x * blockDim.x) {
        float L[4][4], od[4];
        head_L(o + v * kC, L, od);
        const float4 d4 = diag[v];
        const float d[4] = {d4.x, d4.y, d4.z, d4.w};
        float s[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) s[i] = d[i] > floor_d ? rsqrtf(d[i]) : 0.0f;
        float* B = blocks + v * 16;
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float q = (i == j) ? kQeps : 0.f;
#pragma unroll
                for (int k = 0; k < 4; ++k) q += L[i][k] * L[j][k];
                B[i * 4 + j] = s[i] * q * s[j];
            }
    }
}

// Per-voxel input features (channels-last, 16): [0..3] log1p(d_c / dmean_c),
// [4..6] block couplings a.s_k / sqrt(d_k d_sigma), [7..10] g_c / sqrt(d_c)
// divided by gscale and clipped to [-4, 4], [11] occupancy 1 - e^{-sigma}, rest 0.
__global__ void __launch_bounds__(256) k_lpc_features(const float4* __restrict__ x,
                                                     const float4* __restrict__ grad,
                                                     const float4* __restrict__ diag,
                                                     const float4* __restrict__ cross,
                                                     const double* __restrict__ stats,
                                                     __nv_bfloat16* __restrict__ feat,
                                                     long long V, float floor_d) {
    const float dm[4] = {(float)stats[0], (float)stats[1], (float)stats[2], (float)stats[3]};
    const float gs = (float)stats[4];
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < V;
         v += (long long)gridDim.x * blockDim.x) {
        const float4 d4 = diag[v], g4 = grad[v], x4 = x[v];
        const float d[4] = {d4.x, d4.y, d4.z, d4.w}, g[4] = {g4.x, g4.y, g4.z, g4.w};
        float f[kC];
#pragma unroll
        for (int c = 0; c < kC; ++c) f[c] = 0.f;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            f[c] = log1pf(d[c] / (dm[c] > 0.f ? dm[c] : 1.f));
            const float sd = d[c] > floor_d ? sqrtf(d[c]) : 0.f;
            f[7 + c] = sd > 0.f ? fminf(fmaxf(g[c] / (sd * (gs > 0.f ? gs : 1.f)), -4.f), 4.f) : 0.f;
        }
        if (cross) {
            const float4 c4 = cross[v];
            const float cr[3] = {c4.x, c4.y, c4.z};
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float den = d[k] * d[3];
                f[4 + k] = den > floor_d ? cr[k] * rsqrtf(den) : 0.f;
            }
        }
        f[11] = 1.0f - expf(-fmaxf(x4.w, 0.f));
#pragma unroll
        for (int c = 0; c < kC; c += 2)
            *reinterpret_cast<uint32_t*>(feat + v * kC + c) = pack_bf16(f[c], f[c + 1]);
    }
}

// stats[0..3] += d_c (grid voxels); stats[4] += (g_c / sqrt(d_c))^2 summed
// over channels; stats[5] += count of channels with d_c > floor.
__global__ void __launch_bounds__(256) k_lpc_stats(const float4* __restrict__ grad,
                                                  const float4* __restrict__ diag, long long V,
                                                  float floor_d, double* stats) {
    double a[6] = {0, 0, 0, 0, 0, 0};
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < V;
         v += (long long)gridDim.x * blockDim.x) {
        const float4 d4 = diag[v], g4 = grad[v];
        const float d[4] = {d4.x, d4.y, d4.z, d4.w}, g[4] = {g4.x, g4.y, g4.z, g4.w};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            a[c] += d[c];
            if (d[c] > floor_d) {
                a[4] += (double)g[c] * g[c] / d[c];
                a[5] += 1.0;
            }
        }
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) block_add_f64<8>(a[q], stats + q);
}

// Adam on FP32 master weights; writes the bf16 copy used by the kernels.
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ gw, float* __restrict__ m,
                       float* __restrict__ v2, __nv_bfloat16* __restrict__ wb, int n, float lr,
                       float b1, float b2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = gw[i];
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * v2[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v2[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    if (wb) wb[i] = __float2bfloat16(wi);
}

__global__ void k_f32_to_bf16(const float* __restrict__ a, __nv_bfloat16* __restrict__ b, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = __float2bfloat16(a[i]);
}

// Exact block-Jacobi: invert each voxel's 4x4 diagonal block of J^T J.  A
// colour parameter c_k enters only residual k, so the block is
//   [[a I_3, c], [c^T, s]],   a = colour diagonal (equal for r, g, b),
//   c_k = sum_rows (dr/dc_k)(dr/dsigma),  s = opacity diagonal,
// with inverse [[I/a + c c^T / (a^2 q), -c / (a q)], [-c^T / (a q), 1 / q]],
// q = s - c.c / a (Schur complement), evaluated in FP64.  Where the block is
// numerically singular (q <= 1e-4 s: the rays through the voxel have nearly
// proportional derivatives) or unobserved, the voxel falls back to Jacobi
// (1/d_j, 0 for d_j <= floor).
__global__ void __launch_bounds__(256) k_block_jacobi(const float4* __restrict__ diag,
                                                     const float4* __restrict__ cross,
                                                     float* __restrict__ blocks, long long V,
                                                     float floor_d) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < V;
         v += (long long)gridDim.x * blockDim.x) {
        const float4 d4 = diag[v], c4 = cross[v];
        const double d[4] = {d4.x, d4.y, d4.z, d4.w};
        const double c[3] = {c4.x, c4.y, c4.z};
        const double a = d[0], sv = d[3];
        const double q = (a > floor_d) ? sv - (c[0] * c[0] + c[1] * c[1] + c[2] * c[2]) / a : 0.0;
        const bool ok = d[0] > floor_d && d[1] > floor_d && d[2] > floor_d && d[3] > floor_d &&
                        q > 1e-4 * sv;
        float* B = blocks + v * 16;
        if (ok) {
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j)
                    B[i * 4 + j] = (float)((i == j ? 1.0 / a : 0.0) + c[i] * c[j] / (a * a * q));
            for (int i = 0; i < 3; ++i) {
                B[i * 4 + 3] = (float)(-c[i] / (a * q));
                B[12 + i] = (float)(-c[i] / (a * q));
            }
            B[15] = (float)(1.0 / q);
        } else {
            for (int i = 0; i < 4; ++i)
                for (int j = 0; j < 4; ++j)
                    B[i * 4 + j] = (i == j && d[i] > floor_d) ? (float)(1.0 / d[i]) : 0.0f;
        }
    }
}

// out_v = D_v^{-1/2} in_v on the grid voxels (0 where d <= floor, and on
// voxels with mask 0 when mask is given); optionally also writes the mask
// (1 where all four d > floor).
__global__ void __launch_bounds__(256) k_dscale(const float4* __restrict__ diag,
                                               const float4* __restrict__ in,
                                               float4* __restrict__ out,
                                               unsigned char* __restrict__ mask_out, long long V,
                                               float floor_d) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < V;
         v += (long long)gridDim.x * blockDim.x) {
        const float4 d = diag[v], a = in[v];
        const bool ok = d.x > floor_d && d.y > floor_d && d.z > floor_d && d.w > floor_d;
        if (mask_out) mask_out[v] = ok ? 1 : 0;
        out[v] = ok ? make_float4(a.x * rsqrtf(d.x), a.y * rsqrtf(d.y), a.z * rsqrtf(d.z),
                                  a.w * rsqrtf(d.w))
                    : make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// ------------------------------------------------------------- launchers

cudaError_t launch_block_jacobi(const float* diag, const float* cross, float* blocks, long long V,
                                cudaStream_t st);

static int lpc_blocks(long long work, int threads) {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    long long want = (work + threads - 1) / threads;
    long long cap = (long long)sms * 16;
    long long b = want < cap ? want : cap;
    return (int)(b > 0 ? b : 1);
}

cudaError_t lpc_conv_bwd_w(const __nv_bfloat16* in, const __nv_bfloat16* gpre, float* dW,
                           float* dB, int G, cudaStream_t st) {
    const long long V = (long long)G * G * G;
    const long long chunks = (V + 15) / 16;
    int bx = lpc_blocks(chunks * 32, kLThreads) / 8;
    if (bx < 1) bx = 1;
    k_conv_bwd_w<<<dim3(bx, kTaps), kLThreads, 0, st>>>(in, gpre, dW, dB, G);
    count_launch();
    return cudaGetLastError();
}

cudaError_t lpc_conv_flip(const __nv_bfloat16* W, __nv_bfloat16* Wt, cudaStream_t st) {
    k_conv_flip<<<(kTaps * kC * kC + 255) / 256, 256, 0, st>>>(W, Wt);
    count_launch();
    return cudaGetLastError();
}

cudaError_t lpc_relu_bwd(__nv_bfloat16* g, const __nv_bfloat16* act, long long n, cudaStream_t st) {
    k_relu_bwd<<<lpc_blocks(n, 256), 256, 0, st>>>(g, act, n);
    count_launch();
    return cudaGetLastError();
}

cudaError_t lpc_head_train(const __nv_bfloat16* o, const float* ahat, const float* xi,
                           const unsigned char* mask, __nv_bfloat16* gout, long long V, float scale,
                           double* loss, cudaStream_t st) {
    k_head_train<<<lpc_blocks(V, 256), 256, 0, st>>>(o, reinterpret_cast<const float4*>(ahat),
                                                      reinterpret_cast<const float4*>(xi), mask,
                                                      gout, V, scale, loss);
    count_launch();
    return cudaGetLastError();
}

cudaError_t lpc_head_infer(const __nv_bfloat16* o, const float* diag, float* blocks, long long V,
                           cudaStream_t st) {
    k_head_infer<<<lpc_blocks(V, 256), 256, 0, st>>>(o, reinterpret_cast<const float4*>(diag),
                                                      blocks, V, 1e-30f);
    count_launch();
    return cudaGetLastError();
}

cudaError_t lpc_features(const float* x, const float* grad, const float* diag, const float* cross,
                         double* stats, __nv_bfloat16* feat, long long V, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(stats, 0, 6 * sizeof(double), st);
    if (e != cudaSuccess) return e;
    k_lpc_stats<<<lpc_blocks(V, 256), 256, 0, st>>>(reinterpret_cast<const float4*>(grad),
                                                     reinterpret_cast<const float4*>(diag), V,
                                                     1e-30f, stats);
    k_lpc_features<<<lpc_blocks(V, 256), 256, 0, st>>>(
        reinterpret_cast<const float4*>(x), reinterpret_cast<const float4*>(grad),
        reinterpret_cast<const float4*>(diag), reinterpret_cast<const float4*>(cross), stats, feat,
        V, 1e-30f);
    count_launch(2);
    return cudaGetLastError();
}

cudaError_t lpc_adam(float* w, const float* gw, float* m, float* v2, __nv_bfloat16* wb, int n,
                     float lr, int step, cudaStream_t st) {
    const float b1 = 0.9f, b2 = 0.999f;
    float c1 = 1.f, c2 = 1.f;
    for (int i = 0; i < step; ++i) { c1 *= b1; c2 *= b2; }
    k_adam<<<(n + 255) / 256, 256, 0, st>>>(w, gw, m, v2, wb, n, lr, b1, b2, 1e-8f, 1.f - c1, 1.f - c2);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_dscale(const float* diag, const float* in, float* out, unsigned char* mask,
                          long long V, cudaStream_t st) {
    k_dscale<<<lpc_blocks(V, 256), 256, 0, st>>>(reinterpret_cast<const float4*>(diag),
                                                  reinterpret_cast<const float4*>(in),
                                                  reinterpret_cast<float4*>(out), mask, V, 1e-30f);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_block_jacobi(const float* diag, const float* cross, float* blocks, long long V,
                                cudaStream_t st) {
    k_block_jacobi<<<lpc_blocks(V, 256), 256, 0, st>>>(reinterpret_cast<const float4*>(diag),
                                                        reinterpret_cast<const float4*>(cross),
                                                        blocks, V, 1e-30f);
    count_launch();
    return cudaGetLastError();
}

cudaError_t lpc_to_bf16(const float* a, __nv_bfloat16* b, int n, cudaStream_t st) {
    k_f32_to_bf16<<<(n + 255) / 256, 256, 0, st>>>(a, b, n);
    count_launch();
    return cudaGetLastError();
}

}  // namespace perf

// k_hier.cu -- level change of the hierarchical formulation (Section
// "Hierarchical formulation"): the next level doubles the grid and the
// environment-map resolution and is filled from the previous level's result
// by linear interpolation at the new cell centres.
//
// Fine cell i' has its centre at coarse index coordinate u = i'/2 - 1/4;
// the grid uses the ray march's clamp convention (u in [0, G-1], base <=
// G-2), equirectangular maps wrap in longitude and clamp in latitude, and a
// cube map's faces are upsampled one by one, clamped at their edges.  The weights are
// 1/4, 3/4 (or 0, 1 at a clamped edge), exact in binary32.  Opacity is per
// voxel side (Eq. 3 with delta-bar = delta / h), so grid sigma is halved to
// keep every path's optical depth; a shell hit has delta-bar = 1 on every
// level, so shell sigma is kept.
#include "perf_kernels.h"

namespace perf {

namespace {

constexpr int kUpThreads = 256;

__device__ __forceinline__ void axis_up(int i, int n, int& b, float& f) {
    float u = 0.5f * (float)i - 0.25f;
    u = fminf(fmaxf(u, 0.0f), (float)(n - 1));
    float fl = fminf(floorf(u), (float)(n - 2));
    b = (int)fl;
    f = u - fl;
}

__device__ __forceinline__ void acc4(float4& a, float w, float4 v) {
    a.x = fmaf(w, v.x, a.x);
    a.y = fmaf(w, v.y, a.y);
    a.z = fmaf(w, v.z, a.z);
    a.w = fmaf(w, v.w, a.w);
}

__global__ void __launch_bounds__(kUpThreads) k_upsample(const float4* __restrict__ x, int G, int S,
                                                         int He, int We, int cube,
                                                         float4* __restrict__ y, long long n_out) {
    const int G2 = 2 * G, He2 = 2 * He, We2 = 2 * We;
    const long long nv2 = (long long)G2 * G2 * G2;
    const long long nv = (long long)G * G * G;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n_out;
         v += (long long)gridDim.x * blockDim.x) {
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
        if (v < nv2) {
            const int xi = (int)(v % G2), yi = (int)((v / G2) % G2), zi = (int)(v / ((long long)G2 * G2));
            int bx, by, bz;
            float fx, fy, fz;
            axis_up(xi, G, bx, fx);
            axis_up(yi, G, by, fy);
            axis_up(zi, G, bz, fz);
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int dx = c & 1, dy = (c >> 1) & 1, dz = c >> 2;
                const float w = (dx ? fx : 1.0f - fx) * (dy ? fy : 1.0f - fy) * (dz ? fz : 1.0f - fz);
                acc4(a, w, x[((long long)(bz + dz) * G + (by + dy)) * G + (bx + dx)]);
            }
            a.w *= 0.5f;
        } else {
            const long long t = v - nv2;
            const int s = (int)(t / ((long long)He2 * We2));
            const int rem = (int)(t - (long long)s * He2 * We2);
            const int ri = rem / We2, ci = rem - ri * We2;
            int br;
            float fr;
            axis_up(ri, He, br, fr);
            int c0, c1;
            float fc;
            if (cube) {
                // each face (He x He texels) on its own, clamped at its edges
                const int face = ci / (2 * He), cf = ci - face * 2 * He;
                int bc;
                axis_up(cf, He, bc, fc);
                c0 = face * He + bc;
                c1 = c0 + 1;
            } else {
                const float uc = 0.5f * (float)ci - 0.25f;
                const float fl = floorf(uc);
                fc = uc - fl;
                c0 = (int)fl % We;
                if (c0 < 0) c0 += We;
                c1 = c0 + 1 == We ? 0 : c0 + 1;
            }
            const float4* sh = x + nv + (long long)s * He * We;
            acc4(a, (1.0f - fr) * (1.0f - fc), sh[(long long)br * We + c0]);
            acc4(a, (1.0f - fr) * fc, sh[(long long)br * We + c1]);
            acc4(a, fr * (1.0f - fc), sh[(long long)(br + 1) * We + c0]);
            acc4(a, fr * fc, sh[(long long)(br + 1) * We + c1]);
        }
        y[v] = a;
    }
}

}  // namespace

cudaError_t launch_upsample(const float* x, int G, int S, int He, int We, int cube, float* y,
                            cudaStream_t st) {
    const long long G2 = 2ll * G;
    const long long n_out = G2 * G2 * G2 + (long long)S * 4 * He * We;
    if (n_out == 0) return cudaSuccess;
    long long blocks = (n_out + kUpThreads - 1) / kUpThreads;
    if (blocks > 152ll * 32) blocks = 152ll * 32;
    k_upsample<<<(int)blocks, kUpThreads, 0, st>>>(reinterpret_cast<const float4*>(x), G, S, He, We,
                                                 cube, reinterpret_cast<float4*>(y), n_out);
    count_launch();
    return cudaGetLastError();
}

}  // namespace perf

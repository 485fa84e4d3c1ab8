// perf_device.cuh -- device-side geometry of the PERF ray march (sm_103a).
//
// One ray per thread.  The ray itself (pixel -> origin / unit direction, box
// entry and exit, the sample count K and step delta, which shells are hit) is
// computed in IEEE binary32 with every operation rounded separately
// (__fadd_rn & co. block FMA contraction), so that these integer decisions are
// a fixed function of the inputs.  Everything after that is ordinary FP32.
//
// Conventions (PERF Section "Method", Section "Rendering", Section
// "Jittering"):
//   - grid [-1,1]^3, G^3 voxels, voxel side h = 2/G, centres at -1+(i+1/2)h;
//   - K = ceil(L/h) samples (capped at max_samples) at t_in + (k+1/2+j_k) delta,
//     delta = L/K, optical thickness sigma * delta/h (sigma per voxel side);
//   - exact trilinear interpolation clamped to the edge;
//   - shells: far root of |o + t d| = R, composited after the grid in order,
//     with optical thickness sigma (one voxel side); equirectangular bilinear
//     lookup wrapped in azimuth, clamped in polar angle.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

namespace perf {

constexpr int kMaxShells = 8;

struct DevScene {
    int G;
    float halfG;             // G/2
    float h;                 // 2/G in binary32
    int S;
    float R[kMaxShells];
    int He, We;
    int env_kind;            // 0 equirectangular shells, 1 cube maps (We = 6 He)
    long long n_vox;         // G^3
    long long shell_texels;  // He*We
    int W, H, n_cams;
    long long n_rays;
    long long n_tiles;       // tile_w x tile_h pixel tiles over all cameras
    int tiles_x, tiles_y;
    int tile_w, tile_h;      // one warp per tile: tile_w * tile_h = 32
    int cap_per_sm;          // resident-CTA cap of the scatter kernels (0 = none)
    const float* cams;       // n_cams x 16: c2w (12), focal, pad
    int max_samples;
    int jitter;
    unsigned long long seed;
    unsigned epoch;
    int aux;                 // 1: the auxiliary opacity residual (4 residuals per ray)
    float aux_lambda;
    long long tile_lo;       // a launch processes tiles [tile_lo, n_tiles)
    long long coef_tiles;    // tiles [0, coef_tiles) have rows in the coefficient store
    unsigned long long* red_count;   // non-null: count the J^T scatter's vector-atomic lane operations
    // Shell hits per ray (n_rays x S entries, see shell_entry); null: each
    // march computes them itself in FP32.
    const float4* shell_tab;
    // Block order of the grid part of the parameter-space vectors a
    // Gauss-Newton step's PCG works on (p, A p, the diagonal, the gradient,
    // Delta, rho): see LayoutKey.  lay_s = 0: canonical [z][y][x].
    int lay_s, lay_ys, lay_zs;
    // Per-ray length of the coefficient store's non-zero prefix (rays of the
    // store's tiles): grid rows k >= keff[ray] hold only zeros -- samples
    // whose transmittance has underflowed to 0 in binary32 -- so the diagonal
    // march does not write them and the A p neither streams nor visits them.
    // Null: every row up to the ray's sample count is written and read.
    int* keff;
};

// Index of voxel (x, y, z) in a parameter-space vector.  lay_s = 0: the
// canonical order z G^2 + y G + x.  lay_s = s > 0: bricks of B^3 voxels
// (B = 2^s, G a multiple of B), the bricks in [z][y][x] order and the voxels
// of a brick in [z][y][x] order.  Either way the index is a sum of one term
// per axis,
//   f(x) = (x >> s) B^3 + (x & (B-1)),  g(y) = (y >> s) ys + (y & (B-1)) B,
//   h(z) = (z >> s) zs + (z & (B-1)) B^2,
// with ys = (G/B) B^3 and zs = (G/B)^2 B^3 (G and G^2 when s = 0), so the
// index of a neighbour differs in one term only.  Texel blocks follow the
// grid unchanged.
struct LayoutKey {
    int s, m, ys, zs;
    __device__ __forceinline__ int fx(int x) const { return ((x >> s) << (3 * s)) + (x & m); }
    __device__ __forceinline__ int gy(int y) const { return (y >> s) * ys + ((y & m) << s); }
    __device__ __forceinline__ int hz(int z) const { return (z >> s) * zs + ((z & m) << (2 * s)); }
    __device__ __forceinline__ int key(int x, int y, int z) const { return fx(x) + gy(y) + hz(z); }
    __device__ __forceinline__ int shell(int idx) const { return idx; }
};
__device__ __forceinline__ LayoutKey layout_key(const DevScene& sc) {
    return LayoutKey{sc.lay_s, (1 << sc.lay_s) - 1, sc.lay_ys, sc.lay_zs};
}

struct Ray {
    float o[3], d[3];
    float t_in, delta;
    int K;                   // 0: misses the grid
    unsigned shell_hit;
};

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// U[0,1) with 24 bits: SplitMix64 (Steele, Lea, Flood 2014) of (seed+epoch,
// ray, stream); stream 0/1 = pixel jitter, 2+k = sample k.
__device__ __forceinline__ float jitter_u(const DevScene& sc, long long ray, unsigned stream) {
    unsigned long long h = splitmix64(sc.seed + (unsigned long long)sc.epoch);
    h = splitmix64(h + (unsigned long long)ray);
    h = splitmix64(h + (unsigned long long)stream);
    return (float)(h >> 40) * (1.0f / 16777216.0f);
}

// Pixel of lane `lane` in tile `tile` (tiles are tile_w wide, tile_h high,
// row-major over each camera's image, cameras one after the other).
__device__ __forceinline__ bool tile_pixel(const DevScene& sc, long long tile, int lane,
                                           long long& ray) {
    const long long per_cam = (long long)sc.tiles_x * sc.tiles_y;
    const int cam = (int)(tile / per_cam);
    const int t = (int)(tile - (long long)cam * per_cam);
    const int ty = t / sc.tiles_x, tx = t - ty * sc.tiles_x;
    const int col = tx * sc.tile_w + lane % sc.tile_w;
    const int row = ty * sc.tile_h + lane / sc.tile_w;
    if (col >= sc.W || row >= sc.H) return false;
    ray = ((long long)cam * sc.H + row) * sc.W + col;
    return true;
}

__device__ __forceinline__ void ray_setup(const DevScene& sc, long long ray, Ray& R) {
    const long long hw = (long long)sc.W * sc.H;
    const int cam = (int)(ray / hw);
    const long long rem = ray - (long long)cam * hw;
    const int row = (int)(rem / sc.W);
    const int col = (int)(rem - (long long)row * sc.W);
    const float* M = sc.cams + 16 * cam;
    const float f = M[12];
    float jx = 0.5f, jy = 0.5f;
    if (sc.jitter) { jx = jitter_u(sc, ray, 0u); jy = jitter_u(sc, ray, 1u); }
    const float px = __fadd_rn((float)col, jx);
    const float py = __fadd_rn((float)row, jy);
    const float xc = __fdiv_rn(__fsub_rn(px, __fmul_rn(0.5f, (float)sc.W)), f);
    const float yc = -__fdiv_rn(__fsub_rn(py, __fmul_rn(0.5f, (float)sc.H)), f);
    float d[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float u = __fmul_rn(M[4 * a + 0], xc);
        const float v = __fmul_rn(M[4 * a + 1], yc);
        d[a] = __fsub_rn(__fadd_rn(u, v), M[4 * a + 2]);
    }
    const float nn = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(d[0], d[0]), __fmul_rn(d[1], d[1])),
                                          __fmul_rn(d[2], d[2])));
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        R.d[a] = __fdiv_rn(d[a], nn);
        R.o[a] = M[4 * a + 3];
    }
    float lo[3], hi[3];
    bool miss = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (R.d[a] != 0.0f) {
            const float t0 = __fdiv_rn(__fsub_rn(-1.0f, R.o[a]), R.d[a]);
            const float t1 = __fdiv_rn(__fsub_rn(1.0f, R.o[a]), R.d[a]);
            lo[a] = fminf(t0, t1);
            hi[a] = fmaxf(t0, t1);
        } else {
            if (R.o[a] < -1.0f || R.o[a] > 1.0f) miss = true;
            lo[a] = -INFINITY;
            hi[a] = INFINITY;
        }
    }
    const float t_in = fmaxf(fmaxf(fmaxf(lo[0], lo[1]), lo[2]), 0.0f);
    const float t_out = fminf(fminf(hi[0], hi[1]), hi[2]);
    R.t_in = t_in;
    R.K = 0;
    R.delta = 0.0f;
    if (!miss && t_out > t_in) {
        const float L = __fsub_rn(t_out, t_in);
        int K = (int)ceilf(__fdiv_rn(L, sc.h));
        K = min(K, sc.max_samples);
        K = max(K, 1);
        R.K = K;
        R.delta = __fdiv_rn(L, (float)K);
    }
    const float b = __fadd_rn(__fadd_rn(__fmul_rn(R.o[0], R.d[0]), __fmul_rn(R.o[1], R.d[1])),
                              __fmul_rn(R.o[2], R.d[2]));
    const float oo = __fadd_rn(__fadd_rn(__fmul_rn(R.o[0], R.o[0]), __fmul_rn(R.o[1], R.o[1])),
                               __fmul_rn(R.o[2], R.o[2]));
    unsigned hit = 0u;
    for (int s = 0; s < sc.S; ++s) {
        const float c = __fsub_rn(oo, __fmul_rn(sc.R[s], sc.R[s]));
        const float disc = __fsub_rn(__fmul_rn(b, b), c);
        if (disc > 0.0f && (b < 0.0f || c < 0.0f)) hit |= 1u << s;
    }
    R.shell_hit = hit;
}

// Trilinear cell of a sample: base voxel (linear index) and fractions.
struct Cell {
    int bx, by, bz;
    float fx, fy, fz;
};

__device__ __forceinline__ void axis_cell(float p, const DevScene& sc, int& b, float& f) {
    float u = fmaf(p, sc.halfG, sc.halfG - 0.5f);
    u = fminf(fmaxf(u, 0.0f), (float)(sc.G - 1));
    float fl = floorf(u);
    fl = fminf(fl, (float)(sc.G - 2));
    b = (int)fl;
    f = u - fl;
}

__device__ __forceinline__ Cell sample_cell(const DevScene& sc, const Ray& R, long long ray, int k) {
    float jk = 0.0f;
    if (sc.jitter) jk = jitter_u(sc, ray, 2u + (unsigned)k) - 0.5f;
    const float t = fmaf((float)k + 0.5f + jk, R.delta, R.t_in);
    Cell c;
    axis_cell(fmaf(t, R.d[0], R.o[0]), sc, c.bx, c.fx);
    axis_cell(fmaf(t, R.d[1], R.o[1]), sc, c.by, c.fy);
    axis_cell(fmaf(t, R.d[2], R.o[2]), sc, c.bz, c.fz);
    return c;
}

// --- storage access: float4 (FP32) or 4 x bf16 (BF16) per voxel / texel
template <typename T> struct Store;
template <> struct Store<float> {
    static __device__ __forceinline__ float4 ld(const float* x, int v) {
        return __ldg(reinterpret_cast<const float4*>(x) + v);
    }
};
template <> struct Store<__nv_bfloat16> {
    static __device__ __forceinline__ float4 ld(const __nv_bfloat16* x, int v) {
        const uint2 u = __ldg(reinterpret_cast<const uint2*>(x) + v);
        float4 r;
        r.x = __uint_as_float(u.x << 16);
        r.y = __uint_as_float(u.x & 0xffff0000u);
        r.z = __uint_as_float(u.y << 16);
        r.w = __uint_as_float(u.y & 0xffff0000u);
        return r;
    }
};

// Paired FP32 storage: record v holds parameter block v of x (first 16 bytes)
// and of the PCG direction p (last 16 bytes), so the J p sweep of A p
// fetches both with one 256-bit load per corner.  Read through Store it
// yields the x half.  Records are 32-byte aligned (device allocations are).
struct PairF32 {
    float4 x, p;
};
template <> struct Store<PairF32> {
    static __device__ __forceinline__ float4 ld(const PairF32* x, int v) {
        return __ldg(&x[v].x);
    }
};
__device__ __forceinline__ void ld_pair(const PairF32* xp, int v, float4& a, float4& q) {
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(q.x), "=f"(q.y), "=f"(q.z), "=f"(q.w)
        : "l"(xp + v));
}

__device__ __forceinline__ float4 lerp4(float4 a, float4 b, float t) {
    return make_float4(fmaf(t, b.x - a.x, a.x), fmaf(t, b.y - a.y, a.y),
                       fmaf(t, b.z - a.z, a.z), fmaf(t, b.w - a.w, a.w));
}

// Trilinear interpolation as a weighted sum of the 8 corners (corner c:
// bit a = +1 along axis a), weights w_c = prod_a (c_a ? f_a : 1 - f_a).
#ifndef PERF_INTERP_W
#define PERF_INTERP_W 1
#endif
__device__ __forceinline__ void tri_weights(const Cell& c, float (&W)[8]) {
    const float gx[2] = {1.0f - c.fx, c.fx}, gy[2] = {1.0f - c.fy, c.fy}, gz[2] = {1.0f - c.fz, c.fz};
#pragma unroll
    for (int k = 0; k < 8; ++k) W[k] = (gx[k & 1] * gy[(k >> 1) & 1]) * gz[k >> 2];
}

__device__ __forceinline__ float4 wsum8(const float (&W)[8], const float4 (&a)[8]) {
    float4 r = make_float4(W[0] * a[0].x, W[0] * a[0].y, W[0] * a[0].z, W[0] * a[0].w);
#pragma unroll
    for (int k = 1; k < 8; ++k) {
        r.x = fmaf(W[k], a[k].x, r.x);
        r.y = fmaf(W[k], a[k].y, r.y);
        r.z = fmaf(W[k], a[k].z, r.z);
        r.w = fmaf(W[k], a[k].w, r.w);
    }
    return r;
}

template <typename T>
__device__ __forceinline__ float4 interp_grid(const T* x, const DevScene& sc, const Cell& c) {
    // block indices fit in int: a scene has fewer than 2^31 parameter blocks
    const int G = sc.G;
    const int i0 = (c.bz * G + c.by) * G + c.bx;
    const int sy = G, sz = G * G;
    float4 a[8];
    a[0] = Store<T>::ld(x, i0);
    a[1] = Store<T>::ld(x, i0 + 1);
    a[2] = Store<T>::ld(x, i0 + sy);
    a[3] = Store<T>::ld(x, i0 + sy + 1);
    a[4] = Store<T>::ld(x, i0 + sz);
    a[5] = Store<T>::ld(x, i0 + sz + 1);
    a[6] = Store<T>::ld(x, i0 + sz + sy);
    a[7] = Store<T>::ld(x, i0 + sz + sy + 1);
#if PERF_INTERP_W
    float W[8];
    tri_weights(c, W);
    return wsum8(W, a);
#else
    const float4 b00 = lerp4(a[0], a[1], c.fx), b10 = lerp4(a[2], a[3], c.fx);
    const float4 b01 = lerp4(a[4], a[5], c.fx), b11 = lerp4(a[6], a[7], c.fx);
    const float4 c0 = lerp4(b00, b10, c.fy), c1 = lerp4(b01, b11, c.fy);
    return lerp4(c0, c1, c.fz);
#endif
}

// interp_grid for a vector stored in the order of a LayoutKey.
template <typename T>
__device__ __forceinline__ float4 interp_grid_lay(const T* x, const LayoutKey& k, const Cell& c) {
    const int x0 = k.fx(c.bx), x1 = k.fx(c.bx + 1);
    const int y0 = k.gy(c.by), y1 = k.gy(c.by + 1);
    const int z0 = k.hz(c.bz), z1 = k.hz(c.bz + 1);
    float4 a[8];
    a[0] = Store<T>::ld(x, x0 + y0 + z0);
    a[1] = Store<T>::ld(x, x1 + y0 + z0);
    a[2] = Store<T>::ld(x, x0 + y1 + z0);
    a[3] = Store<T>::ld(x, x1 + y1 + z0);
    a[4] = Store<T>::ld(x, x0 + y0 + z1);
    a[5] = Store<T>::ld(x, x1 + y0 + z1);
    a[6] = Store<T>::ld(x, x0 + y1 + z1);
    a[7] = Store<T>::ld(x, x1 + y1 + z1);
#if PERF_INTERP_W
    float W[8];
    tri_weights(c, W);
    return wsum8(W, a);
#else
    const float4 b00 = lerp4(a[0], a[1], c.fx), b10 = lerp4(a[2], a[3], c.fx);
    const float4 b01 = lerp4(a[4], a[5], c.fx), b11 = lerp4(a[6], a[7], c.fx);
    const float4 c0 = lerp4(b00, b10, c.fy), c1 = lerp4(b01, b11, c.fy);
    return lerp4(c0, c1, c.fz);
#endif
}

// Trilinear interpolation of x (a) and p (q) from paired storage.
__device__ __forceinline__ void interp_grid_pair(const PairF32* xp, const DevScene& sc,
                                                 const Cell& c, float4& a, float4& q) {
    const int G = sc.G;
    const int i0 = (c.bz * G + c.by) * G + c.bx;
    const int sy = G, sz = G * G;
    float4 ax[8], ap[8];
    ld_pair(xp, i0, ax[0], ap[0]);
    ld_pair(xp, i0 + 1, ax[1], ap[1]);
    ld_pair(xp, i0 + sy, ax[2], ap[2]);
    ld_pair(xp, i0 + sy + 1, ax[3], ap[3]);
    ld_pair(xp, i0 + sz, ax[4], ap[4]);
    ld_pair(xp, i0 + sz + 1, ax[5], ap[5]);
    ld_pair(xp, i0 + sz + sy, ax[6], ap[6]);
    ld_pair(xp, i0 + sz + sy + 1, ax[7], ap[7]);
#if PERF_INTERP_W
    float W[8];
    tri_weights(c, W);
    a = wsum8(W, ax);
    q = wsum8(W, ap);
#else
    a = lerp4(lerp4(lerp4(ax[0], ax[1], c.fx), lerp4(ax[2], ax[3], c.fx), c.fy),
              lerp4(lerp4(ax[4], ax[5], c.fx), lerp4(ax[6], ax[7], c.fx), c.fy), c.fz);
    q = lerp4(lerp4(lerp4(ap[0], ap[1], c.fx), lerp4(ap[2], ap[3], c.fx), c.fy),
              lerp4(lerp4(ap[4], ap[5], c.fx), lerp4(ap[6], ap[7], c.fx), c.fy), c.fz);
#endif
}

// Coordinate along one axis of the voxel with parity bit `pa` in the 2x2x2
// window whose lower corner is at `base`.
__device__ __forceinline__ int par_coord(int base, int pa) { return base + ((pa ^ base) & 1); }

// The 8 corner values of the current sample's cell, held between samples.
// Slot p holds the window voxel whose coordinate parities are p, so when the
// cell moves only the voxels that enter the window are loaded (consecutive
// samples one voxel side apart share half their corners or more).
template <typename T>
struct Corners {
    float4 v[8];
    int b[3];

    __device__ __forceinline__ void reset() { b[0] = b[1] = b[2] = -(1 << 28); }

    __device__ __forceinline__ float4 interp(const T* __restrict__ x, const DevScene& sc,
                                             const Cell& cl) {
        const int G = sc.G;
#pragma unroll
        for (int p = 0; p < 8; ++p) {
            const int nx = par_coord(cl.bx, p & 1), ny = par_coord(cl.by, (p >> 1) & 1),
                      nz = par_coord(cl.bz, p >> 2);
            const bool same = nx == par_coord(b[0], p & 1) && ny == par_coord(b[1], (p >> 1) & 1) &&
                              nz == par_coord(b[2], p >> 2);
            if (!same) v[p] = Store<T>::ld(x, (nz * G + ny) * G + nx);
        }
        b[0] = cl.bx; b[1] = cl.by; b[2] = cl.bz;
        const bool sx = cl.bx & 1, sy = cl.by & 1, sz = cl.bz & 1;
        const float wx[2] = {sx ? cl.fx : 1.0f - cl.fx, sx ? 1.0f - cl.fx : cl.fx};
        const float wy[2] = {sy ? cl.fy : 1.0f - cl.fy, sy ? 1.0f - cl.fy : cl.fy};
        const float wz[2] = {sz ? cl.fz : 1.0f - cl.fz, sz ? 1.0f - cl.fz : cl.fz};
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int p = 0; p < 8; ++p) {
            const float W = wx[p & 1] * wy[(p >> 1) & 1] * wz[p >> 2];
            acc.x = fmaf(W, v[p].x, acc.x);
            acc.y = fmaf(W, v[p].y, acc.y);
            acc.z = fmaf(W, v[p].z, acc.z);
            acc.w = fmaf(W, v[p].w, acc.w);
        }
        return acc;
    }
};

// Bilinear texels of one shell hit: 4 parameter-block indices and weights.
struct ShellHit {
    int idx[4];
    float w[4];
};

// Cube-map shell-hit entry (perf.h, PERF_ENV_CUBE): the far-root hit point,
// the face of its largest coordinate and the face's texel coordinates in
// binary32 with every operation rounded once (no contraction), so the face
// and texel decisions are a fixed function of the ray.  Entry layout as in
// shell_decode: (first texel index, fu, fv, column step 1).
__device__ __forceinline__ float4 cube_entry(const DevScene& sc, const Ray& R, int s) {
    const float b = __fadd_rn(__fadd_rn(__fmul_rn(R.o[0], R.d[0]), __fmul_rn(R.o[1], R.d[1])),
                              __fmul_rn(R.o[2], R.d[2]));
    const float oo = __fadd_rn(__fadd_rn(__fmul_rn(R.o[0], R.o[0]), __fmul_rn(R.o[1], R.o[1])),
                               __fmul_rn(R.o[2], R.o[2]));
    const float c = __fsub_rn(oo, __fmul_rn(sc.R[s], sc.R[s]));
    const float disc = fmaxf(__fsub_rn(__fmul_rn(b, b), c), 0.0f);
    const float sq = __fsqrt_rn(disc);
    const float t = (b < 0.0f) ? __fsub_rn(sq, b) : __fdiv_rn(c, __fsub_rn(-b, sq));
    const float q[3] = {__fmaf_rn(t, R.d[0], R.o[0]), __fmaf_rn(t, R.d[1], R.o[1]),
                        __fmaf_rn(t, R.d[2], R.o[2])};
    const float ax = fabsf(q[0]), ay = fabsf(q[1]), az = fabsf(q[2]);
    int a = 2;
    if (ax >= ay && ax >= az) a = 0;
    else if (ay >= az) a = 1;
    const float qa = a == 0 ? q[0] : (a == 1 ? q[1] : q[2]);
    const float qb = a == 0 ? q[1] : q[0];
    const float qc = a == 2 ? q[1] : q[2];
    const int face = 2 * a + (qa < 0.0f ? 1 : 0);
    const int F = sc.He;
    const float m = fabsf(qa);
    const float hf = 0.5f * (float)F;
    float u = __fmaf_rn(__fdiv_rn(qb, m), hf, hf - 0.5f);
    float v = __fmaf_rn(__fdiv_rn(qc, m), hf, hf - 0.5f);
    u = fminf(fmaxf(u, 0.0f), (float)(F - 1));
    v = fminf(fmaxf(v, 0.0f), (float)(F - 1));
    const float j0 = fminf(floorf(u), (float)(F - 2));
    const float i0 = fminf(floorf(v), (float)(F - 2));
    const int base = (int)(sc.n_vox + (long long)s * sc.shell_texels);
    const int idx0 = base + (int)i0 * sc.We + face * F + (int)j0;
    return make_float4(__int_as_float(idx0), u - j0, v - i0, __int_as_float(1));
}

// Bilinear texels from a shell-hit entry: (first texel index, fu, fv, column
// step to the second texel) -- the step is 1, or 1 - We across an
// equirectangular map's longitude seam.
__device__ __forceinline__ void shell_decode(const DevScene& sc, float4 e, ShellHit& hs) {
    const int i0 = __float_as_int(e.x), dc = __float_as_int(e.w);
    const float fu = e.y, fv = e.z;
    hs.idx[0] = i0;
    hs.idx[1] = i0 + dc;
    hs.idx[2] = i0 + sc.We;
    hs.idx[3] = i0 + sc.We + dc;
    hs.w[0] = (1.0f - fu) * (1.0f - fv);
    hs.w[1] = fu * (1.0f - fv);
    hs.w[2] = (1.0f - fu) * fv;
    hs.w[3] = fu * fv;
}

// The shell-hit entry of a ray that hits shell s.  Equirectangular maps: the
// texel coordinates in FP64 from the binary32 ray (far root of |o + t d| = R,
// azimuth atan2(y, x), polar angle from +z): a binary32 coordinate of a map
// 1024 texels wide resolves only ~6e-5 of a texel, which moves the bilinear
// weights by ~1e-4 relative.  Cube maps: the binary32 lookup (exact decisions).
__device__ __forceinline__ float4 shell_entry(const DevScene& sc, const Ray& R, int s) {
    if (sc.env_kind == 1) return cube_entry(sc, R, s);
    const int base = (int)(sc.n_vox + (long long)s * sc.shell_texels);
    const double o0 = R.o[0], o1 = R.o[1], o2 = R.o[2];
    const double d0 = R.d[0], d1 = R.d[1], d2 = R.d[2];
    const double b = o0 * d0 + o1 * d1 + o2 * d2;
    const double oo = o0 * o0 + o1 * o1 + o2 * o2;
    const double rad = (double)sc.R[s];
    const double c = oo - rad * rad;
    const double disc = fmax(b * b - c, 0.0);
    const double sq = sqrt(disc);
    const double t = (b < 0.0) ? (-b + sq) : (c / (-b - sq));
    const double qx = o0 + t * d0, qy = o1 + t * d1, qz = o2 + t * d2;
    const double r = sqrt(qx * qx + qy * qy + qz * qz);
    const double wx = qx / r, wy = qy / r, wz = qz / r;
    const double phi = atan2(wy, wx);
    const double theta = atan2(sqrt(wx * wx + wy * wy), wz);
    const double u = (phi / (2.0 * 3.141592653589793) + 0.5) * (double)sc.We - 0.5;
    double v = theta / 3.141592653589793 * (double)sc.He - 0.5;
    const double j0 = floor(u);
    const double fu = u - j0;
    int c0 = (int)((long long)j0 % sc.We);
    if (c0 < 0) c0 += sc.We;
    const int dcol = c0 + 1 < sc.We ? 1 : 1 - sc.We;
    v = fmin(fmax(v, 0.0), (double)(sc.He - 1));
    const double i0 = fmin(floor(v), (double)(sc.He - 2));
    const double fv = v - i0;
    const int idx0 = base + (int)i0 * sc.We + c0;
    return make_float4(__int_as_float(idx0), (float)fu, (float)fv, __int_as_float(dcol));
}

__device__ __forceinline__ bool shell_lookup(const DevScene& sc, const Ray& R, long long ray, int s,
                                             ShellHit& hs) {
    if (!(R.shell_hit & (1u << s))) return false;
    if (sc.shell_tab) {
        shell_decode(sc, __ldg(sc.shell_tab + ray * sc.S + s), hs);
        return true;
    }
    if (sc.env_kind == 1) {
        shell_decode(sc, cube_entry(sc, R, s), hs);
        return true;
    }
    const float b = R.o[0] * R.d[0] + R.o[1] * R.d[1] + R.o[2] * R.d[2];
    const float c = R.o[0] * R.o[0] + R.o[1] * R.o[1] + R.o[2] * R.o[2] - sc.R[s] * sc.R[s];
    const float disc = fmaxf(b * b - c, 0.0f);
    const float sq = sqrtf(disc);
    const float t = (b < 0.0f) ? (sq - b) : (c / (-b - sq));
    const float qx = fmaf(t, R.d[0], R.o[0]);
    const float qy = fmaf(t, R.d[1], R.o[1]);
    const float qz = fmaf(t, R.d[2], R.o[2]);
    const float phi = atan2f(qy, qx);
    const float theta = atan2f(sqrtf(qx * qx + qy * qy), qz);
    const float u = (phi * 0.15915494309189535f + 0.5f) * (float)sc.We - 0.5f;
    float v = theta * 0.31830988618379067f * (float)sc.He - 0.5f;
    const float j0 = floorf(u);
    const float fu = u - j0;
    int c0 = (int)j0 % sc.We;
    if (c0 < 0) c0 += sc.We;
    int c1 = c0 + 1;
    if (c1 >= sc.We) c1 -= sc.We;
    v = fminf(fmaxf(v, 0.0f), (float)(sc.He - 1));
    float i0 = floorf(v);
    i0 = fminf(i0, (float)(sc.He - 2));
    const float fv = v - i0;
    const int r0 = (int)i0;
    const int base = (int)(sc.n_vox + (long long)s * sc.shell_texels);
    hs.idx[0] = base + r0 * sc.We + c0;
    hs.idx[1] = base + r0 * sc.We + c1;
    hs.idx[2] = base + (r0 + 1) * sc.We + c0;
    hs.idx[3] = base + (r0 + 1) * sc.We + c1;
    hs.w[0] = (1.0f - fu) * (1.0f - fv);
    hs.w[1] = fu * (1.0f - fv);
    hs.w[2] = (1.0f - fu) * fv;
    hs.w[3] = fu * fv;
    return true;
}

template <typename T>
__device__ __forceinline__ float4 interp_shell(const T* x, const ShellHit& hs) {
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float4 a = Store<T>::ld(x, hs.idx[q]);
        acc.x = fmaf(hs.w[q], a.x, acc.x);
        acc.y = fmaf(hs.w[q], a.y, acc.y);
        acc.z = fmaf(hs.w[q], a.z, acc.z);
        acc.w = fmaf(hs.w[q], a.w, acc.w);
    }
    return acc;
}

__device__ __forceinline__ void interp_shell_pair(const PairF32* xp, const ShellHit& hs,
                                                  float4& a, float4& q) {
    a = make_float4(0.f, 0.f, 0.f, 0.f);
    q = a;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        float4 u, w;
        ld_pair(xp, hs.idx[k], u, w);
        a.x = fmaf(hs.w[k], u.x, a.x);
        a.y = fmaf(hs.w[k], u.y, a.y);
        a.z = fmaf(hs.w[k], u.z, a.z);
        a.w = fmaf(hs.w[k], u.w, a.w);
        q.x = fmaf(hs.w[k], w.x, q.x);
        q.y = fmaf(hs.w[k], w.y, q.y);
        q.z = fmaf(hs.w[k], w.z, q.z);
        q.w = fmaf(hs.w[k], w.w, q.w);
    }
}

// FP64 block reduction into one device double (one atomic per block).
template <int NWARPS>
__device__ __forceinline__ void block_add_f64(double v, double* dst) {
    __shared__ double red[NWARPS];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < NWARPS ? red[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0 && v != 0.0) atomicAdd(dst, v);
    }
    __syncthreads();   // red[] may be reused by a following call
}

}  // namespace perf

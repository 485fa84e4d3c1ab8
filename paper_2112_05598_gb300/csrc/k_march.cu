// k_march.cu -- ray-march kernels of the PERF Gauss-Newton step (sm_103a).
//
//   k_forward     Eq. 3-4 composite: image, residual r = H^ - C, F (Eq. 5-6)
//   k_jvp         J p by the back-to-front recurrence of Algorithm 1
//   k_scatter     J^T v, the fused A p = J^T (J p), and diag(J^T J) with J^T r
//                 (the latter also fills the per-sample coefficient store)
//   k_apply_coef  A p from the coefficient store of the Gauss-Newton step
//   *_batch       the same over many scenes from a work queue
//
// Derivatives (Algorithm 1, Section "Computation of partial derivatives"):
// for sample i with optical thickness s_i = sigma_i dbar_i, transmittance
// T_i = e^{-V_i} (V_i = sum_{j<i} s_j), alpha_i = 1 - e^{-s_i} and weight
// w_i = T_i alpha_i,
//   dH/dc_i       = w_i
//   dH_k/dsigma_i = dbar_i (T_i e^{-s_i} c_ik - G_ik),  G_i = sum_{j>i} w_j c_j.
// The scatter kernels take Algorithm 1's order: a first front-to-back sweep
// gives the total optical depth V (grid samples and shell hits), then a
// back-to-front sweep subtracts s_i from V (so e^{-V} = T_i) and accumulates
// G after each use.  G is a sum of non-negative terms, so every partial has
// full relative accuracy even where T_i is tiny -- which matters because the
// Jacobi preconditioner rescales every parameter to unit diagonal.  V is kept
// as an unevaluated FP32 sum (hi + lo, TwoSum) so that T_i stays accurate in
// front of optically deep media.
//
// Scatter: consecutive samples of one ray share most of their 8 trilinear
// voxels.  A register window of the 2x2x2 voxels of the current sample keeps
// one running sum per voxel; a voxel is flushed when the window slides past
// it.  A voxel's trilinear support is a box, so the samples of one ray that
// touch it are consecutive and each voxel is flushed exactly once per ray --
// which also makes the window compute the EXACT diag(J^T J): a row's entry for
// a voxel is complete before it is squared (Section "Preconditioner").
// Window slots are indexed by the parity of the voxel's coordinates, and the
// sample loop is warp-uniform, so lanes of a warp (an 8x4 pixel tile) that
// evict the same voxel in the same iteration do it in the same 16-byte
// vector atomic, which the load/store unit merges.  (Measured: neighbouring
// rays reach a shared voxel at different sample indices often enough that
// the vector atomics still cost about one L1 wavefront per lane and voxel;
// they are the limiter of the A p kernels.)
#include <type_traits>
#include "perf_device.cuh"
#include "perf_kernels.h"

namespace perf {

constexpr int kThreads = 128;
constexpr int kWarps = kThreads / 32;
// Build-time tuning of the ray-march kernels: reuse of gathered corner values
// of x (PERF_CACHE_X) and of p (PERF_CACHE_P) between samples, and the
// minimum resident CTAs per SM requested from the register allocator.  Reuse
// is off by default: on GB300 it raised the A p kernel from 128 to 238
// registers and ran slower (37.5 ms plain vs 50.7-71.6 ms with reuse on
// 20 cameras of the 128^3 workload).
#ifndef PERF_CACHE_X
#define PERF_CACHE_X 0
#endif
#ifndef PERF_CACHE_P
#define PERF_CACHE_P 0
#endif
#ifndef PERF_MIN_CTAS
#define PERF_MIN_CTAS 1
#endif
// The A p kernels ask for 5 resident CTAs per SM (96 registers; a few spill
// slots): on GB300 at 128^3, 100 cameras, 167 ms per launch against 175 ms
// with the allocator unconstrained (150 registers, 3 CTAs) and 169 ms at 4.
#ifndef PERF_APPLY_MIN_CTAS
#define PERF_APPLY_MIN_CTAS 5
#endif

// Corner interpolation with (Corners) or without (plain gathers) reuse.
template <typename T, bool CACHE>
struct Interp {
    Corners<T> c;
    __device__ __forceinline__ void reset() { if (CACHE) c.reset(); }
    __device__ __forceinline__ float4 at(const T* __restrict__ x, const DevScene& sc, const Cell& cl) {
        return CACHE ? c.interp(x, sc, cl) : interp_grid(x, sc, cl);
    }
};
constexpr unsigned kFull = 0xffffffffu;

// ------------------------------------------------------------------ helpers

// Per-ray intermediates (targets, residuals) are stored in the scene's type.
__device__ __forceinline__ float ldv(const float* p, long long i) { return p[i]; }
__device__ __forceinline__ float ldv(const __nv_bfloat16* p, long long i) { return __bfloat162float(p[i]); }
__device__ __forceinline__ void stv(float* p, long long i, float v) { p[i] = v; }
__device__ __forceinline__ void stv(__nv_bfloat16* p, long long i, float v) { p[i] = __float2bfloat16_rn(v); }

// 1 - e^{-x} with full relative accuracy: for |x| < 1/4 the Taylor series
// x (1 - x/2 (1 - x/3 (1 - x/4 (1 - x/5 (1 - x/6 (1 - x/7)))))) (truncation
// below 2e-9 relative), elsewhere 1 - e (no cancellation there).
__device__ __forceinline__ float one_minus_exp_neg(float x, float e) {
    if (fabsf(x) < 0.25f) {
        float p = fmaf(-x, 1.0f / 7.0f, 1.0f);
        p = fmaf(-x * (1.0f / 6.0f), p, 1.0f);
        p = fmaf(-x * (1.0f / 5.0f), p, 1.0f);
        p = fmaf(-x * (1.0f / 4.0f), p, 1.0f);
        p = fmaf(-x * (1.0f / 3.0f), p, 1.0f);
        p = fmaf(-x * 0.5f, p, 1.0f);
        return x * p;
    }
    return 1.0f - e;
}

// Compensated running sum (Knuth's TwoSum): value = hi + lo.
struct CSum {
    float hi, lo;
};
__device__ __forceinline__ void csum_add(CSum& s, float a) {
    const float t = __fadd_rn(s.hi, a);
    const float bp = __fsub_rn(t, s.hi);
    const float err = __fadd_rn(__fsub_rn(s.hi, __fsub_rn(t, bp)), __fsub_rn(a, bp));
    s.hi = t;
    s.lo = __fadd_rn(s.lo, err);
}

// Running composite of one ray.  The transmittance is e^{-V} with V the
// optical depth so far, kept as a compensated sum, rather than a running
// product: a product of several hundred rounded factors drifts by up to
// ~1e-4 relative on the longest rays, e^{-V} stays within a few ulps.
struct Comp {
    float T, H[3];
    CSum V;
};

__device__ __forceinline__ void comp_reset(Comp& s) {
    s.T = 1.0f;
    s.H[0] = s.H[1] = s.H[2] = 0.0f;
    s.V.hi = s.V.lo = 0.0f;
}

__device__ __forceinline__ void comp_step(Comp& s, const float4 a, float dbar) {
    const float sd = __fmul_rn(a.w, dbar);
    const float e = expf(-sd);
    const float w = __fmul_rn(s.T, one_minus_exp_neg(sd, e));
    s.H[0] = fmaf(w, a.x, s.H[0]);
    s.H[1] = fmaf(w, a.y, s.H[1]);
    s.H[2] = fmaf(w, a.z, s.H[2]);
    csum_add(s.V, sd);
    s.T = expf(-fmaxf(s.V.hi + s.V.lo, 0.0f));
}

// Eq. 3-4 over the grid samples and then the shells.  cut > 0: the
// rendering threshold of Section "Rendering" -- a ray whose total opacity
// within the volume, 1 - T_exit, is below cut sees the volume as fully
// transparent (only the shells).
template <typename T>
__device__ __forceinline__ void composite(const DevScene& sc, const T* __restrict__ x,
                                          const Ray& R, long long ray, Comp& s, float& T_exit,
                                          float cut = 0.0f) {
    comp_reset(s);
    const float dbar = R.delta * sc.halfG;
    Interp<T, PERF_CACHE_X != 0> cx;
    cx.reset();
    for (int k = 0; k < R.K; ++k) {
        const Cell cl = sample_cell(sc, R, ray, k);
        comp_step(s, cx.at(x, sc, cl), dbar);
    }
    T_exit = s.T;
    if (cut > 0.0f && 1.0f - s.T < cut) comp_reset(s);
    for (int q = 0; q < sc.S; ++q) {
        ShellHit hs;
        if (shell_lookup(sc, R, ray, q, hs)) comp_step(s, interp_shell(x, hs), 1.0f);
    }
}

// Total optical depth of a ray (grid samples, then shell hits), compensated;
// *Vg (may be null) gets the grid part.
template <typename T>
__device__ __forceinline__ CSum optical_depth(const DevScene& sc, const T* __restrict__ x,
                                              const Ray& R, long long ray, CSum* Vg = nullptr) {
    CSum V = {0.0f, 0.0f};
    const float dbar = R.delta * sc.halfG;
    Interp<T, PERF_CACHE_X != 0> cx;
    cx.reset();
    for (int k = 0; k < R.K; ++k) {
        const Cell cl = sample_cell(sc, R, ray, k);
        csum_add(V, __fmul_rn(cx.at(x, sc, cl).w, dbar));
    }
    if (Vg) *Vg = V;
    for (int q = 0; q < sc.S; ++q) {
        ShellHit hs;
        if (shell_lookup(sc, R, ray, q, hs)) csum_add(V, interp_shell(x, hs).w);
    }
    return V;
}

// J p of one ray (V: the total optical depth from the first sweep; with
// paired storage x holds both operands and p is not read) by
// Algorithm 1's back-to-front recurrence: the same w_i and dH/dsigma_i as
// the scatter sweep (backward_sweep), with the same operations in the same
// order, so that J p and J^T v apply one matrix and its transpose and the
// fused A p = J^T (J p) is symmetric.  A forward tangent sweep of Eq. 3 gives
// the same J p in exact arithmetic, but its binary32 rounding differs from
// the scatter's: behind opaque media dH/dsigma_i is a small difference of
// two nearly equal terms, so along Jacobi-scaled directions (which blow up
// barely observed parameters) the two roundings disagree by up to ~10% in
// v.(J p) against p.(J^T v), and CG stalls.  psum = the sum of p~sigma over
// the grid samples (the auxiliary row's J p is proportional to it).
template <typename T, typename TP>
__device__ __forceinline__ void jvp_backward(const DevScene& sc, const T* __restrict__ x,
                                             const TP* __restrict__ p, const Ray& R, long long ray,
                                             CSum V, float (&J)[3], float& psum) {
    float G[3] = {0.0f, 0.0f, 0.0f};
    J[0] = J[1] = J[2] = 0.0f;
    psum = 0.0f;
    for (int q = sc.S - 1; q >= 0; --q) {
        ShellHit hs;
        if (!shell_lookup(sc, R, ray, q, hs)) continue;
        float4 a, pv;
        if constexpr (std::is_same<T, PairF32>::value) {
            interp_shell_pair(x, hs, a, pv);
        } else {
            a = interp_shell(x, hs);
            pv = interp_shell(p, hs);
        }
        const float sd = a.w;
        csum_add(V, -sd);
        const float Ti = expf(-fmaxf(V.hi + V.lo, 0.0f));
        const float e = expf(-sd);
        const float wi = Ti * one_minus_exp_neg(sd, e);
        const float te = Ti * e;
        const float ds0 = te * a.x - G[0], ds1 = te * a.y - G[1], ds2 = te * a.z - G[2];
        G[0] = fmaf(wi, a.x, G[0]);
        G[1] = fmaf(wi, a.y, G[1]);
        G[2] = fmaf(wi, a.z, G[2]);
        J[0] = fmaf(wi, pv.x, fmaf(ds0, pv.w, J[0]));
        J[1] = fmaf(wi, pv.y, fmaf(ds1, pv.w, J[1]));
        J[2] = fmaf(wi, pv.z, fmaf(ds2, pv.w, J[2]));
    }
    const float dbar = R.delta * sc.halfG;
    for (int k = R.K - 1; k >= 0; --k) {
        const Cell cl = sample_cell(sc, R, ray, k);
        float4 a, pv;
        if constexpr (std::is_same<T, PairF32>::value) {
            interp_grid_pair(x, sc, cl, a, pv);
        } else {
            a = interp_grid(x, sc, cl);
            pv = interp_grid(p, sc, cl);
        }
        const float sd = __fmul_rn(a.w, dbar);
        csum_add(V, -sd);
        const float Ti = expf(-fmaxf(V.hi + V.lo, 0.0f));
        const float e = expf(-sd);
        const float wi = Ti * one_minus_exp_neg(sd, e);
        const float te = Ti * e;
        const float ds0 = dbar * (te * a.x - G[0]);
        const float ds1 = dbar * (te * a.y - G[1]);
        const float ds2 = dbar * (te * a.z - G[2]);
        G[0] = fmaf(wi, a.x, G[0]);
        G[1] = fmaf(wi, a.y, G[1]);
        G[2] = fmaf(wi, a.z, G[2]);
        J[0] = fmaf(wi, pv.x, fmaf(ds0, pv.w, J[0]));
        J[1] = fmaf(wi, pv.y, fmaf(ds1, pv.w, J[1]));
        J[2] = fmaf(wi, pv.z, fmaf(ds2, pv.w, J[2]));
        psum += pv.w;
    }
}

// ------------------------------------------------------- voxel window

__device__ __forceinline__ void red_add4(float* base, int blk, float4 v) {
    atomicAdd(reinterpret_cast<float4*>(base) + blk, v);
}

// The 2x2x2 window of the current sample holds exactly one voxel of each
// coordinate-parity class, so slot p (bit a = parity along axis a) always
// holds the window's voxel of parity p.  A voxel therefore sits in the same
// slot on every lane of the warp, and lanes that evict it in the same
// iteration do so in the same vector atomic, which the hardware merges.
template <int NV>
struct Window {
    float v[8][NV];
    int b[3];
};


// Index of a voxel / texel block in a scatter target.
struct CanonKey {
    int G;
    __device__ __forceinline__ int key(int x, int y, int z) const { return (z * G + y) * G + x; }
    __device__ __forceinline__ int shell(int idx) const { return idx; }
};

// VJP sink: slot = (a, s) with a = sum W w_i and s = sum W v.dH/dsigma_i;
// the parameter block receives (a v_0, a v_1, a v_2, s).  put() is called by
// all 32 lanes of a warp together; with cnt set (instrumentation) it also
// counts the vector-atomic lane operations it issues (COUNT: a separate
// instantiation, so that the timed kernels carry no trace of it).
template <class Key, bool COUNT = false>
struct VjpSink {
    float* out;
    float v0, v1, v2;
    Key km;
    unsigned long long* cnt;
    __device__ __forceinline__ void put(bool ev, int key, const float (&a)[2]) {
        const bool red = ev && (a[0] != 0.0f || a[1] != 0.0f);
        if constexpr (COUNT) {
            const unsigned b = __ballot_sync(kFull, red);
            if ((threadIdx.x & 31) == 0 && b) atomicAdd(cnt, (unsigned long long)__popc(b));
        }
        if (red) red_add4(out, key, make_float4(a[0] * v0, a[0] * v1, a[0] * v2, a[1]));
    }
};

// Diagonal sink: slot = (a, s_0, s_1, s_2[, s_3]), the ray's row entries for
// the voxel (colour: a for each channel's residual; opacity: s_k for residual
// k; s_3 for the auxiliary residual when NV = 5), squared into diag and
// multiplied by r into the gradient.
// With `cross`, also the off-diagonal entries of the voxel's 4x4 block of
// J^T J: (colour k, opacity) = sum_rays a s_k (colour-colour entries vanish,
// and colour does not enter the auxiliary residual).
template <int NV, class Key = CanonKey>
struct DiagSink {
    float* diag;
    float* grad;
    float* cross;
    float r0, r1, r2;
    long long n_vox;
    Key km;                   // the block order of diag, grad and cross
    float r3;
    __device__ __forceinline__ void put(bool ev, int key, const float (&a)[NV]) {
        const float s3 = NV == 5 ? a[(NV - 1) % NV] : 0.0f;
        if (!(ev && (a[0] != 0.0f || a[1] != 0.0f || a[2] != 0.0f || a[3] != 0.0f || s3 != 0.0f)))
            return;
        const float aa = a[0] * a[0];
        red_add4(diag, key, make_float4(aa, aa, aa, a[1] * a[1] + a[2] * a[2] + a[3] * a[3] + s3 * s3));
        if (grad)
            red_add4(grad, key, make_float4(a[0] * r0, a[0] * r1, a[0] * r2,
                                            a[1] * r0 + a[2] * r1 + a[3] * r2 + s3 * r3));
        if (cross && key < n_vox) red_add4(cross, key, make_float4(a[0] * a[1], a[0] * a[2], a[0] * a[3], 0.0f));
    }
};

// Move the window (all lanes; `on` = this lane moves) to base nb, handing the
// voxels that leave it to the sink.  A voxel never re-enters a ray's window:
// its trilinear support meets the ray in one run of samples.  Every slot is
// tested on every lane (predicated, no branches): skipping the slots no lane
// evicts behind a warp-uniform mask measured slower on GB300 (89.7 vs 84.4 ms
// per A p at 128^3), since the warp's lanes together evict most slots.
template <int NV, class Sink>
__device__ __forceinline__ void win_move(Window<NV>& w, const int (&nb)[3], bool on, int G, Sink& sk) {
#pragma unroll
    for (int p = 0; p < 8; ++p) {
        const int ox = par_coord(w.b[0], p & 1), oy = par_coord(w.b[1], (p >> 1) & 1),
                  oz = par_coord(w.b[2], p >> 2);
        const int nx = par_coord(nb[0], p & 1), ny = par_coord(nb[1], (p >> 1) & 1),
                  nz = par_coord(nb[2], p >> 2);
        const bool ev = on && (ox != nx || oy != ny || oz != nz);
        sk.put(ev, sk.km.key(ox, oy, oz), w.v[p]);
        if (ev) {
#pragma unroll
            for (int q = 0; q < NV; ++q) w.v[p][q] = 0.0f;
        }
    }
    if (on) { w.b[0] = nb[0]; w.b[1] = nb[1]; w.b[2] = nb[2]; }
}

// Add a sample's contribution val (per unit weight) to the 8 window voxels.
template <int NV>
__device__ __forceinline__ void win_add(Window<NV>& w, const Cell& cl, const float (&val)[NV]) {
    // weight of the corner whose parity is p: corner offset = p ^ (base parity)
    const bool sx = cl.bx & 1, sy = cl.by & 1, sz = cl.bz & 1;
    const float wx[2] = {sx ? cl.fx : 1.0f - cl.fx, sx ? 1.0f - cl.fx : cl.fx};
    const float wy[2] = {sy ? cl.fy : 1.0f - cl.fy, sy ? 1.0f - cl.fy : cl.fy};
    const float wz[2] = {sz ? cl.fz : 1.0f - cl.fz, sz ? 1.0f - cl.fz : cl.fz};
#pragma unroll
    for (int p = 0; p < 8; ++p) {
        const float W = wx[p & 1] * wy[(p >> 1) & 1] * wz[p >> 2];
#pragma unroll
        for (int q = 0; q < NV; ++q) w.v[p][q] = fmaf(W, val[q], w.v[p][q]);
    }
}

// Back-to-front sweep of Algorithm 1 for the 32 rays of a warp (all lanes
// call it; `act` marks lanes with a ray to scatter).  V = total optical depth
// from the first sweep; vv = the ray's weights on its three residuals (VJP:
// v; diagonal: r).  NV = 2 (VJP), 4 (diagonal) or 5 (diagonal with the
// auxiliary row).  aux_v: the auxiliary residual's opacity derivative per
// unit interpolation weight, the same for every grid sample of the ray
// (8 lambda (T^ - 1/2) T^ dbar), times v_aux for the VJP.  The loop over
// samples is warp-uniform (sample k of every lane in the same iteration), so
// coherent rays evict a shared voxel in the same instruction.
template <int NV, typename T, class Sink>
__device__ __forceinline__ int backward_sweep(const DevScene& sc, const T* __restrict__ x,
                                              const Ray& R, long long ray, bool act, CSum V,
                                              const float (&vv)[3], Sink& sk,
                                              float4* __restrict__ crow = nullptr,
                                              float aux_v = 0.0f) {
    float G[3] = {0.0f, 0.0f, 0.0f};
    const int Kl = act ? R.K : 0;
    const int Kmax = __reduce_max_sync(kFull, Kl);
    // kf: 1 + the largest k whose coefficient row is non-zero (0: none yet;
    // the sweep runs back to front).  With the auxiliary residual's per-sample
    // term in play (aux_v != 0) every row counts.
    int kf = (NV == 5 && aux_v != 0.0f) ? Kl : 0;
    const bool skip_zero_tail = crow != nullptr && sc.keff != nullptr;
    // the auxiliary row's per-ray factor goes to the store's last row
    if (NV == 5 && crow && act) __stcs(crow + (long long)(Kmax + sc.S) * 32,
                                       make_float4(aux_v, 0.0f, 0.0f, 0.0f));
    // shells, outermost first
    for (int q = sc.S - 1; q >= 0; --q) {
        ShellHit hs;
        const bool hit = act && shell_lookup(sc, R, ray, q, hs);
        float wi = 0.0f, ds[3] = {0.0f, 0.0f, 0.0f};
        if (hit) {
            const float4 a = interp_shell(x, hs);
            const float sd = a.w;
            csum_add(V, -sd);
            const float Ti = expf(-fmaxf(V.hi + V.lo, 0.0f));
            const float e = expf(-sd);
            wi = Ti * one_minus_exp_neg(sd, e);
            const float te = Ti * e;
            ds[0] = te * a.x - G[0];
            ds[1] = te * a.y - G[1];
            ds[2] = te * a.z - G[2];
            G[0] = fmaf(wi, a.x, G[0]);
            G[1] = fmaf(wi, a.y, G[1]);
            G[2] = fmaf(wi, a.z, G[2]);
            if (crow) __stcs(crow + (long long)(Kmax + q) * 32, make_float4(wi, ds[0], ds[1], ds[2]));
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float W = hit ? hs.w[c] : 0.0f;
            float val[NV];
            val[0] = W * wi;
            if (NV == 2) {
                val[1 % NV] = W * (vv[0] * ds[0] + vv[1] * ds[1] + vv[2] * ds[2]);
            } else {
                val[1 % NV] = W * ds[0];
                val[2 % NV] = W * ds[1];
                val[3 % NV] = W * ds[2];
                if (NV == 5) val[(NV - 1) % NV] = 0.0f;
            }
            sk.put(hit, hit ? sk.km.shell(hs.idx[c]) : 0, val);
        }
    }
    // grid samples, last to first (warp-uniform loop; lane active while k < K)
    const float dbar = R.delta * sc.halfG;
    Window<NV> w;
#pragma unroll
    for (int c = 0; c < 8; ++c)
#pragma unroll
        for (int q = 0; q < NV; ++q) w.v[c][q] = 0.0f;
    w.b[0] = w.b[1] = w.b[2] = 0;
    Interp<T, PERF_CACHE_X != 0> cx;
    cx.reset();
    for (int k = Kmax - 1; k >= 0; --k) {
        const bool on = k < Kl;
        Cell cl;
        cl.bx = w.b[0]; cl.by = w.b[1]; cl.bz = w.b[2];
        cl.fx = cl.fy = cl.fz = 0.0f;
        if (on) {
            cl = sample_cell(sc, R, ray, k);
            if (k == Kl - 1) { w.b[0] = cl.bx; w.b[1] = cl.by; w.b[2] = cl.bz; }
        }
        const int nb[3] = {cl.bx, cl.by, cl.bz};
        win_move(w, nb, on, sc.G, sk);
        if (on) {
            const float4 a = cx.at(x, sc, cl);
            const float sd = __fmul_rn(a.w, dbar);
            csum_add(V, -sd);
            const float Ti = expf(-fmaxf(V.hi + V.lo, 0.0f));
            const float e = expf(-sd);
            const float wi = Ti * one_minus_exp_neg(sd, e);
            const float te = Ti * e;
            const float ds0 = dbar * (te * a.x - G[0]);
            const float ds1 = dbar * (te * a.y - G[1]);
            const float ds2 = dbar * (te * a.z - G[2]);
            G[0] = fmaf(wi, a.x, G[0]);
            G[1] = fmaf(wi, a.y, G[1]);
            G[2] = fmaf(wi, a.z, G[2]);
            if (kf == 0 && (wi != 0.0f || ds0 != 0.0f || ds1 != 0.0f || ds2 != 0.0f)) kf = k + 1;
            if (crow && (kf > 0 || !skip_zero_tail))
                __stcs(crow + (long long)k * 32, make_float4(wi, ds0, ds1, ds2));
            float val[NV];
            val[0] = wi;
            if (NV == 2) {
                val[1 % NV] = vv[0] * ds0 + vv[1] * ds1 + vv[2] * ds2 + aux_v;
            } else {
                val[1 % NV] = ds0;
                val[2 % NV] = ds1;
                val[3 % NV] = ds2;
                if (NV == 5) val[(NV - 1) % NV] = aux_v;
            }
            win_add(w, cl, val);
        }
    }
    // the remaining window
#pragma unroll
    for (int p = 0; p < 8; ++p)
        sk.put(Kl > 0, sk.km.key(par_coord(w.b[0], p & 1), par_coord(w.b[1], (p >> 1) & 1),
                                 par_coord(w.b[2], p >> 2)),
               w.v[p]);
    return kf;
}

// ------------------------------------------------------------- kernels

// Per-tile bodies: one warp marches the 32 rays of one pixel tile.  The
// single-scene kernels stride over tiles; the batched kernels take tiles of
// many scenes from a work queue.

template <typename T, int MODE>   // 0 render, 1 residual (+F), 2 F only
__device__ __forceinline__ void forward_tile(const DevScene& sc, const T* __restrict__ x,
                                             const T* __restrict__ target, float* __restrict__ img,
                                             T* __restrict__ res, float* __restrict__ T_out,
                                             long long tile, int lane, double& facc,
                                             float cut = 0.0f) {
    long long ray;
    if (!tile_pixel(sc, tile, lane, ray)) return;
    Ray R;
    ray_setup(sc, ray, R);
    Comp s;
    float Te;
    composite(sc, x, R, ray, s, Te, MODE == 0 ? cut : 0.0f);
    if (MODE == 0) {
        img[3 * ray + 0] = s.H[0];
        img[3 * ray + 1] = s.H[1];
        img[3 * ray + 2] = s.H[2];
        if (T_out) T_out[ray] = Te;
    } else {
        const long long R3 = 3 + sc.aux;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float r = s.H[k] - ldv(target, 3 * ray + k);
            if (MODE == 1 && res) stv(res, R3 * ray + k, r);
            facc += 0.5 * (double)r * (double)r;
        }
        if (sc.aux) {   // Section "Auxiliary terms": L = lambda (1 - 4 (T^ - 1/2)^2)
            const float d = Te - 0.5f;
            const float L = sc.aux_lambda * (1.0f - 4.0f * d * d);
            if (MODE == 1 && res) stv(res, R3 * ray + 3, L);
            facc += 0.5 * (double)L * (double)L;
        }
    }
}

// All 32 lanes call it (the back-to-front sweep is warp-synchronous).
// LAY (MODE 2): the diagonal, gradient and couplings go to the block order of
// sc's LayoutKey (a brick order when a Gauss-Newton step's PCG vectors are
// bricked); otherwise canonical.
template <typename T, typename TP, int MODE, typename TV,   // 0 vjp, 1 apply A, 2 diag (+grad)
          bool COUNT = false, bool LAY = false>
__device__ __forceinline__ void scatter_tile(const DevScene& sc, const T* __restrict__ x,
                                             const TP* __restrict__ p, const TV* __restrict__ v,
                                             float* __restrict__ out, float* __restrict__ out2,
                                             float* __restrict__ out3, long long tile, int lane,
                                             double& acc, float4* __restrict__ coef = nullptr,
                                             const long long* __restrict__ tile_off = nullptr,
                                             long long coef_tiles = 0) {
    long long ray = 0;
    bool act = tile_pixel(sc, tile, lane, ray);
    Ray R;
    R.K = 0;
    R.shell_hit = 0u;
    R.delta = 0.0f;
    float vr[3] = {0.0f, 0.0f, 0.0f};
    float va = 0.0f, kap = 0.0f;   // auxiliary residual: its weight, and its d/dsigma per unit W
    CSum V = {0.0f, 0.0f};
    if (act) {
        ray_setup(sc, ray, R);
        const float dbar = R.delta * sc.halfG;
        if (MODE == 1) {
            // A p: first sweep V, second J p by Algorithm 1 (see jvp_backward),
            // third the scatter below
            CSum Vg = {0.0f, 0.0f};
            V = optical_depth(sc, x, R, ray, &Vg);
            float psum;
            jvp_backward(sc, x, p, R, ray, V, vr, psum);
            if (sc.aux) {   // L = lambda (1 - 4 (T^ - 1/2)^2): dL/dsigma_i = kap per unit weight
                const float Te = expf(-fmaxf(Vg.hi + Vg.lo, 0.0f));
                kap = 8.0f * sc.aux_lambda * (Te - 0.5f) * Te * dbar;
                va = kap * psum;
            }
            acc += (double)vr[0] * vr[0] + (double)vr[1] * vr[1] + (double)vr[2] * vr[2] +
                   (double)va * va;
        } else {
            const int R3 = 3 + sc.aux;
            if (MODE == 0 || v != nullptr) {
                vr[0] = ldv(v, (long long)R3 * ray);
                vr[1] = ldv(v, (long long)R3 * ray + 1);
                vr[2] = ldv(v, (long long)R3 * ray + 2);
                if (sc.aux) va = ldv(v, (long long)R3 * ray + 3);
            }
            if (MODE == 2 || vr[0] != 0.0f || vr[1] != 0.0f || vr[2] != 0.0f || va != 0.0f) {
                CSum Vg = {0.0f, 0.0f};
                V = optical_depth(sc, x, R, ray, &Vg);
                if (sc.aux) {
                    const float Te = expf(-fmaxf(Vg.hi + Vg.lo, 0.0f));
                    kap = 8.0f * sc.aux_lambda * (Te - 0.5f) * Te * dbar;
                }
            }
        }
        if (MODE != 2 && vr[0] == 0.0f && vr[1] == 0.0f && vr[2] == 0.0f && va == 0.0f) act = false;
    }
    float4* crow = (MODE == 2 && coef && tile < coef_tiles) ? coef + tile_off[tile] * 32 + lane : nullptr;
    using DKey = typename std::conditional<LAY, LayoutKey, CanonKey>::type;
    DKey dk;
    if constexpr (LAY) dk = layout_key(sc);
    else dk = CanonKey{sc.G};
    if (MODE == 2) {
        int kf;
        if (sc.aux) {
            DiagSink<5, DKey> sk{out, out2, out3, vr[0], vr[1], vr[2], sc.n_vox, dk, va};
            kf = backward_sweep<5>(sc, x, R, ray, act, V, vr, sk, crow, kap);
        } else {
            DiagSink<4, DKey> sk{out, out2, out3, vr[0], vr[1], vr[2], sc.n_vox, dk, 0.0f};
            kf = backward_sweep<4>(sc, x, R, ray, act, V, vr, sk, crow);
        }
        if (crow && act && sc.keff) sc.keff[ray] = kf;
    } else {
        VjpSink<CanonKey, COUNT> sk{out, vr[0], vr[1], vr[2], CanonKey{sc.G}, sc.red_count};
        backward_sweep<2>(sc, x, R, ray, act, V, vr, sk, nullptr, va * kap);
    }
}

#define PERF_TILE_LOOP                                                              \
    const int lane = threadIdx.x & 31;                                              \
    const long long nw = (long long)gridDim.x * kWarps;                             \
    for (long long tile = sc.tile_lo + (long long)blockIdx.x * kWarps + (threadIdx.x >> 5); \
         tile < sc.n_tiles; tile += nw)

template <typename T, int MODE>
__global__ void __launch_bounds__(kThreads) k_forward(DevScene sc, const T* __restrict__ x,
                                                      const T* __restrict__ target,
                                                      float* __restrict__ img,
                                                      T* __restrict__ res,
                                                      float* __restrict__ T_out, double* F,
                                                      float cut) {
    double facc = 0.0;
    PERF_TILE_LOOP { forward_tile<T, MODE>(sc, x, target, img, res, T_out, tile, lane, facc, cut); }
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
        CSum Vg = {0.0f, 0.0f};
        const CSum V = optical_depth(sc, x, R, ray, &Vg);
        float J[3], psum;
        jvp_backward(sc, x, p, R, ray, V, J, psum);
        const long long R3 = 3 + sc.aux;
        out[R3 * ray + 0] = J[0];
        out[R3 * ray + 1] = J[1];
        out[R3 * ray + 2] = J[2];
        if (sc.aux) {   // dL = -8 lambda (T^ - 1/2) dT^, dT^ = -T^ dbar sum_i p~sigma_i
            const float Te = expf(-fmaxf(Vg.hi + Vg.lo, 0.0f));
            out[R3 * ray + 3] = 8.0f * sc.aux_lambda * (Te - 0.5f) * Te * R.delta * sc.halfG * psum;
        }
    }
}

template <typename T, typename TP, int MODE, typename TV, bool COUNT = false, bool LAY = false>
__global__ void __launch_bounds__(kThreads, MODE == 1 ? PERF_APPLY_MIN_CTAS : PERF_MIN_CTAS)
    k_scatter(DevScene sc, const T* __restrict__ x,
                                                      const TP* __restrict__ p,
                                                      const TV* __restrict__ v,
                                                      float* __restrict__ out,
                                                      float* __restrict__ out2,
                                                      float* __restrict__ out3, double* pap,
                                                      float4* __restrict__ coef,
                                                      const long long* __restrict__ tile_off) {
    double acc = 0.0;
    PERF_TILE_LOOP {
        scatter_tile<T, TP, MODE, TV, COUNT, LAY>(sc, x, p, v, out, out2, out3, tile, lane, acc, coef,
                                             tile_off, sc.coef_tiles);
    }
    if (MODE == 1 && pap) block_add_f64<kWarps>(acc, pap);
}

// ------------------------------------------- coefficient-cached A p
//
// Within one Gauss-Newton step x is fixed, so every sample's derivatives are
// fixed too: J_ray p = sum_i [w_i p~c_i + dH/dsigma_i p~sigma_i] (p~ = p
// interpolated at sample i) and the scatter of J^T v uses the same
// (w_i, dH/dsigma_i).  The diagonal march of the step (Algorithm 1, run once)
// stores these four numbers per sample; each PCG iteration's A p then
// gathers only p and streams the coefficients -- no interpolation of x,
// no exponentials, no transmittance recurrence.
//
// Store layout: per pixel tile, rows of 32 float4 (one per lane): rows
// 0..Kmax-1 the grid samples (Kmax = the tile's largest sample count), then
// one row per shell.  tile_off[t] = first row of tile t (exclusive prefix sum
// of Kmax + S over tiles).  Entries of samples a lane does not have (k >= K,
// a shell it misses) are never read.

// rows[t] = Kmax of tile t + S (+ 1: the auxiliary residual's per-ray factor).
// Shell-hit table: entry (ray, s) for every ray of [ray_lo, ray_lo + n) and
// shell s it hits (others are left untouched and never read).
__global__ void __launch_bounds__(kThreads) k_shell_table(DevScene sc, long long ray_lo,
                                                          long long n, float4* tab) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long ray = ray_lo + i;
        Ray R;
        ray_setup(sc, ray, R);
        for (int s = 0; s < sc.S; ++s)
            if (R.shell_hit & (1u << s)) tab[ray * sc.S + s] = shell_entry(sc, R, s);
    }
}

__global__ void __launch_bounds__(kThreads) k_tile_rows(DevScene sc, int* rows) {
    PERF_TILE_LOOP {
        long long ray;
        int K = 0;
        if (tile_pixel(sc, tile, lane, ray)) {
            Ray R;
            ray_setup(sc, ray, R);
            K = R.K;
        }
        K = __reduce_max_sync(kFull, K);
        if (lane == 0) rows[tile] = K + sc.S + sc.aux;
    }
}

// Store rows each ray's A p reads (its non-zero prefix) and its grid samples,
// summed over the rays of the tiles [tile_lo, n_tiles): one 64-bit atomic per
// warp and sum.
__global__ void __launch_bounds__(kThreads) k_coef_prefix(DevScene sc, const int* __restrict__ keff,
                                                          unsigned long long* sums) {
    unsigned long long a = 0ull, b = 0ull;
    PERF_TILE_LOOP {
        long long ray;
        if (!tile_pixel(sc, tile, lane, ray)) continue;
        Ray R;
        ray_setup(sc, ray, R);
        a += (unsigned long long)keff[ray];
        b += (unsigned long long)R.K;
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(kFull, a, o);
        b += __shfl_down_sync(kFull, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(sums, a);
        atomicAdd(sums + 1, b);
    }
}

// The coefficient-cached A p of one lane's ray: J p, then the scatter of
// J^T (J p).  Splitting the two halves into two launches, with v = J p of
// every ray stored in between, measured slower on GB300 (102-113 against
// 95.4 ms per launch at 128^3): the scatter half needs as many registers as
// the fused kernel, and one warp's J p no longer overlaps another's scatter.
// BRICK: p and A p are in the block order of sc's LayoutKey (else canonical).
template <typename TP, bool COUNT = false, bool BRICK = false>
__device__ __forceinline__ void coef_apply_tile(const DevScene& sc, const TP* __restrict__ p,
                                                const float4* __restrict__ coef,
                                                const long long* __restrict__ tile_off,
                                                float* __restrict__ out, long long tile, int lane,
                                                double& acc) {
    long long ray = 0;
    bool act = tile_pixel(sc, tile, lane, ray);
    Ray R;
    R.K = 0;
    R.shell_hit = 0u;
    R.delta = 0.0f;
    if (act) {
        ray_setup(sc, ray, R);
        // rows past the non-zero prefix are zeros: J p and the scatter skip them
        if (sc.keff) R.K = min(R.K, sc.keff[ray]);
    }
    const long long r0 = tile_off[tile];
    const int kmax_rows = (int)(tile_off[tile + 1] - r0) - sc.S - sc.aux;
    const float4* crow = coef + r0 * 32 + lane;
    // J p (with the auxiliary residual: kap sum of p~sigma over the grid samples)
    float J[3] = {0.0f, 0.0f, 0.0f};
    float kap = 0.0f, Ja = 0.0f, psum = 0.0f;
    if (act) {
        if (sc.aux) kap = __ldcs(crow + (long long)(kmax_rows + sc.S) * 32).x;
        for (int k = 0; k < R.K; ++k) {
            const float4 c = __ldcs(crow + (long long)k * 32);
            const Cell cl = sample_cell(sc, R, ray, k);
            float4 q;
            if constexpr (BRICK) q = interp_grid_lay(p, layout_key(sc), cl);
            else q = interp_grid(p, sc, cl);
            J[0] = fmaf(c.x, q.x, fmaf(c.y, q.w, J[0]));
            J[1] = fmaf(c.x, q.y, fmaf(c.z, q.w, J[1]));
            J[2] = fmaf(c.x, q.z, fmaf(c.w, q.w, J[2]));
            psum += q.w;
        }
        Ja = kap * psum;
        for (int s = 0; s < sc.S; ++s) {
            ShellHit hs;
            if (shell_lookup(sc, R, ray, s, hs)) {
                const float4 q = interp_shell(p, hs);
                const float4 c = __ldcs(crow + (long long)(kmax_rows + s) * 32);
                J[0] = fmaf(c.x, q.x, fmaf(c.y, q.w, J[0]));
                J[1] = fmaf(c.x, q.y, fmaf(c.z, q.w, J[1]));
                J[2] = fmaf(c.x, q.z, fmaf(c.w, q.w, J[2]));
            }
        }
        acc += (double)J[0] * J[0] + (double)J[1] * J[1] + (double)J[2] * J[2] + (double)Ja * Ja;
        if (J[0] == 0.0f && J[1] == 0.0f && J[2] == 0.0f && Ja == 0.0f) act = false;
    }
    const float aux_v = Ja * kap;   // v_aux dL/dsigma per unit interpolation weight
    // J^T (J p): the scatter of Algorithm 1 with v = J p
    using Key = typename std::conditional<BRICK, LayoutKey, CanonKey>::type;
    Key km;
    if constexpr (BRICK) km = layout_key(sc);
    else km = CanonKey{sc.G};
    VjpSink<Key, COUNT> sk{out, J[0], J[1], J[2], km, sc.red_count};
    for (int s = sc.S - 1; s >= 0; --s) {
        ShellHit hs;
        const bool hit = act && shell_lookup(sc, R, ray, s, hs);
        float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
        if (hit) c = __ldcs(crow + (long long)(kmax_rows + s) * 32);
        const float sv = J[0] * c.y + J[1] * c.z + J[2] * c.w;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float W = hit ? hs.w[k] : 0.0f;
            const float val[2] = {W * c.x, W * sv};
            sk.put(hit, hit ? sk.km.shell(hs.idx[k]) : 0, val);
        }
    }
    const int Kl = act ? R.K : 0;
    const int Kmax = __reduce_max_sync(kFull, Kl);
    Window<2> w;
#pragma unroll
    for (int c = 0; c < 8; ++c) w.v[c][0] = w.v[c][1] = 0.0f;
    w.b[0] = w.b[1] = w.b[2] = 0;
    for (int k = Kmax - 1; k >= 0; --k) {
        const bool on = k < Kl;
        // issued first: its latency overlaps the cell and window work
        const float4 c = on ? __ldcs(crow + (long long)k * 32) : make_float4(0.f, 0.f, 0.f, 0.f);
        Cell cl;
        cl.bx = w.b[0]; cl.by = w.b[1]; cl.bz = w.b[2];
        cl.fx = cl.fy = cl.fz = 0.0f;
        if (on) {
            cl = sample_cell(sc, R, ray, k);
            if (k == Kl - 1) { w.b[0] = cl.bx; w.b[1] = cl.by; w.b[2] = cl.bz; }
        }
        const int nb[3] = {cl.bx, cl.by, cl.bz};
        win_move(w, nb, on, sc.G, sk);
        if (on) {
            const float val[2] = {c.x, J[0] * c.y + J[1] * c.z + J[2] * c.w + aux_v};
            win_add(w, cl, val);
        }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q)
        sk.put(Kl > 0, sk.km.key(par_coord(w.b[0], q & 1), par_coord(w.b[1], (q >> 1) & 1),
                                 par_coord(w.b[2], q >> 2)),
               w.v[q]);
}

template <typename TP, bool COUNT = false, bool BRICK = false>
__global__ void __launch_bounds__(kThreads, PERF_APPLY_MIN_CTAS)
    k_apply_coef(DevScene sc, const TP* __restrict__ p, const float4* __restrict__ coef,
                 const long long* __restrict__ tile_off, float* __restrict__ out, double* pap) {
    double acc = 0.0;
    PERF_TILE_LOOP { coef_apply_tile<TP, COUNT, BRICK>(sc, p, coef, tile_off, out, tile, lane, acc); }
    if (pap) block_add_f64<kWarps>(acc, pap);
}

// ------------------------------------------------------ batched (many scenes)

constexpr int kBatchSmem = 48;   // scene descriptors staged in shared memory

// Next tile of the work queue for this warp (-1: queue empty) and its scene.
__device__ __forceinline__ long long batch_next(unsigned long long* counter, long long total,
                                                const long long* __restrict__ start, int n,
                                                int lane, int& scene) {
    unsigned long long t = 0;
    if (lane == 0) t = atomicAdd(counter, 1ull);
    t = __shfl_sync(kFull, t, 0);
    if ((long long)t >= total) return -1;
    int lo = 0, hi = n - 1;               // last scene with start <= t
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= (long long)t) lo = mid; else hi = mid - 1;
    }
    scene = lo;
    return (long long)t - start[lo];
}

__device__ __forceinline__ const BatchItem* stage_items(const BatchItem* items, int n,
                                                        BatchItem* smem) {
    if (n > kBatchSmem) return items;
    const int words = (int)(n * sizeof(BatchItem) / sizeof(int));
    const int* src = reinterpret_cast<const int*>(items);
    int* dst = reinterpret_cast<int*>(smem);
    for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
    __syncthreads();
    return smem;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// mode 0: image into img; 1: residual into res (+ F per scene); 2: F per scene only.
template <int MODE>
__global__ void __launch_bounds__(kThreads) k_forward_batch(const BatchItem* __restrict__ items,
                                                            const long long* __restrict__ start,
                                                            int n, long long total,
                                                            unsigned long long* counter,
                                                            const float* __restrict__ x,
                                                            const float* __restrict__ target,
                                                            float* __restrict__ res, double* F,
                                                            const int* __restrict__ active,
                                                            float* __restrict__ img) {
    __shared__ BatchItem s_items[kBatchSmem];
    const BatchItem* it = stage_items(items, n, s_items);
    const int lane = threadIdx.x & 31;
    for (;;) {
        int sidx = 0;
        const long long tile = batch_next(counter, total, start, n, lane, sidx);
        if (tile < 0) break;
        if (active && !active[sidx]) continue;
        const BatchItem& b = it[sidx];
        double facc = 0.0;
        forward_tile<float, MODE>(b.sc, x + b.x_off, target ? target + 3 * b.r_off : nullptr,
                                  img ? img + 3 * b.r_off : nullptr,
                                  res ? res + 3 * b.r_off : nullptr, nullptr, tile, lane, facc);
        if (MODE != 0) {
            facc = warp_sum(facc);
            if (lane == 0 && facc != 0.0) atomicAdd(&F[sidx], facc);
        }
    }
}

// mode 1: A p (+ p^T A p per scene into pap[scene * pap_stride]),
// mode 2: diag (+ grad with v = residuals).  pcg (may be null): per-scene
// Algorithm 2 state; tiles of scenes whose solve has exited are skipped (the
// early exit of a graph-captured PCG loop).
template <int MODE, bool LAY = false>
__global__ void __launch_bounds__(kThreads, MODE == 1 ? PERF_APPLY_MIN_CTAS : PERF_MIN_CTAS)
    k_scatter_batch(const BatchItem* __restrict__ items,
                                                            const long long* __restrict__ start,
                                                            int n, long long total,
                                                            unsigned long long* counter,
                                                            const float* __restrict__ x,
                                                            const float* __restrict__ p,
                                                            const float* __restrict__ v,
                                                            float* __restrict__ out,
                                                            float* __restrict__ out2, double* pap,
                                                            int pap_stride,
                                                            const PcgScalars* __restrict__ pcg,
                                                            float4* __restrict__ coef,
                                                            const long long* __restrict__ tile_off) {
    __shared__ BatchItem s_items[kBatchSmem];
    const BatchItem* it = stage_items(items, n, s_items);
    const int lane = threadIdx.x & 31;
    for (;;) {
        int sidx = 0;
        const long long tile = batch_next(counter, total, start, n, lane, sidx);
        if (tile < 0) break;
        if (pcg && pcg[sidx].done) continue;
        const BatchItem& b = it[sidx];
        double acc = 0.0;
        scatter_tile<float, float, MODE, float, false, LAY>(b.sc, x + b.x_off, p ? p + b.x_off : nullptr,
                                                v ? v + 3 * b.r_off : nullptr, out + b.x_off,
                                                out2 ? out2 + b.x_off : nullptr, nullptr, tile,
                                                lane, acc, coef,
                                                tile_off ? tile_off + b.tile_off : nullptr,
                                                b.sc.n_tiles);
        if (MODE == 1) {
            acc = warp_sum(acc);
            if (lane == 0 && acc != 0.0) atomicAdd(&pap[(long long)sidx * pap_stride], acc);
        }
    }
}

// Coefficient-cached A p over a batch (tile_off: rows of the global tile list;
// scenes whose PCG has exited are skipped).  BRICK: each scene's p and A p
// are in the block order of its own LayoutKey (canonical for lay_s = 0).
template <bool BRICK>
__global__ void __launch_bounds__(kThreads, PERF_APPLY_MIN_CTAS)
    k_apply_coef_batch(const BatchItem* __restrict__ items, const long long* __restrict__ start,
                       int n, long long total, unsigned long long* counter,
                       const float* __restrict__ p, const float4* __restrict__ coef,
                       const long long* __restrict__ tile_off, float* __restrict__ out, double* pap,
                       int pap_stride, const PcgScalars* __restrict__ pcg) {
    __shared__ BatchItem s_items[kBatchSmem];
    const BatchItem* it = stage_items(items, n, s_items);
    const int lane = threadIdx.x & 31;
    for (;;) {
        int sidx = 0;
        const long long tile = batch_next(counter, total, start, n, lane, sidx);
        if (tile < 0) break;
        if (pcg && pcg[sidx].done) continue;
        const BatchItem& b = it[sidx];
        double acc = 0.0;
        coef_apply_tile<float, false, BRICK>(b.sc, p + b.x_off, coef, tile_off + b.tile_off,
                                             out + b.x_off, tile, lane, acc);
        acc = warp_sum(acc);
        if (lane == 0 && acc != 0.0) atomicAdd(&pap[(long long)sidx * pap_stride], acc);
    }
}

// rows[t] for every tile t of the batch's global tile list.
__global__ void __launch_bounds__(kThreads) k_tile_rows_batch(const BatchItem* __restrict__ items,
                                                              const long long* __restrict__ start,
                                                              int n, long long total, int* rows) {
    const int lane = threadIdx.x & 31;
    const long long nw = (long long)gridDim.x * kWarps;
    for (long long t = (long long)blockIdx.x * kWarps + (threadIdx.x >> 5); t < total; t += nw) {
        int lo = 0, hi = n - 1;               // last scene with start <= t
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (start[mid] <= t) lo = mid; else hi = mid - 1;
        }
        const DevScene& sc = items[lo].sc;
        long long ray;
        int K = 0;
        if (tile_pixel(sc, t - start[lo], lane, ray)) {
            Ray R;
            ray_setup(sc, ray, R);
            K = R.K;
        }
        K = __reduce_max_sync(kFull, K);
        if (lane == 0) rows[t] = K + sc.S + sc.aux;
    }
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

static int grid_blocks(const void* fn, long long n_tiles, int cap_per_sm = 0) {
    // the SM count of the current device (queried per launch: it may change)
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
        sms = 1;
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kThreads, 0);
    if (occ <= 0) occ = 1;
    if (cap_per_sm > 0 && cap_per_sm < occ) occ = cap_per_sm;
    long long want = (n_tiles + kWarps - 1) / kWarps;
    long long cap = (long long)sms * occ;
    long long b = want < cap ? want : cap;
    return (int)(b > 0 ? b : 1);
}

cudaError_t launch_count_samples(const DevScene& sc, unsigned long long* out, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess || sc.n_tiles <= sc.tile_lo) return e;
    k_count<<<grid_blocks((const void*)k_count, sc.n_tiles - sc.tile_lo), kThreads, 0, st>>>(sc, out);
    count_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_forward_t(const DevScene& sc, const void* x, const void* target, void* out,
                             float* T_out, double* F, int mode, cudaStream_t st, float cut) {
    const T* xx = static_cast<const T*>(x);
    const T* tt = static_cast<const T*>(target);
    if (sc.n_tiles <= sc.tile_lo) return cudaSuccess;
    if (mode == 0) {
        auto fn = k_forward<T, 0>;
        fn<<<grid_blocks((const void*)fn, sc.n_tiles - sc.tile_lo), kThreads, 0, st>>>(
            sc, xx, tt, static_cast<float*>(out), nullptr, T_out, F, cut);
    } else if (mode == 1) {
        auto fn = k_forward<T, 1>;
        fn<<<grid_blocks((const void*)fn, sc.n_tiles - sc.tile_lo), kThreads, 0, st>>>(
            sc, xx, tt, nullptr, static_cast<T*>(out), T_out, F, 0.0f);
    } else {
        auto fn = k_forward<T, 2>;
        fn<<<grid_blocks((const void*)fn, sc.n_tiles - sc.tile_lo), kThreads, 0, st>>>(sc, xx, tt, nullptr,
                                                                           nullptr, T_out, F, 0.0f);
    }
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_forward(const DevScene& sc, int dtype, const void* x, const void* target,
                           void* out, float* T_out, double* F, int mode, cudaStream_t st,
                           float cut) {
    return dtype == 1 ? launch_forward_t<__nv_bfloat16>(sc, x, target, out, T_out, F, mode, st, cut)
                      : launch_forward_t<float>(sc, x, target, out, T_out, F, mode, st, cut);
}

template <typename T, typename TP>
cudaError_t launch_jvp_t(const DevScene& sc, const void* x, const void* p, float* out,
                         cudaStream_t st) {
    if (sc.n_tiles <= sc.tile_lo) return cudaSuccess;
    auto fn = k_jvp<T, TP>;
    fn<<<grid_blocks((const void*)fn, sc.n_tiles - sc.tile_lo), kThreads, 0, st>>>(
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

template <typename T, typename TP, int MODE, typename TV>
cudaError_t launch_scatter_t(const DevScene& sc, const void* x, const void* p, const void* v,
                             float* out, float* out2, double* pap, cudaStream_t st,
                             float* out3 = nullptr, float* coef = nullptr,
                             const long long* tile_off = nullptr) {
    if (sc.n_tiles <= sc.tile_lo) return cudaSuccess;
    auto fn = k_scatter<T, TP, MODE, TV, false>;
    if constexpr (MODE == 1) {   // A p: the counting instantiation when instrumented
        if (sc.red_count) fn = k_scatter<T, TP, MODE, TV, true>;
    }
    if constexpr (MODE == 2) {   // the diagonal in a brick order
        if (sc.lay_s) fn = k_scatter<T, TP, MODE, TV, false, true>;
    }
    fn<<<grid_blocks((const void*)fn, sc.n_tiles - sc.tile_lo, sc.cap_per_sm), kThreads, 0, st>>>(
        sc, static_cast<const T*>(x), static_cast<const TP*>(p), static_cast<const TV*>(v), out,
        out2, out3, pap, reinterpret_cast<float4*>(coef), tile_off);
    count_launch();
    return cudaGetLastError();
}

// v: float32 for the VJP (mode 0); the scene's storage type for the residual
// of the diagonal / gradient (mode 2).
cudaError_t launch_scatter(const DevScene& sc, int dtype, int mode, const void* x, const void* p,
                           int p_dtype, const void* v, float* out, float* out2, double* pap,
                           cudaStream_t st, float* out3, float* coef, const long long* tile_off) {
    typedef __nv_bfloat16 B;
    if (dtype == 1) {
        if (mode == 1)
            return p_dtype == 1 ? launch_scatter_t<B, B, 1, float>(sc, x, p, v, out, out2, pap, st)
                                : launch_scatter_t<B, float, 1, float>(sc, x, p, v, out, out2, pap, st);
        if (mode == 0) return launch_scatter_t<B, float, 0, float>(sc, x, p, v, out, out2, pap, st);
        return launch_scatter_t<B, float, 2, B>(sc, x, p, v, out, out2, pap, st, out3, coef,
                                                tile_off);
    }
    if (mode == 1) return launch_scatter_t<float, float, 1, float>(sc, x, p, v, out, out2, pap, st);
    if (mode == 0) return launch_scatter_t<float, float, 0, float>(sc, x, p, v, out, out2, pap, st);
    return launch_scatter_t<float, float, 2, float>(sc, x, p, v, out, out2, pap, st, out3, coef,
                                                    tile_off);
}

// A p from paired x / p storage (FP32 scenes).
cudaError_t launch_apply_pair(const DevScene& sc, const float* xp, float* out, double* pap,
                              cudaStream_t st) {
    return launch_scatter_t<PairF32, PairF32, 1, float>(sc, xp, xp, nullptr, out, nullptr, pap, st);
}

cudaError_t launch_shell_table(const DevScene& sc, float4* tab, cudaStream_t st) {
    if (sc.S == 0 || sc.n_rays == 0) return cudaSuccess;
    const long long blocks = (sc.n_rays + kThreads - 1) / kThreads;
    const int grid = (int)(blocks < 152 * 64 ? blocks : 152 * 64);
    k_shell_table<<<grid, kThreads, 0, st>>>(sc, 0, sc.n_rays, tab);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_coef_prefix(const DevScene& sc, const int* keff, unsigned long long* sums,
                               cudaStream_t st) {
    if (sc.n_tiles <= sc.tile_lo) return cudaSuccess;
    k_coef_prefix<<<grid_blocks((const void*)k_coef_prefix, sc.n_tiles - sc.tile_lo), kThreads, 0,
                    st>>>(sc, keff, sums);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_tile_rows(const DevScene& sc, int* rows, cudaStream_t st) {
    if (sc.n_tiles <= sc.tile_lo) return cudaSuccess;
    k_tile_rows<<<grid_blocks((const void*)k_tile_rows, sc.n_tiles - sc.tile_lo), kThreads, 0, st>>>(sc, rows);
    count_launch();
    return cudaGetLastError();
}

template <typename TP>
cudaError_t launch_apply_coef_t(const DevScene& sc, const void* p, const float* coef,
                                const long long* tile_off, float* out, double* pap,
                                cudaStream_t st) {
    if (sc.n_tiles <= sc.tile_lo) return cudaSuccess;
    auto fn = sc.lay_s ? (sc.red_count ? k_apply_coef<TP, true, true> : k_apply_coef<TP, false, true>)
                       : (sc.red_count ? k_apply_coef<TP, true, false> : k_apply_coef<TP, false, false>);
    fn<<<grid_blocks((const void*)fn, sc.n_tiles - sc.tile_lo, sc.cap_per_sm), kThreads, 0, st>>>(
        sc, static_cast<const TP*>(p), reinterpret_cast<const float4*>(coef), tile_off, out, pap);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_apply_coef(const DevScene& sc, const void* p, int p_dtype, const float* coef,
                              const long long* tile_off, float* out, double* pap, cudaStream_t st) {
    return p_dtype == 1 ? launch_apply_coef_t<__nv_bfloat16>(sc, p, coef, tile_off, out, pap, st)
                        : launch_apply_coef_t<float>(sc, p, coef, tile_off, out, pap, st);
}

// ------------------------------------------------------ batched launchers

static int batch_blocks(const void* fn, int cap_per_sm) {
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kThreads, 0);
    if (occ <= 0) occ = 1;
    if (cap_per_sm > 0 && cap_per_sm < occ) occ = cap_per_sm;
    return (sms > 0 ? sms : 1) * occ;
}

cudaError_t launch_forward_batch(const BatchItem* items, const long long* start, int n,
                                 long long total, unsigned long long* counter, const float* x,
                                 const float* target, float* res, double* F, const int* active,
                                 int mode, int cap_per_sm, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess || total == 0) return e;
    if (mode == 0) {
        auto fn = k_forward_batch<0>;
        fn<<<batch_blocks((const void*)fn, cap_per_sm), kThreads, 0, st>>>(
            items, start, n, total, counter, x, nullptr, nullptr, nullptr, active, res);
    } else if (mode == 1) {
        auto fn = k_forward_batch<1>;
        fn<<<batch_blocks((const void*)fn, cap_per_sm), kThreads, 0, st>>>(
            items, start, n, total, counter, x, target, res, F, active, nullptr);
    } else {
        auto fn = k_forward_batch<2>;
        fn<<<batch_blocks((const void*)fn, cap_per_sm), kThreads, 0, st>>>(
            items, start, n, total, counter, x, target, nullptr, F, active, nullptr);
    }
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_scatter_batch(const BatchItem* items, const long long* start, int n,
                                 long long total, unsigned long long* counter, const float* x,
                                 const float* p, const float* v, float* out, float* out2,
                                 double* pap, int pap_stride, int mode, int cap_per_sm,
                                 cudaStream_t st, const PcgScalars* pcg, float* coef,
                                 const long long* tile_off, bool brick) {
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess || total == 0) return e;
    if (mode == 1) {
        auto fn = k_scatter_batch<1>;
        fn<<<batch_blocks((const void*)fn, cap_per_sm), kThreads, 0, st>>>(
            items, start, n, total, counter, x, p, v, out, out2, pap, pap_stride, pcg, nullptr,
            nullptr);
    } else {
        auto fn = brick ? k_scatter_batch<2, true> : k_scatter_batch<2, false>;
        fn<<<batch_blocks((const void*)fn, cap_per_sm), kThreads, 0, st>>>(
            items, start, n, total, counter, x, p, v, out, out2, pap, pap_stride, pcg,
            reinterpret_cast<float4*>(coef), tile_off);
    }
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_apply_coef_batch(const BatchItem* items, const long long* start, int n,
                                    long long total, unsigned long long* counter, const float* p,
                                    const float* coef, const long long* tile_off, float* out,
                                    double* pap, int pap_stride, int cap_per_sm, cudaStream_t st,
                                    const PcgScalars* pcg, bool brick) {
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess || total == 0) return e;
    auto fn = brick ? k_apply_coef_batch<true> : k_apply_coef_batch<false>;
    fn<<<batch_blocks((const void*)fn, cap_per_sm), kThreads, 0, st>>>(
        items, start, n, total, counter, p, reinterpret_cast<const float4*>(coef), tile_off, out,
        pap, pap_stride, pcg);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_tile_rows_batch(const BatchItem* items, const long long* start, int n,
                                   long long total, int* rows, cudaStream_t st) {
    if (total == 0) return cudaSuccess;
    k_tile_rows_batch<<<batch_blocks((const void*)k_tile_rows_batch, 0), kThreads, 0, st>>>(
        items, start, n, total, rows);
    count_launch();
    return cudaGetLastError();
}

}  // namespace perf

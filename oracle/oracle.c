/*
 * oracle.c -- plain FP64 CPU oracle for the PERF Gauss-Newton path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark do.  It shares no code with the CUDA path.
 *
 * What it computes (PERF, Rasmuson, Sintorn, Assarsson):
 *   - the discrete ray march of Eq. 3-4 through the RGBA voxel grid, followed
 *     by the environment-map shells intersected in order from the grid exit
 *     outwards (Section "Volume Rendering", Section "Rendering");
 *   - residuals r = H^ - C and the objective of Eq. 5-6;
 *   - the analytic partial derivatives of Eq. 3 (dH/dc_i and dH/dsigma_i,
 *     Section "Computation of partial derivatives"), written out from their
 *     definition with prefix transmittances and tail sums, chained through
 *     the trilinear / bilinear interpolation weights;
 *   - J p, J^T v and the exact diag(J^T J) of Section "Preconditioner"
 *     together with the gradient J^T r.
 *
 * Readings of the paper taken here (each is listed with its reason in the
 * design notes of the repository):
 *   - delta is measured in voxel sides (delta_bar = delta / h), so sigma is an
 *     opacity per voxel side; a shell hit counts as one sample with
 *     delta_bar = 1.
 *   - The step is the voxel side shortened to split the chord evenly:
 *     K = ceil(L / h) samples at t_in + (k + 1/2 + j_k) delta, delta = L / K.
 *   - Interpolation is exact trilinear (grid) / bilinear (shells), clamped to
 *     the edge, in place of texture hardware.
 *   - The ray itself (pixel -> origin and unit direction, the box entry and
 *     exit, K, delta, and which shells are hit) and each grid sample's index
 *     coordinates are defined in IEEE binary32 (ray set-up without
 *     contraction; the sample coordinates by single-rounding fmaf), the
 *     precision in which the kernels take these integer decisions (K, hits,
 *     the sample's cell); every later quantity is FP64.
 *   - Jitter uses SplitMix64 (Steele, Lea, Flood 2014) of (seed, epoch, ray,
 *     stream); it is fixed within one Gauss-Newton step.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -fPIC -shared (see build.py).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OC_MAX_SHELLS 8

typedef struct {
    int G;              /* grid resolution per axis */
    int S;              /* number of shells */
    int env_h, env_w;   /* shell texels (rows = theta, cols = phi) */
    float radii[OC_MAX_SHELLS];
    int n_cams, width, height;
    const float* c2w;   /* n_cams x 3 x 4, row-major */
    const float* focal; /* n_cams, pixels */
    int max_samples;
    int jitter;
    uint64_t seed;
    uint32_t epoch;
    int n_threads;      /* <= 0: OpenMP default */
    int aux;            /* 1: one auxiliary opacity residual per ray */
    double aux_lambda;  /* its factor (the paper's 0.1) */
    int env_kind;       /* 0: equirectangular shells, 1: cube-map shells */
} oc_problem;

/* ---------------------------------------------------------------- jitter */
static uint64_t splitmix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* U[0,1) with 24 random bits, exactly representable in binary32. */
static float oc_uniform(const oc_problem* P, int64_t ray, uint32_t stream) {
    uint64_t h = splitmix64(P->seed + (uint64_t)P->epoch);
    h = splitmix64(h + (uint64_t)ray);
    h = splitmix64(h + (uint64_t)stream);
    return (float)(h >> 40) * (1.0f / 16777216.0f);
}

/* --------------------------------------------------- binary32 ray set-up */
typedef struct {
    float o[3], d[3];
    float t_in, t_out, delta;
    int K;              /* 0: the ray misses the grid */
    unsigned shell_hit; /* bit s: shell s is hit */
} oc_ray;

static void oc_ray_setup(const oc_problem* P, int64_t ray, oc_ray* R) {
    const int64_t hw = (int64_t)P->width * P->height;
    const int cam = (int)(ray / hw);
    const int64_t rem = ray % hw;
    const int row = (int)(rem / P->width);
    const int col = (int)(rem % P->width);
    const float* M = P->c2w + 12 * cam;
    const float f = P->focal[cam];
    float jx = 0.5f, jy = 0.5f;
    if (P->jitter) {
        jx = oc_uniform(P, ray, 0u);
        jy = oc_uniform(P, ray, 1u);
    }
    const float px = (float)col + jx;
    const float py = (float)row + jy;
    const float xc = (px - 0.5f * (float)P->width) / f;
    const float yc = -((py - 0.5f * (float)P->height) / f);
    float d[3];
    for (int a = 0; a < 3; ++a) {
        const float u = M[4 * a + 0] * xc;
        const float v = M[4 * a + 1] * yc;
        d[a] = (u + v) - M[4 * a + 2];
    }
    const float s0 = d[0] * d[0];
    const float s1 = d[1] * d[1];
    const float s2 = d[2] * d[2];
    const float nn = sqrtf((s0 + s1) + s2);
    for (int a = 0; a < 3; ++a) {
        R->d[a] = d[a] / nn;
        R->o[a] = M[4 * a + 3];
    }
    float lo[3], hi[3];
    int miss = 0;
    for (int a = 0; a < 3; ++a) {
        if (R->d[a] != 0.0f) {
            const float t0 = (-1.0f - R->o[a]) / R->d[a];
            const float t1 = (1.0f - R->o[a]) / R->d[a];
            lo[a] = fminf(t0, t1);
            hi[a] = fmaxf(t0, t1);
        } else {
            if (R->o[a] < -1.0f || R->o[a] > 1.0f) miss = 1;
            lo[a] = -INFINITY;
            hi[a] = INFINITY;
        }
    }
    R->t_in = fmaxf(fmaxf(fmaxf(lo[0], lo[1]), lo[2]), 0.0f);
    R->t_out = fminf(fminf(hi[0], hi[1]), hi[2]);
    R->K = 0;
    R->delta = 0.0f;
    if (!miss && R->t_out > R->t_in) {
        const float h = 2.0f / (float)P->G;
        const float L = R->t_out - R->t_in;
        int K = (int)ceilf(L / h);
        if (K > P->max_samples) K = P->max_samples;
        if (K < 1) K = 1;
        R->K = K;
        R->delta = L / (float)K;
    }
    /* far-root shell hits: the ray leaves sphere s at t > 0 */
    const float b = (R->o[0] * R->d[0] + R->o[1] * R->d[1]) + R->o[2] * R->d[2];
    const float oo = (R->o[0] * R->o[0] + R->o[1] * R->o[1]) + R->o[2] * R->o[2];
    R->shell_hit = 0u;
    for (int s = 0; s < P->S; ++s) {
        const float rr = P->radii[s] * P->radii[s];
        const float c = oo - rr;
        const float bb = b * b;
        const float disc = bb - c;
        if (disc > 0.0f && (b < 0.0f || c < 0.0f)) R->shell_hit |= 1u << s;
    }
}

/* ------------------------------------------------------- sample records */
typedef struct {
    int64_t idx[8];     /* voxel / texel index (parameter block of 4) */
    double w[8];        /* interpolation weights */
    int nc;             /* 8 (grid) or 4 (shell) */
    int is_grid;
    double sigma, c[3], dbar;
} oc_sample;

/* Trilinear interpolation at grid index coordinates u[3] (voxel i centred at
 * u = i): clamped to [0, G-1], cell base floor(u) (at most G-2), fractions
 * u - base. */
static void oc_trilinear(const oc_problem* P, const float u_in[3], oc_sample* s) {
    const int G = P->G;
    int64_t b[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
        double u = (double)u_in[a];
        if (u < 0.0) u = 0.0;
        if (u > (double)(G - 1)) u = (double)(G - 1);
        double fl = floor(u);
        if (fl > (double)(G - 2)) fl = (double)(G - 2);
        b[a] = (int64_t)fl;
        f[a] = u - fl;
    }
    s->nc = 8;
    s->is_grid = 1;
    for (int c = 0; c < 8; ++c) {
        const int cx = c & 1, cy = (c >> 1) & 1, cz = (c >> 2) & 1;
        const int64_t ix = b[0] + cx, iy = b[1] + cy, iz = b[2] + cz;
        s->idx[c] = (iz * G + iy) * G + ix;
        s->w[c] = (cx ? f[0] : 1.0 - f[0]) * (cy ? f[1] : 1.0 - f[1]) *
                  (cz ? f[2] : 1.0 - f[2]);
    }
}

/* Grid index coordinates of sample k of a ray, in binary32 (each fmaf
 * rounded once): t_k = t_in + (k + 1/2 + j_k) delta, position o + t_k d,
 * u = position * G/2 + (G/2 - 1/2) (voxel i centred at -1 + (i + 1/2) h).
 * These coordinates decide the sample's cell, an integer, so they are
 * defined in the precision in which the kernels take that decision; the
 * interpolation and everything after it is FP64. */
static void oc_sample_coords(const oc_problem* P, const oc_ray* R, int64_t ray, int k,
                             float u[3]) {
    float jk = 0.0f;
    if (P->jitter) jk = oc_uniform(P, ray, 2u + (uint32_t)k) - 0.5f;
    const float kk = ((float)k + 0.5f) + jk;
    const float t = fmaf(kk, R->delta, R->t_in);
    const float hg = 0.5f * (float)P->G;
    for (int a = 0; a < 3; ++a) u[a] = fmaf(fmaf(t, R->d[a], R->o[a]), hg, hg - 0.5f);
}

static void oc_bilinear(const oc_problem* P, int shell, const double q[3],
                        oc_sample* s) {
    const int He = P->env_h, We = P->env_w;
    const double r = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
    const double wx = q[0] / r, wy = q[1] / r, wz = q[2] / r;
    const double phi = atan2(wy, wx);
    const double theta = atan2(sqrt(wx * wx + wy * wy), wz);
    const double u = (phi / (2.0 * M_PI) + 0.5) * We - 0.5;
    double v = theta / M_PI * He - 0.5;
    const double j0 = floor(u);
    const double fu = u - j0;
    int64_t c0 = ((int64_t)j0 % We + We) % We;
    int64_t c1 = (c0 + 1) % We;
    if (v < 0.0) v = 0.0;
    if (v > (double)(He - 1)) v = (double)(He - 1);
    double i0 = floor(v);
    if (i0 > (double)(He - 2)) i0 = (double)(He - 2);
    const double fv = v - i0;
    const int64_t r0 = (int64_t)i0, r1 = r0 + 1;
    const int64_t base = (int64_t)P->G * P->G * P->G + (int64_t)shell * He * We;
    s->nc = 4;
    s->is_grid = 0;
    s->idx[0] = base + r0 * We + c0; s->w[0] = (1.0 - fu) * (1.0 - fv);
    s->idx[1] = base + r0 * We + c1; s->w[1] = fu * (1.0 - fv);
    s->idx[2] = base + r1 * We + c0; s->w[2] = (1.0 - fu) * fv;
    s->idx[3] = base + r1 * We + c1; s->w[3] = fu * fv;
    for (int c = 4; c < 8; ++c) { s->idx[c] = 0; s->w[c] = 0.0; }
}

/* Section "Implementation": environment maps as cube maps.  Shell s is an
 * env_h x env_w image with env_w = 6 F, F = env_h: face f (0..5 = +x, -x,
 * +y, -y, +z, -z) occupies columns [f F, (f + 1) F).  A hit point q (binary32,
 * see oc_shell_hit_f32) lies on the face of its largest |q_a| (ties go to
 * the lower axis); with (b, c) the other two axes in increasing order,
 * s = q_b / |q_a| and t = q_c / |q_a| in [-1, 1], and the face's texel
 * coordinates are u = s F/2 + (F/2 - 1/2) (column) and v = t F/2 + (F/2 - 1/2)
 * (row), texel i centred at i.  Face, u and v are binary32 (they decide
 * integers: the face and the texels); the bilinear weights, clamped to the
 * face's edge texels (no filtering across faces), are FP64. */
static void oc_cube(const oc_problem* P, int shell, const float q[3], oc_sample* s) {
    const int F = P->env_h, We = P->env_w;
    const float ax = fabsf(q[0]), ay = fabsf(q[1]), az = fabsf(q[2]);
    int a = 2;
    if (ax >= ay && ax >= az) a = 0;
    else if (ay >= az) a = 1;
    const int face = 2 * a + (q[a] < 0.0f ? 1 : 0);
    const int b = a == 0 ? 1 : 0, c = a == 2 ? 1 : 2;
    const float m = fabsf(q[a]);
    const float hf = 0.5f * (float)F;
    const float uf = fmaf(q[b] / m, hf, hf - 0.5f);
    const float vf = fmaf(q[c] / m, hf, hf - 0.5f);
    double uv[2] = {(double)uf, (double)vf};
    int64_t base2[2];
    double fr[2];
    for (int i = 0; i < 2; ++i) {
        double u = uv[i];
        if (u < 0.0) u = 0.0;
        if (u > (double)(F - 1)) u = (double)(F - 1);
        double fl = floor(u);
        if (fl > (double)(F - 2)) fl = (double)(F - 2);
        base2[i] = (int64_t)fl;
        fr[i] = u - fl;
    }
    const int64_t c0 = (int64_t)face * F + base2[0], r0 = base2[1];
    const int64_t base = (int64_t)P->G * P->G * P->G + (int64_t)shell * P->env_h * We;
    s->nc = 4;
    s->is_grid = 0;
    s->idx[0] = base + r0 * We + c0;           s->w[0] = (1.0 - fr[0]) * (1.0 - fr[1]);
    s->idx[1] = base + r0 * We + c0 + 1;       s->w[1] = fr[0] * (1.0 - fr[1]);
    s->idx[2] = base + (r0 + 1) * We + c0;     s->w[2] = (1.0 - fr[0]) * fr[1];
    s->idx[3] = base + (r0 + 1) * We + c0 + 1; s->w[3] = fr[0] * fr[1];
    for (int k = 4; k < 8; ++k) { s->idx[k] = 0; s->w[k] = 0.0; }
}

/* Far-root hit point of a ray with the sphere of radius `radius`, in binary32
 * with every operation rounded once (the precision in which the kernels
 * decide a cube map's face and texels). */
static void oc_shell_hit_f32(const oc_ray* R, float radius, float q[3]) {
    const float b = (R->o[0] * R->d[0] + R->o[1] * R->d[1]) + R->o[2] * R->d[2];
    const float oo = (R->o[0] * R->o[0] + R->o[1] * R->o[1]) + R->o[2] * R->o[2];
    const float c = oo - radius * radius;
    float disc = b * b - c;
    if (disc < 0.0f) disc = 0.0f;
    const float sq = sqrtf(disc);
    const float t = (b < 0.0f) ? (sq - b) : (c / (-b - sq));
    for (int a = 0; a < 3; ++a) q[a] = fmaf(t, R->d[a], R->o[a]);
}

static void oc_interp(const double* x, oc_sample* s) {
    double acc[4] = {0, 0, 0, 0};
    for (int c = 0; c < s->nc; ++c)
        for (int ch = 0; ch < 4; ++ch) acc[ch] += s->w[c] * x[4 * s->idx[c] + ch];
    s->c[0] = acc[0]; s->c[1] = acc[1]; s->c[2] = acc[2];
    s->sigma = acc[3];
}

/* Build the ordered sample list of one ray: K grid samples, then the shells
 * that the ray hits, innermost first.  Returns the count; *n_grid gets K. */
static int oc_collect(const oc_problem* P, const double* x, int64_t ray,
                      oc_sample* out, int* n_grid) {
    oc_ray R;
    oc_ray_setup(P, ray, &R);
    const double o[3] = {R.o[0], R.o[1], R.o[2]};
    const double d[3] = {R.d[0], R.d[1], R.d[2]};
    const double delta = (double)R.delta;
    const double dbar = delta * (0.5 * P->G); /* delta / h */
    int n = 0;
    for (int k = 0; k < R.K; ++k) {
        float u[3];
        oc_sample_coords(P, &R, ray, k, u);
        oc_trilinear(P, u, &out[n]);
        oc_interp(x, &out[n]);
        out[n].dbar = dbar;
        ++n;
    }
    *n_grid = n;
    const double b = o[0] * d[0] + o[1] * d[1] + o[2] * d[2];
    const double oo = o[0] * o[0] + o[1] * o[1] + o[2] * o[2];
    for (int s = 0; s < P->S; ++s) {
        if (!(R.shell_hit & (1u << s))) continue;
        const double rad = (double)P->radii[s];
        const double c = oo - rad * rad;
        double disc = b * b - c;
        if (disc < 0.0) disc = 0.0;
        const double sq = sqrt(disc);
        const double t = (b < 0.0) ? (-b + sq) : (c / (-b - sq));
        if (P->env_kind == 1) {
            float qf[3];
            oc_shell_hit_f32(&R, P->radii[s], qf);
            oc_cube(P, s, qf, &out[n]);
        } else {
            const double q[3] = {o[0] + t * d[0], o[1] + t * d[1], o[2] + t * d[2]};
            oc_bilinear(P, s, q, &out[n]);
        }
        oc_interp(x, &out[n]);
        out[n].dbar = 1.0;
        ++n;
    }
    return n;
}

/* Eq. 3-4: H^ = sum_i T_i (1 - e^{-sigma_i dbar_i}) c_i. */
static void oc_composite(const oc_sample* s, int n, int n_grid, double H[3],
                         double* T_exit, double* T_final) {
    double T = 1.0;
    H[0] = H[1] = H[2] = 0.0;
    *T_exit = 1.0;
    for (int i = 0; i < n; ++i) {
        const double alpha = -expm1(-s[i].sigma * s[i].dbar);
        for (int k = 0; k < 3; ++k) H[k] += T * alpha * s[i].c[k];
        T *= exp(-s[i].sigma * s[i].dbar);
        if (i + 1 == n_grid) *T_exit = T;
    }
    if (n_grid == 0) *T_exit = 1.0;
    *T_final = T;
}

/* Partial derivatives of Eq. 3, written out from the definition (Section
 * "Computation of partial derivatives" states the same quantities; this is
 * not its recurrence).  With s_i = sigma_i dbar_i,
 *   T_i = exp(-sum_{j<i} s_j)          (transmittance in front of sample i)
 *   w_i = T_i (1 - e^{-s_i})           (its weight in H^)
 *   H^  = sum_i w_i c_i.
 * c_i enters only term i:            dH/dc_i = w_i.
 * sigma_i enters term i through 1 - e^{-s_i} (derivative dbar_i e^{-s_i})
 * and every later term j > i through T_j (dT_j/dsigma_i = -dbar_i T_j):
 *   dH_k/dsigma_i = dbar_i (T_i e^{-s_i} c_ik - sum_{j>i} w_j c_jk).
 * T_i is formed from its prefix sum of optical depth, and the tail sums
 * sum_{j>i} w_j c_j from the array of all weights, each on its own.
 * dHdc[i] = dH/dc_i (same for the three channels), dHds[3 i + k] =
 * dH_k/dsigma_i. */
static void oc_partials(const oc_sample* s, int n, double* dHdc, double* dHds) {
    double* T = (double*)malloc(sizeof(double) * (size_t)(n + 1));
    double* w = (double*)malloc(sizeof(double) * (size_t)(n + 1));
    double* tail = (double*)malloc(sizeof(double) * 3 * (size_t)(n + 1));
    double depth = 0.0;                      /* sum_{j<i} s_j */
    for (int i = 0; i < n; ++i) {
        const double si = s[i].sigma * s[i].dbar;
        T[i] = exp(-depth);
        w[i] = T[i] * -expm1(-si);
        depth += si;
    }
    /* tail[3 i + k] = sum_{j > i} w_j c_jk */
    for (int k = 0; k < 3; ++k) tail[3 * (n > 0 ? n - 1 : 0) + k] = 0.0;
    for (int i = n - 2; i >= 0; --i)
        for (int k = 0; k < 3; ++k)
            tail[3 * i + k] = tail[3 * (i + 1) + k] + w[i + 1] * s[i + 1].c[k];
    for (int i = 0; i < n; ++i) {
        const double si = s[i].sigma * s[i].dbar;
        dHdc[i] = w[i];
        for (int k = 0; k < 3; ++k)
            dHds[3 * i + k] = s[i].dbar * (T[i] * exp(-si) * s[i].c[k] - tail[3 * i + k]);
    }
    free(T); free(w); free(tail);
}

static int oc_nthreads(const oc_problem* P) {
#ifdef _OPENMP
    return P->n_threads > 0 ? P->n_threads : omp_get_max_threads();
#else
    (void)P;
    return 1;
#endif
}

static int64_t oc_n_rays(const oc_problem* P) {
    return (int64_t)P->n_cams * P->width * P->height;
}

static int64_t oc_n_params(const oc_problem* P) {
    return 4 * ((int64_t)P->G * P->G * P->G + (int64_t)P->S * P->env_h * P->env_w);
}

static int oc_cap(const oc_problem* P) { return P->max_samples + P->S + 1; }

/* Residuals per ray: the three colour channels, plus the auxiliary one. */
static int oc_nres(const oc_problem* P) { return P->aux ? 4 : 3; }

/* Section "Auxiliary terms": L = lambda (1 - 4 (T^ - 1/2)^2), T^ the
 * transmittance at grid exit (Eq. 4 over the grid samples).  With
 * dT^/dsigma_i = -dbar_i T^ for a grid sample, dL/dsigma_i =
 * 8 lambda (T^ - 1/2) T^ dbar_i; *dfac gets 8 lambda (T^ - 1/2) T^. */
static void oc_aux(const oc_problem* P, const oc_sample* s, int n_grid, double* L,
                   double* dfac) {
    double V = 0.0;
    for (int i = 0; i < n_grid; ++i) V += s[i].sigma * s[i].dbar;
    const double T = exp(-V);
    *L = P->aux_lambda * (1.0 - 4.0 * (T - 0.5) * (T - 0.5));
    *dfac = 8.0 * P->aux_lambda * (T - 0.5) * T;
}

/* ---------------------------------------------------------- public API */

int oc_param_count(const oc_problem* P, int64_t* n) { *n = oc_n_params(P); return 0; }

/* Render: rgb[3 * j], T_exit[j] (transmittance at the grid exit) and
 * T_final[j] for ray ids[j] (ids == NULL: all rays in order). */
int oc_render(const oc_problem* P, const double* x, const int64_t* ids, int64_t n_ids,
              double* rgb, double* T_exit, double* T_final) {
    const int64_t N = ids ? n_ids : oc_n_rays(P);
    const int cap = oc_cap(P);
#pragma omp parallel num_threads(oc_nthreads(P))
    {
        oc_sample* buf = (oc_sample*)malloc(sizeof(oc_sample) * cap);
#pragma omp for schedule(dynamic, 256)
        for (int64_t j = 0; j < N; ++j) {
            const int64_t ray = ids ? ids[j] : j;
            int ng;
            const int n = oc_collect(P, x, ray, buf, &ng);
            double H[3], Te, Tf;
            oc_composite(buf, n, ng, H, &Te, &Tf);
            if (rgb) { rgb[3 * j] = H[0]; rgb[3 * j + 1] = H[1]; rgb[3 * j + 2] = H[2]; }
            if (T_exit) T_exit[j] = Te;
            if (T_final) T_final[j] = Tf;
        }
        free(buf);
    }
    return 0;
}

/* Residuals r = H^ - C (Eq. 5, C8 sign) and F = 1/2 sum r^2 (Eq. 6); with
 * aux, r has 4 entries per ray, the 4th the auxiliary term L. */
int oc_residual(const oc_problem* P, const double* x, const double* target,
                const int64_t* ids, int64_t n_ids, double* r, double* F) {
    const int64_t N = ids ? n_ids : oc_n_rays(P);
    const int cap = oc_cap(P);
    double acc = 0.0;
#pragma omp parallel num_threads(oc_nthreads(P)) reduction(+:acc)
    {
        oc_sample* buf = (oc_sample*)malloc(sizeof(oc_sample) * cap);
#pragma omp for schedule(dynamic, 256)
        for (int64_t j = 0; j < N; ++j) {
            const int64_t ray = ids ? ids[j] : j;
            int ng;
            const int n = oc_collect(P, x, ray, buf, &ng);
            double H[3], Te, Tf;
            oc_composite(buf, n, ng, H, &Te, &Tf);
            const int R = oc_nres(P);
            for (int k = 0; k < 3; ++k) {
                const double rk = H[k] - target[3 * j + k];
                if (r) r[R * j + k] = rk;
                acc += 0.5 * rk * rk;
            }
            if (P->aux) {
                double L, dfac;
                oc_aux(P, buf, ng, &L, &dfac);
                if (r) r[R * j + 3] = L;
                acc += 0.5 * L * L;
            }
        }
        free(buf);
    }
    if (F) *F = acc;
    return 0;
}

/* (J p) for the listed rays: sum over samples and interpolation corners of
 * dH/dx_j p_j, with the partials of Eq. 3 (oc_partials). */
int oc_jvp_mag(const oc_problem* P, const double* x, const double* p, const int64_t* ids,
               int64_t n_ids, double* out, double* mag);

int oc_jvp(const oc_problem* P, const double* x, const double* p, const int64_t* ids,
           int64_t n_ids, double* out) {
    return oc_jvp_mag(P, x, p, ids, n_ids, out, NULL);
}

/* oc_jvp, and (mag != NULL) the sum of the absolute values of the terms of
 * each entry, mag = |J| |p| (the scale of its floating-point rounding). */
int oc_jvp_mag(const oc_problem* P, const double* x, const double* p, const int64_t* ids,
               int64_t n_ids, double* out, double* mag) {
    const int64_t N = ids ? n_ids : oc_n_rays(P);
    const int cap = oc_cap(P);
#pragma omp parallel num_threads(oc_nthreads(P))
    {
        oc_sample* buf = (oc_sample*)malloc(sizeof(oc_sample) * cap);
        double* dc = (double*)malloc(sizeof(double) * cap);
        double* ds = (double*)malloc(sizeof(double) * 3 * cap);
#pragma omp for schedule(dynamic, 256)
        for (int64_t j = 0; j < N; ++j) {
            const int64_t ray = ids ? ids[j] : j;
            int ng;
            const int n = oc_collect(P, x, ray, buf, &ng);
            oc_partials(buf, n, dc, ds);
            double acc[4] = {0, 0, 0, 0}, am[4] = {0, 0, 0, 0};
            double L = 0.0, dfac = 0.0;
            if (P->aux) oc_aux(P, buf, ng, &L, &dfac);
            for (int i = 0; i < n; ++i)
                for (int c = 0; c < buf[i].nc; ++c) {
                    const int64_t q = 4 * buf[i].idx[c];
                    const double w = buf[i].w[c];
                    for (int k = 0; k < 3; ++k) {
                        acc[k] += w * (dc[i] * p[q + k] + ds[3 * i + k] * p[q + 3]);
                        am[k] += fabs(w) * (fabs(dc[i] * p[q + k]) + fabs(ds[3 * i + k] * p[q + 3]));
                    }
                    if (i < ng) {
                        acc[3] += w * dfac * buf[i].dbar * p[q + 3];
                        am[3] += fabs(w * dfac * buf[i].dbar * p[q + 3]);
                    }
                }
            const int R = oc_nres(P);
            for (int k = 0; k < R; ++k) out[R * j + k] = acc[k];
            if (mag)
                for (int k = 0; k < R; ++k) mag[R * j + k] = am[k];
        }
        free(buf); free(dc); free(ds);
    }
    return 0;
}

/* Reduce per-thread n-vectors into out (fixed thread order). */
static void oc_reduce(double** parts, int nt, int64_t n, double* out, int accumulate) {
    for (int64_t q = 0; q < n; ++q) {
        double s = accumulate ? out[q] : 0.0;
        for (int t = 0; t < nt; ++t) s += parts[t][q];
        out[q] = s;
    }
}

/* out = J^T v (all rays): out_j = sum_rays sum_k v_k dr_k/dx_j (v has 3,
 * or with aux 4, entries per ray). */
int oc_vjp_mag(const oc_problem* P, const double* x, const double* v, double* out,
               int accumulate, double* mag);

int oc_vjp(const oc_problem* P, const double* x, const double* v, double* out,
           int accumulate) {
    return oc_vjp_mag(P, x, v, out, accumulate, NULL);
}

/* oc_vjp, and (mag != NULL) mag = |J|^T |v|, the sum of the absolute values
 * of the terms of each entry. */
int oc_vjp_mag(const oc_problem* P, const double* x, const double* v, double* out,
               int accumulate, double* mag) {
    const int64_t N = oc_n_rays(P);
    const int64_t np = oc_n_params(P);
    const int cap = oc_cap(P);
    const int nt = oc_nthreads(P);
    double** parts = (double**)calloc(nt, sizeof(double*));
    double** mparts = (double**)calloc(nt, sizeof(double*));
#pragma omp parallel num_threads(nt)
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double* acc = (double*)calloc(np, sizeof(double));
        double* am = mag ? (double*)calloc(np, sizeof(double)) : NULL;
        parts[tid] = acc;
        mparts[tid] = am;
        oc_sample* buf = (oc_sample*)malloc(sizeof(oc_sample) * cap);
        double* dc = (double*)malloc(sizeof(double) * cap);
        double* ds = (double*)malloc(sizeof(double) * 3 * cap);
#pragma omp for schedule(dynamic, 256)
        for (int64_t ray = 0; ray < N; ++ray) {
            const double* vr = v + oc_nres(P) * ray;
            const double va = P->aux ? vr[3] : 0.0;
            if (vr[0] == 0.0 && vr[1] == 0.0 && vr[2] == 0.0 && va == 0.0) continue;
            int ng;
            const int n = oc_collect(P, x, ray, buf, &ng);
            oc_partials(buf, n, dc, ds);
            double L = 0.0, dfac = 0.0;
            if (P->aux) oc_aux(P, buf, ng, &L, &dfac);
            for (int i = 0; i < n; ++i) {
                double gs = vr[0] * ds[3 * i] + vr[1] * ds[3 * i + 1] + vr[2] * ds[3 * i + 2];
                double gm = fabs(vr[0] * ds[3 * i]) + fabs(vr[1] * ds[3 * i + 1]) +
                            fabs(vr[2] * ds[3 * i + 2]);
                if (i < ng) {
                    gs += va * dfac * buf[i].dbar;
                    gm += fabs(va * dfac * buf[i].dbar);
                }
                for (int c = 0; c < buf[i].nc; ++c) {
                    const int64_t q = 4 * buf[i].idx[c];
                    const double w = buf[i].w[c];
                    for (int k = 0; k < 3; ++k) acc[q + k] += w * dc[i] * vr[k];
                    acc[q + 3] += w * gs;
                    if (am) {
                        for (int k = 0; k < 3; ++k) am[q + k] += fabs(w * dc[i] * vr[k]);
                        am[q + 3] += fabs(w) * gm;
                    }
                }
            }
        }
        free(buf); free(dc); free(ds);
    }
    int used = 0;
    for (int t = 0; t < nt; ++t) if (parts[t]) used = t + 1;
    oc_reduce(parts, used, np, out, accumulate);
    if (mag) oc_reduce(mparts, used, np, mag, 0);
    for (int t = 0; t < nt; ++t) { free(parts[t]); if (mparts[t]) free(mparts[t]); }
    free(parts);
    free(mparts);
    return 0;
}

typedef struct { int64_t q; int k; double val; } oc_entry;

static int oc_entry_cmp(const void* a, const void* b) {
    const oc_entry* x = (const oc_entry*)a;
    const oc_entry* y = (const oc_entry*)b;
    if (x->q != y->q) return x->q < y->q ? -1 : 1;
    return x->k - y->k;
}

/* Exact Jacobi diagonal diag(J^T J)_q = sum_rows (dr/dx_q)^2 and (when r is
 * given) the gradient J^T r.  Each row's entry for parameter q is first
 * summed over all samples of the ray that touch q, then squared. */
static int oc_diag_impl(const oc_problem* P, const double* x, const double* r, double* diag,
                        double* grad, double* cross);

int oc_diag_grad(const oc_problem* P, const double* x, const double* r, double* diag,
                 double* grad) {
    return oc_diag_impl(P, x, r, diag, grad, NULL);
}

/* Off-diagonal entries of each grid voxel's 4x4 block of J^T J: cross[4v+k] =
 * sum_rows (dr/dc_{v,k}) (dr/dsigma_v) for k < 3 (colour-colour entries vanish
 * since colour k only enters residual k); cross[4v+3] = 0. */
int oc_block_cross(const oc_problem* P, const double* x, double* diag, double* cross) {
    return oc_diag_impl(P, x, NULL, diag, NULL, cross);
}

static int oc_diag_impl(const oc_problem* P, const double* x, const double* r, double* diag,
                        double* grad, double* cross) {
    const int64_t N = oc_n_rays(P);
    const int64_t np = oc_n_params(P);
    const int cap = oc_cap(P);
    const int nt = oc_nthreads(P);
    double** pd = (double**)calloc(nt, sizeof(double*));
    double** pg = (double**)calloc(nt, sizeof(double*));
    double** pc = (double**)calloc(nt, sizeof(double*));
    const int64_t nvox = (int64_t)P->G * P->G * P->G;
#pragma omp parallel num_threads(nt)
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double* ad = (double*)calloc(np, sizeof(double));
        double* ag = (double*)calloc(np, sizeof(double));
        double* ac = cross ? (double*)calloc(4 * nvox, sizeof(double)) : NULL;
        pd[tid] = ad;
        pg[tid] = ag;
        pc[tid] = ac;
        oc_sample* buf = (oc_sample*)malloc(sizeof(oc_sample) * cap);
        double* dc = (double*)malloc(sizeof(double) * cap);
        double* ds = (double*)malloc(sizeof(double) * 3 * cap);
        oc_entry* ent = (oc_entry*)malloc(sizeof(oc_entry) * (size_t)cap * 8 * 7);
#pragma omp for schedule(dynamic, 64)
        for (int64_t ray = 0; ray < N; ++ray) {
            int ng;
            const int n = oc_collect(P, x, ray, buf, &ng);
            oc_partials(buf, n, dc, ds);
            double L = 0.0, dfac = 0.0;
            if (P->aux) oc_aux(P, buf, ng, &L, &dfac);
            const int R = oc_nres(P);
            int64_t ne = 0;
            for (int i = 0; i < n; ++i)
                for (int c = 0; c < buf[i].nc; ++c) {
                    const int64_t q = 4 * buf[i].idx[c];
                    const double w = buf[i].w[c];
                    for (int k = 0; k < 3; ++k) {
                        ent[ne].q = q + k; ent[ne].k = k; ent[ne].val = w * dc[i]; ++ne;
                        ent[ne].q = q + 3; ent[ne].k = k; ent[ne].val = w * ds[3 * i + k]; ++ne;
                    }
                    if (P->aux && i < ng) {   /* the auxiliary row: sigma only */
                        ent[ne].q = q + 3; ent[ne].k = 3; ent[ne].val = w * dfac * buf[i].dbar; ++ne;
                    }
                }
            qsort(ent, (size_t)ne, sizeof(oc_entry), oc_entry_cmp);
            int64_t a = 0;
            int64_t cur_vox = -1;
            double gv[4][3];
            memset(gv, 0, sizeof(gv));
            while (a < ne) {
                int64_t b = a;
                double g[4] = {0, 0, 0, 0};
                while (b < ne && ent[b].q == ent[a].q) { g[ent[b].k] += ent[b].val; ++b; }
                const int64_t q = ent[a].q;
                ad[q] += g[0] * g[0] + g[1] * g[1] + g[2] * g[2] + g[3] * g[3];
                if (r) {
                    ag[q] += g[0] * r[R * ray] + g[1] * r[R * ray + 1] + g[2] * r[R * ray + 2];
                    if (P->aux) ag[q] += g[3] * r[R * ray + 3];
                }
                if (ac && q / 4 < nvox) {
                    if (q / 4 != cur_vox) {
                        if (cur_vox >= 0)
                            for (int k = 0; k < 3; ++k) ac[4 * cur_vox + k] += gv[k][k] * gv[3][k];
                        cur_vox = q / 4;
                        memset(gv, 0, sizeof(gv));
                    }
                    for (int k = 0; k < 3; ++k) gv[q % 4][k] = g[k];
                }
                a = b;
            }
            if (ac && cur_vox >= 0)
                for (int k = 0; k < 3; ++k) ac[4 * cur_vox + k] += gv[k][k] * gv[3][k];
        }
        free(buf); free(dc); free(ds); free(ent);
    }
    int used = 0;
    for (int t = 0; t < nt; ++t) if (pd[t]) used = t + 1;
    if (diag) oc_reduce(pd, used, np, diag, 0);
    if (grad && r) oc_reduce(pg, used, np, grad, 0);
    if (cross) oc_reduce(pc, used, 4 * nvox, cross, 0);
    for (int t = 0; t < nt; ++t) { free(pd[t]); free(pg[t]); if (pc[t]) free(pc[t]); }
    free(pd); free(pg); free(pc);
    return 0;
}

/* Per-sample record of one ray, for invariant checks: returns the number of
 * samples n (grid first, then shells) and fills, for i < min(n, cap):
 * T_before[i], alpha[i], sigma[i], c[3i..3i+2], dbar[i]; *n_grid = K. */
int oc_ray_samples(const oc_problem* P, const double* x, int64_t ray, int cap,
                   double* T_before, double* alpha, double* sigma, double* c,
                   double* dbar, int* n_grid) {
    const int cc = oc_cap(P);
    oc_sample* buf = (oc_sample*)malloc(sizeof(oc_sample) * cc);
    int ng;
    const int n = oc_collect(P, x, ray, buf, &ng);
    double T = 1.0;
    for (int i = 0; i < n && i < cap; ++i) {
        const double a = -expm1(-buf[i].sigma * buf[i].dbar);
        T_before[i] = T;
        alpha[i] = a;
        sigma[i] = buf[i].sigma;
        for (int k = 0; k < 3; ++k) c[3 * i + k] = buf[i].c[k];
        dbar[i] = buf[i].dbar;
        T *= exp(-buf[i].sigma * buf[i].dbar);
    }
    *n_grid = ng;
    free(buf);
    return n;
}

/* The binary32 ray definition, exposed for checks of the host-side logic. */
int oc_ray_info(const oc_problem* P, int64_t ray, float* o, float* d, float* t_in,
                float* t_out, float* delta, int* K, unsigned* shell_hit) {
    oc_ray R;
    oc_ray_setup(P, ray, &R);
    for (int a = 0; a < 3; ++a) { o[a] = R.o[a]; d[a] = R.d[a]; }
    *t_in = R.t_in; *t_out = R.t_out; *delta = R.delta; *K = R.K;
    *shell_hit = R.shell_hit;
    return 0;
}

/* SplitMix64 uniform draw, exposed for cross-checks. */
float oc_jitter_uniform(const oc_problem* P, int64_t ray, uint32_t stream) {
    return oc_uniform(P, ray, stream);
}

/*
 * perf.h -- C ABI of libperf: the matrix-free Gauss-Newton step of PERF
 * (Performant, Explicit Radiance Fields; Rasmuson, Sintorn, Assarsson) on one
 * GB300 GPU.
 *
 * Problem (Section "Method"): the unknowns x are an RGBA voxel grid of G^3
 * cells on [-1, 1]^3 followed by S equirectangular RGBA environment-map
 * shells; every training pixel is one ray with three residuals
 * r = H^ - C (Eq. 5-6); J is the m x n Jacobian of r, A = J^T J and
 * b = -J^T r (Section "Update step"); the Gauss-Newton step solves A Delta = b
 * by Jacobi-preconditioned CG (Algorithm 2) and scales it by the
 * backtracking line search of Algorithm 3 (Eq. 7).
 *
 * Layouts (all little-endian, C order):
 *   x       n = 4 (G^3 + S H_e W_e) values: grid [z][y][x][4], then shell 0,
 *           1, ... each [row][col][4]; channels (r, g, b, sigma).  Row 0 of a
 *           shell is its +z pole; columns run in azimuth from -pi.  sigma is
 *           an opacity per voxel side.  Storage is float32, or bfloat16 when
 *           the scene's dtype is PERF_BF16 (per-call entry points only).
 *   rays    N_r = n_cams * height * width, ray = (cam * height + row) * width
 *           + col; an image or target has 3 N_r values indexed
 *           ray * 3 + channel; a residual, J p or J^T-input vector has
 *           R N_r values indexed ray * R + k, R = 3 (R = 4 with the
 *           auxiliary residual, perf_options.aux: k = 3 is that term).
 *           Images and J p are float32; targets and residuals (the per-ray
 *           intermediates of a step) are float32, or bfloat16 when the
 *           scene's dtype is PERF_BF16.
 * Pointers are DEVICE pointers unless a comment says HOST.  The caller owns
 * every buffer it passes in; the context owns only its workspace (PCG
 * vectors, residual buffer, FP64 scalars) and frees it in perf_destroy.
 * Every call is asynchronous on the given stream (a cudaStream_t; NULL = the
 * legacy default stream) unless it writes a HOST output, in which case it
 * synchronises that stream before returning.
 *
 * Errors: every call returns a perf_status; nothing throws.  Arguments are
 * validated before any launch (PERF_ERR_INVALID_ARG); CUDA failures return
 * PERF_ERR_CUDA; perf_last_error() gives a message for the context's last
 * failure.  A context is not thread-safe: one host thread at a time.
 */
#ifndef PERF_H
#define PERF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PERF_OK = 0,
    PERF_ERR_INVALID_ARG = 1,
    PERF_ERR_CUDA = 2,
    PERF_ERR_NONFINITE = 3,   /* a PCG scalar or the objective is NaN / Inf */
    PERF_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up */
    PERF_ERR_NOT_SPD = 5,     /* p^T A p <= 0 in PCG */
    PERF_ERR_UNSUPPORTED = 6
} perf_status;

enum { PERF_F32 = 0, PERF_BF16 = 1 };
enum { PERF_PRECOND_JACOBI = 0,        /* diag(J^T J) (Section "Preconditioner") */
       PERF_PRECOND_BLOCK4 = 1,        /* 4x4 block per voxel: learned (perf_set_lpc) or
                                          caller-supplied (perf_pcg_set_blocks) */
       PERF_PRECOND_BLOCK_JACOBI = 2   /* exact inverse of each voxel's 4x4 block of J^T J */ };
/* What decides that a Gauss-Newton step's PCG with the learned blocks is
 * rerun with Jacobi (perf_options.precond_judge).  Either way a breakdown, a
 * non-finite scalar or a convolution whose bounded wait ran out falls back,
 * and a step of a block preconditioner that no trial point of the line
 * search can use is redone with Jacobi. */
enum { PERF_JUDGE_RESIDUAL = 0,   /* the true PCG residual: r^T r after PCG must
                                     be below r_0^T r_0 */
       PERF_JUDGE_OBJECTIVE = 1   /* the objective: the line search judges the
                                     step (CG's residual norm is not monotone, and
                                     after the 1-3 iterations a step runs it is often
                                     above r_0 for a good direction) */ };
enum { PERF_EXIT_FIXED = 0, PERF_EXIT_EPS = 1, PERF_EXIT_STALL = 2,
       PERF_EXIT_BREAKDOWN = 3, PERF_EXIT_NONFINITE = 4 };

#define PERF_MAX_SHELLS 8

typedef struct perf_ctx perf_ctx;
typedef struct perf_lpc perf_lpc;

/* Scene geometry (Section "Method"; Fig. "scene"). */
typedef struct {
    int32_t grid_res;                      /* 2 <= G <= 1024 */
    int32_t n_shells;                      /* S in [0, 8] */
    float shell_radii[PERF_MAX_SHELLS];    /* increasing, each > sqrt(3) */
    int32_t env_h, env_w;                  /* texels per shell, >= 2 if S > 0 */
    int32_t dtype;                         /* PERF_F32 or PERF_BF16 */
    int32_t env_kind;                      /* PERF_ENV_EQUIRECT or PERF_ENV_CUBE */
} perf_scene;

/* Shell parametrisations.  Equirectangular: texel (row, col) of an env_h x
 * env_w map, row 0 at the +z pole, u = (atan2(y, x) / 2 pi + 1/2) env_w - 1/2
 * wrapped in azimuth, v = (polar angle / pi) env_h - 1/2 clamped.  Cube map
 * (Section "Implementation": the paper's environment maps are cube maps):
 * env_w = 6 env_h, F = env_h texels per face edge, face f = +x, -x, +y, -y,
 * +z, -z in columns [f F, (f + 1) F); a hit point q lies on the face of its
 * largest |q_a| (ties to the lower axis); with (b, c) the other axes in
 * increasing order, column coordinate u = (q_b / |q_a|) F/2 + F/2 - 1/2 and row
 * coordinate v = (q_c / |q_a|) F/2 + F/2 - 1/2 (texel i centred at i),
 * bilinear, clamped to the face's edge texels.  The hit point, face and
 * (u, v) are binary32 with every operation rounded once. */
enum { PERF_ENV_EQUIRECT = 0, PERF_ENV_CUBE = 1 };

/* Pinhole cameras: pixel (col, row) has its centre at (col+1/2, row+1/2);
 * camera-space ray ((col+1/2 - W/2)/f, -(row+1/2 - H/2)/f, -1). */
typedef struct {
    int32_t n_cams, width, height;
    const float* c2w;     /* HOST, n_cams x 3 x 4 row-major camera-to-world; copied */
    const float* focal;   /* HOST, n_cams focal lengths in pixels; copied */
} perf_cameras;

typedef struct {
    int32_t max_samples;  /* cap on grid samples per ray (Section "Rendering") */
    int32_t jitter;       /* 1: jitter pixel and sample positions (Section "Jittering") */
    uint64_t seed;        /* jitter seed (SplitMix64 counter stream) */
    uint32_t epoch;       /* jitter epoch; perf_gn_solve uses epoch + step index */
    int32_t pcg_iters;    /* PCG iteration limit per GN step */
    int32_t pcg_fixed;    /* 1: run exactly pcg_iters iterations (no exit test) */
    double pcg_eps_rel;   /* paper mode: exit when R < eps^2 R_0 (Algorithm 2 EPS) */
    double pcg_stall;     /* paper mode: exit when R / R_prev > stall (0.85) */
    double ls_alpha;      /* Algorithm 3 decimation factor (0.7) */
    int32_t ls_max;       /* at most ls_max decimations (the printed loop has no cap) */
    int32_t project;      /* 1: trial points are projected to sigma >= 0, 0 <= c <= 1 */
    int32_t precond;      /* PERF_PRECOND_*; texels always use Jacobi */
    int32_t aux;          /* 1: the auxiliary opacity residual of Section "Auxiliary
                             terms", L = aux_lambda (1 - 4 (T^ - 1/2)^2) with T^ the
                             transmittance at grid exit: every per-ray residual
                             vector (r, J p, the v of J^T v) then has 4 entries per
                             ray, [r_0, r_1, r_2, L] (targets stay 3 per ray).
                             Single-scene contexts only. */
    double aux_lambda;    /* its factor (the paper's 0.1), >= 0 */
    int32_t precond_judge;  /* PERF_JUDGE_* (default PERF_JUDGE_RESIDUAL) */
} perf_options;

typedef struct {
    int32_t iters;        /* PCG iterations taken */
    int32_t exit_reason;  /* PERF_EXIT_* */
    double R0;            /* r_0^T r_0 */
    double R;             /* r_k^T r_k after the last iteration */
    double rz;            /* r_k^T z_k */
} perf_pcg_info;

typedef struct {
    double F_before;      /* F(x) at the start of the step (Eq. 5) */
    double F_after;       /* F at the accepted point (F_before if rejected) */
    double gamma;         /* step length from Algorithm 3 */
    int32_t accepted;     /* 1 if F fell and x was updated */
    int32_t ls_evals;     /* Error(gamma) evaluations */
    perf_pcg_info pcg;
    float ms;             /* device time of the step */
    int32_t precond_fallback;  /* 1: the step's PCG was rerun with Jacobi -- the learned
                                  blocks failed the true-residual test (r^T r after PCG
                                  not below r_0^T r_0, a breakdown or a non-finite
                                  scalar), or no trial point of the line search lowered
                                  F with the step of a block preconditioner (learned or
                                  exact block-Jacobi) */
} perf_gn_stats;

/* Device time per kernel family, from CUDA events recorded on the launching
 * stream around each launch while timing is enabled. */
enum { PERF_T_APPLY = 0,    /* A p: the fused J p / J^T (J p) ray march */
       PERF_T_FORWARD = 1,  /* line-search objective marches (F only) */
       PERF_T_DIAG = 2,     /* diag(J^T J) with J^T r */
       PERF_T_VECTOR = 3,   /* PCG vector kernels (update, exit test, direction) */
       PERF_T_PRECOND = 4,  /* block preconditioner construction (network or block inverse) */
       PERF_T_RESIDUAL = 5, /* the Gauss-Newton step's residual march (r = H^ - C and F) */
       PERF_T_COUNT = 6 };
typedef struct {
    double ms[PERF_T_COUNT];
    int64_t launches[PERF_T_COUNT];
} perf_timing;

/* Ray-tile shape, resident-CTA cap and parameter layout chosen by an
 * autotuner. */
typedef struct {
    int32_t tile_w, tile_h;   /* pixels per warp tile (tile_w * tile_h = 32) */
    int32_t ctas_per_sm;      /* 0 = as many as fit */
    float apply_ms;           /* time of the fastest A p launch */
    int32_t paired;           /* 1: perf_gn_solve's A p reads x and p from paired
                                 32-byte records (FP32 scenes); 0: two arrays */
    int32_t coef;             /* 1: the coefficient-cached A p was timed (it is
                                 what perf_gn_solve runs while the store fits) */
    int32_t brick;            /* block order of a Gauss-Newton step's PCG vectors:
                                 1 canonical, 4 or 8 bricks of that many voxels
                                 per edge (see perf_set_brick) */
} perf_tuning;

/* Fills the defaults: max_samples 512, no jitter, 20 fixed PCG iterations,
 * eps 1e-3, stall 0.85, ls_alpha 0.7, ls_max 20, projection on, Jacobi, no
 * auxiliary residual (aux_lambda 0.1). */
perf_status perf_default_options(perf_options* out);

/* Creates a context for one scene and camera set.  Validates everything
 * (2 <= G <= 1024, 0 <= S <= 8, radii increasing and > sqrt(3), env size >= 2,
 * fewer than 2^31 parameter blocks,
 * cameras >= 0, max_samples >= 1), copies the cameras to the device and
 * allocates the workspace.  On failure *out is NULL. */
perf_status perf_create(perf_ctx** out, const perf_scene* scene,
                        const perf_cameras* cams, const perf_options* opts);
perf_status perf_destroy(perf_ctx* ctx);
perf_status perf_set_options(perf_ctx* ctx, const perf_options* opts);
int64_t perf_param_count(const perf_ctx* ctx);   /* n, or -1 */
int64_t perf_ray_count(const perf_ctx* ctx);     /* N_r, or -1 */
const char* perf_last_error(const perf_ctx* ctx);

/* Eq. 3-4: rgb_out[3 N_r] = H^ per ray (grid march, then the shells in order
 * from the grid exit outwards, Section "Rendering"); T_out[N_r] (may be NULL)
 * = transmittance at the grid exit. */
perf_status perf_render(perf_ctx* ctx, const void* x, float* rgb_out,
                        float* T_out, void* stream);

/* Eq. 5-6: r_out[R N_r] = H^ - C (may be NULL), *F_out (device double,
 * overwritten) = 1/2 sum r^2 accumulated in FP64. */
perf_status perf_residual(perf_ctx* ctx, const void* x, const void* target,
                          void* r_out, double* F_out, void* stream);

/* jp_out[R N_r] = J p: the directional derivative of every ray along p, the
 * per-sample partials of Algorithm 1 chained through the interpolation. */
perf_status perf_jvp(perf_ctx* ctx, const void* x, const float* p,
                     float* jp_out, void* stream);

/* out[n] (+)= J^T v for v[R N_r] (Section "Update step", the scatter of
 * grad r_i (grad r_i^T p)); accumulate = 0 overwrites out. */
perf_status perf_vjp(perf_ctx* ctx, const void* x, const float* v, float* out,
                     int32_t accumulate, void* stream);

/* Section "Preconditioner": diag_out[n] = diag(J^T J) (each row's entry for a
 * parameter is summed over all samples of that ray before squaring);
 * grad_out[n] = J^T r when r[R N_r] and grad_out are given (both or neither). */
perf_status perf_diag_jtj(perf_ctx* ctx, const void* x, const void* r,
                          float* diag_out, float* grad_out, void* stream);

/* A p = J^T (J p) = sum_i grad r_i (grad r_i^T p) without forming J
 * (Section "Update step"); ap_out[n] is overwritten; *pap_out (device double,
 * may be NULL) = p^T A p = |J p|^2 in FP64. */
perf_status perf_apply_normal(perf_ctx* ctx, const void* x, const float* p,
                              float* ap_out, double* pap_out, void* stream);

/* Algorithm 2 on the context's workspace.  perf_pcg_begin starts from
 * Delta_0 = 0 with b = -grad (grad[n] = J^T r) and M = diag(diag[n]);
 * perf_pcg_step runs one iteration at x (A p, the fused vector updates with
 * FP64 inner products, the exit test on the device); *done_out (HOST, may be
 * NULL; synchronises) = 1 once PCG has exited.  perf_pcg_result copies
 * Delta to delta_out[n] (may be NULL) and fills *info (HOST, may be NULL;
 * synchronises). */
perf_status perf_pcg_begin(perf_ctx* ctx, const float* grad, const float* diag,
                           void* stream);
perf_status perf_pcg_step(perf_ctx* ctx, const void* x, int32_t* done_out,
                          void* stream);
perf_status perf_pcg_result(perf_ctx* ctx, float* delta_out,
                            perf_pcg_info* info, void* stream);

/* n_steps Gauss-Newton steps (Eq. 7) on x_inout[n] (float32 master copy, in
 * place; the scene dtype decides the storage the ray marches read): residual
 * and F, gradient and Jacobi diagonal, PCG, Algorithm 3 line search on
 * F(P(x + gamma Delta)), accept only if F falls.  The step's diagonal march
 * also fills the coefficient store when it fits its budget (see
 * perf_set_coef_budget), and the PCG iterations' A p then read it.  stats
 * (HOST, may be NULL) receives n_steps records.  Synchronises (the line
 * search reads one FP64 scalar per trial step). */
perf_status perf_gn_solve(perf_ctx* ctx, float* x_inout, const void* target,
                          int32_t n_steps, perf_gn_stats* stats, void* stream);

/* Block preconditioners for Algorithm 2.  perf_pcg_set_blocks: caller-owned
 * row-major 4x4 blocks (16 floats) for the first n_block grid voxels, used by
 * perf_pcg_* and by perf_gn_solve when precond = PERF_PRECOND_BLOCK4 and no
 * network is set.  perf_set_lpc: a learned preconditioner (not owned) whose
 * blocks perf_gn_solve recomputes every step from that step's x, J^T r,
 * diag(J^T J) and block couplings; PCG is rerun with Jacobi when the learned
 * blocks leave the true residual r^T r not below r_0^T r_0 (the residual
 * judges).  perf_diag_cross: diag(J^T J) and, per grid voxel, the cross
 * entries (colour k, opacity) of its 4x4 block of J^T J (4 floats, the 4th 0). */
perf_status perf_pcg_set_blocks(perf_ctx* ctx, const float* blocks, int64_t n_block);
/* Coefficient-cached A p (no counterpart in the paper: a memory-for-compute
 * trade of this implementation).  Within one Gauss-Newton step x is fixed,
 * so the derivatives of every ray-march sample are too; perf_gn_solve's
 * diagonal march stores them (w_i and dH/dsigma_i, 16 bytes per sample and
 * shell hit, one row of 32 per pixel tile up to the tile's largest sample
 * count) and every PCG iteration's A p then gathers only p and reads the
 * stored values -- the same A p up to rounding.  The store holds the
 * longest prefix of pixel tiles that fits the budget (bytes = -1, default:
 * the free device memory minus 6 GiB at the time of the step; 0: never --
 * marches recompute everything, the store is freed; > 0: at most that many
 * bytes; the store's rows and 4 bytes per ray of prefix lengths, below);
 * the A p of the remaining tiles is recomputed.  A ray's rows past its last
 * non-zero one (samples whose transmittance has underflowed to 0 in
 * binary32, where w_i and dH/dsigma_i are exactly 0) are neither written
 * nor read: the A p adds exactly the same terms.  With the auxiliary
 * residual and a non-zero per-ray factor every row is kept.  The per-call
 * entry points (perf_apply_normal, perf_pcg_step) always recompute.
 * perf_coef_info: bytes held by the store's rows, whether the last
 * Gauss-Newton step (or perf_autotune) used it, and the fraction of tiles
 * it covered (HOST pointers, may be NULL).
 * perf_coef_prefix: after a perf_gn_solve step that used the store, the
 * grid-sample rows its A p reads (sum over the store's rays of the non-zero
 * prefix) and the grid samples of those rays (HOST pointers); synchronises
 * the stream.  PERF_ERR_INVALID_ARG when the last step did not fill the
 * store (or the tiling changed since). */
perf_status perf_set_coef_budget(perf_ctx* ctx, int64_t bytes);
/* Block order of the vectors a Gauss-Newton step's PCG works on (p, A p, the
 * Jacobi diagonal, the gradient, Delta, rho; an implementation choice the
 * paper does not discuss): edge 1 = canonical [z][y][x]; edge 2, 4 or 8 =
 * bricks of edge^3 voxels, bricks and the voxels in a brick each in
 * [z][y][x] order (texel blocks unchanged), so that the 8 corners a sample
 * gathers and the voxels a ray's window flushes share fewer cache lines.  G
 * must be a multiple of edge (else PERF_ERR_INVALID_ARG).  perf_gn_solve
 * applies it to a step only when every A p of the step runs from the
 * coefficient store and the preconditioner works per voxel (Jacobi, exact
 * block-Jacobi); otherwise that step is canonical.  x, the targets and every
 * per-call entry point stay canonical.  perf_autotune sets it. */
perf_status perf_set_brick(perf_ctx* ctx, int32_t edge);
/* With on = 1 (the default), perf_gn_solve runs a fixed-iteration PCG
 * (opts.pcg_fixed, pcg_iters > 1, kernel timing off) as one CUDA graph:
 * captured on a stream of the context, replayed on the caller's stream, and
 * captured again whenever the scene descriptor, the iteration count, the
 * preconditioner or a workspace buffer it uses changes.  The graph takes
 * the per-kernel launch work off the host; on = 0 launches every kernel from
 * the host. */
perf_status perf_set_pcg_graph(perf_ctx* ctx, int32_t on);
perf_status perf_coef_info(perf_ctx* ctx, int64_t* bytes_held, int32_t* last_used,
                           double* coverage);
perf_status perf_coef_prefix(perf_ctx* ctx, int64_t* rows_read, int64_t* rows_total,
                             void* stream);
/* Residual history of the context's last PCG solve (perf_pcg_begin /
 * perf_pcg_step, or the last Gauss-Newton step of perf_gn_solve):
 * R_out[k - 1] = r_k^T r_k after iteration k (Algorithm 2's R), HOST, at most
 * cap values; *count_out = how many were written.  Synchronises. */
perf_status perf_pcg_history(perf_ctx* ctx, double* R_out, int32_t cap, int32_t* count_out);

/* One step of Adam (Kingma & Ba 2015) on the same objective and gradient --
 * the first-order method the paper contrasts Gauss-Newton with (Fig. 1) --
 * for comparisons on equal terms: r = H^ - C and F(x) (Eq. 5-6) into the
 * context's workspace, g = J^T r, then per parameter m = beta1 m + (1 -
 * beta1) g, v = beta2 v + (1 - beta2) g^2 and
 * x = P(x - lr (m / (1 - beta1^t)) / (sqrt(v / (1 - beta2^t)) + eps)), P the
 * projection of perf_options.project.  x, m, v: DEVICE, n floats each (m and
 * v start at zero, t counts steps from 1); target: DEVICE, 3 N_r floats;
 * F_out (DEVICE double, may be NULL) gets F at the x the step started from.
 * FP32 scenes without the auxiliary term (else PERF_ERR_UNSUPPORTED). */
perf_status perf_adam_step(perf_ctx* ctx, float* x, const void* target, float* m, float* v,
                           int32_t t, float lr, float beta1, float beta2, float eps,
                           double* F_out, void* stream);
/* Times the A p launch at x along p (both in the scene storage type; p NULL:
 * p = x) over tile shapes 8x4, 4x8, 16x2, 32x1 and resident-CTA caps
 * {all, 3, 2} (two timed launches each), keeps the fastest for every later
 * ray march of the context unless the default (8x4, no cap) is within 3%,
 * then, for FP32 scenes, times A p from separate x and p arrays against the
 * paired records that perf_gn_solve uses by default and keeps the separate
 * arrays only when 3% faster.  When the coefficient store fits its budget it
 * instead lays the store out for every tile shape, fills it at x and times
 * the coefficient-cached A p over the CTA caps and, at each shape's best cap,
 * in the 4^3 and 8^3 brick orders of perf_set_brick where G allows (same 3%
 * rule; it sets the brick order too).  Reports the choice in *out (HOST, may
 * be NULL).  Uses the PCG workspace; synchronises. */
perf_status perf_autotune(perf_ctx* ctx, const void* x, const void* p, perf_tuning* out,
                          void* stream);
perf_status perf_set_lpc(perf_ctx* ctx, perf_lpc* lpc);
perf_status perf_diag_cross(perf_ctx* ctx, const void* x, float* diag_out, float* cross_out,
                            void* stream);

/* Kernel timing (instrumentation, off by default).  perf_get_timing
 * synchronises the context's pending events and copies the totals to *out
 * (HOST); reset = 1 clears them afterwards. */
perf_status perf_enable_timing(perf_ctx* ctx, int32_t on);
/* Number of kernels this library has launched in the process so far. */
uint64_t perf_launch_count(void);
/* *out (HOST; synchronises) = grid samples + shell hits of one march over all
 * rays of the context (the units of work of every ray-march kernel). */
perf_status perf_sample_count(perf_ctx* ctx, uint64_t* out, void* stream);
/* Counting the A p scatter's vector atomics (instrumentation, off by
 * default).  With device_counter set (DEVICE uint64, zeroed by the caller;
 * NULL turns counting off), every later A p launch of this context
 * (perf_apply_normal and the PCG of perf_pcg_step / perf_gn_solve, from the
 * coefficient store or recomputed) adds to *device_counter the 16-byte
 * vector-atomic lane operations its window flushes issue -- one per active
 * lane of each atomic instruction, the unit of work that bounds A p.  J^T v
 * alone, the diagonal march and the batched forms are not counted.  While
 * on, A p runs a separate instantiation that also votes and counts once per
 * flush instruction (several times slower); the default kernels are
 * unchanged. */
perf_status perf_set_atomic_counter(perf_ctx* ctx, uint64_t* device_counter);
/* *lane_ops_per_s (HOST) = the best rate of 16-byte global vector atomic
 * adds (red.global.add.v4.f32) a plain microbenchmark reaches on the current
 * device: 1216 CTAs x 256 threads, 200 atomics per lane, all lanes active,
 * 1, 4 or 32 distinct addresses per warp instruction (best of the three,
 * each timed after one warm-up run).  Allocates and frees 256 MiB of device
 * memory; synchronises the device. */
perf_status perf_measure_atomic_peak(double* lane_ops_per_s);
perf_status perf_get_timing(perf_ctx* ctx, perf_timing* out, int32_t reset);

/* ------------------------------------------------------------------------
 * Learned block preconditioner (a 4-layer 3x3x3 convolutional network, 16
 * channels, bfloat16 activations and weights copies, FP32 accumulation and
 * master weights).  It maps per-voxel features of one Gauss-Newton system to
 * P_v = D_v^{-1/2} (L_v L_v^T + 1e-3 I) D_v^{-1/2} (D_v: the voxel's Jacobi
 * diagonal; L_v lower triangular with a softplus diagonal), so P is SPD by
 * construction and the initial network (L = I) is Jacobi.  Weights: per
 * layer W[27 taps][16 out][16 in] then bias[16]; perf_lpc_weight_count floats.
 * Features: G^3 x 16 bfloat16.  Probe pairs for training: xi (G^3 x 4) and
 * a_hat = D^{-1/2} A D^{-1/2} xi on the grid voxels, mask (G^3 bytes, may be
 * NULL) selects voxels whose four parameters are observed. */
int64_t perf_lpc_weight_count(void);
perf_status perf_lpc_create(perf_lpc** out, uint64_t seed);
perf_status perf_lpc_destroy(perf_lpc* lpc);
const char* perf_lpc_last_error(const perf_lpc* lpc);
perf_status perf_lpc_get_weights(perf_lpc* lpc, float* host_out);
perf_status perf_lpc_set_weights(perf_lpc* lpc, const float* host_in);
/* feat_out = features from x (G^3 grid blocks), J^T r, diag and cross. */
perf_status perf_lpc_features(perf_lpc* lpc, int32_t G, const float* x, const float* grad,
                              const float* diag, const float* cross, void* feat_out, void* stream);
/* Relative loss sum_v |Q_v a_hat_v - xi_v|^2 / sum |xi|^2 (HOST *loss_out) and
 * its gradient with respect to all weights (grad_out: device floats, may be
 * NULL).  Synchronises. */
perf_status perf_lpc_loss_grad(perf_lpc* lpc, int32_t G, const void* feat, const float* ahat,
                               const float* xi, const uint8_t* mask, double* loss_out,
                               float* grad_out, void* stream);
/* One Adam step (lr) on that loss.  Synchronises. */
perf_status perf_lpc_train_step(perf_lpc* lpc, int32_t G, const void* feat, const float* ahat,
                                const float* xi, const uint8_t* mask, float lr,
                                double* loss_out, void* stream);
/* Raw head outputs (G^3 x 16 bfloat16; channels 0-9 used). */
perf_status perf_lpc_head_outputs(perf_lpc* lpc, int32_t G, const void* feat, void* out,
                                  void* stream);
/* blocks_out (G^3 x 16 floats) = P_v for every grid voxel. */
perf_status perf_lpc_infer(perf_lpc* lpc, int32_t G, const void* feat, const float* diag,
                           float* blocks_out, void* stream);
/* Failure detection of the tcgen05 convolution (Section "Preconditioner" has
 * no counterpart: this is the library's own bounded-wait protocol).  Every
 * wait of the convolution kernel for its TMA loads or its MMAs polls a
 * bounded number of rounds; when one runs out the kernel raises a device
 * flag, waits (bounded) for its loads still in flight, frees its tensor
 * memory and returns, leaving the context usable.  perf_lpc_conv_status
 * reads and clears that flag into HOST *timed_out (1: some convolution since
 * the last read gave up; its outputs are incomplete) and synchronises the
 * device.  perf_lpc_loss_grad / perf_lpc_train_step return PERF_ERR_TIMEOUT
 * when the flag is set; perf_gn_solve falls back to Jacobi for that step.
 * perf_lpc_test_conv_wait_limit is a test hook: later launches give each
 * CTA's first wait `rounds` polling rounds (0: it gives up at once; the
 * default and maximum is 2^20); every other wait keeps the normal limit.
 * Process-wide, not thread-safe. */
perf_status perf_lpc_conv_status(int32_t* timed_out);
perf_status perf_lpc_test_conv_wait_limit(uint32_t rounds);
/* out_v = D_v^{-1/2} in_v on the G^3 grid voxels (4 floats each; 0 where a
 * voxel has an unobserved parameter); mask_out (may be NULL) = 1 where all
 * four parameters are observed.  Prepares probe pairs for training. */
perf_status perf_lpc_dscale(int32_t G, const float* diag, const float* in, float* out,
                            uint8_t* mask_out, void* stream);
/* Exact block-Jacobi: blocks_out = inverse of each voxel's 4x4 block of J^T J
 * (closed form through the Schur complement q of the opacity entry; Jacobi
 * where the block is unobserved or numerically singular, q <= 1e-4 times the
 * opacity diagonal). */
perf_status perf_block_jacobi(int32_t G, const float* diag, const float* cross,
                              float* blocks_out, void* stream);

/* ------------------------------------------------------------------------
 * Batched form: many independent scenes (each its own grid, shells and
 * cameras; float32) solved together.  Parameters, rays, targets and
 * residuals of all scenes are concatenated in scene order; use
 * perf_batch_param_offset / perf_batch_ray_offset (scene = n_scenes gives the
 * totals).  Every ray march is one persistent launch taking (scene, pixel
 * tile) items from a work queue; each scene has its own PCG scalars and its
 * own line search; the PCG loop of opts.pcg_iters iterations is captured
 * once as a CUDA graph (on an internal stream) and replayed each
 * Gauss-Newton step.
 * scenes and cams are HOST arrays of n_scenes entries (cameras copied);
 * validation as perf_create; dtype must be PERF_F32. */
typedef struct perf_batch perf_batch;

perf_status perf_batch_create(perf_batch** out, int32_t n_scenes, const perf_scene* scenes,
                              const perf_cameras* cams, const perf_options* opts);
perf_status perf_batch_destroy(perf_batch* b);
int64_t perf_batch_param_offset(const perf_batch* b, int32_t scene);
int64_t perf_batch_ray_offset(const perf_batch* b, int32_t scene);
const char* perf_batch_last_error(const perf_batch* b);
/* rgb_out[3 N_r total] = H^ of every scene's rays (Eq. 3-4). */
perf_status perf_batch_render(perf_batch* b, const float* x, float* rgb_out, void* stream);
/* r_out (may be NULL) = H^ - C; F_out[n_scenes] (device doubles) = 1/2 sum r^2 per scene. */
perf_status perf_batch_residual(perf_batch* b, const float* x, const float* target,
                                float* r_out, double* F_out, void* stream);
/* Times the A p launch at x over tile shapes 8x4, 4x8, 16x2, 32x1 and CTA caps
 * {all, 3, 2}, keeps the fastest (used by every later launch) and reports it
 * in *out (HOST, may be NULL); with the coefficient store (when it fits) the
 * coefficient-cached A p is timed, its store filled at x, and at each tile
 * shape's best cap also in the 4^3 and 8^3 brick orders (perf_batch_set_brick;
 * scenes whose G the edge does not divide stay canonical).  Synchronises. */
perf_status perf_batch_autotune(perf_batch* b, const float* x, perf_tuning* out, void* stream);
/* The coefficient store of perf_set_coef_budget for a batch (rows over the
 * batch's global pixel-tile list; perf_batch_gn_solve's diagonal march fills
 * it and the captured PCG loop reads it). */
perf_status perf_batch_set_coef_budget(perf_batch* b, int64_t bytes);
/* perf_set_brick for a batch: edge 1, 2, 4 or 8; each scene whose G is a
 * multiple of edge takes that brick order in the Gauss-Newton steps whose A p
 * runs from the store, the others stay canonical.  perf_batch_autotune sets
 * it. */
perf_status perf_batch_set_brick(perf_batch* b, int32_t edge);
perf_status perf_batch_coef_info(perf_batch* b, int64_t* bytes_held, int32_t* last_used);
/* n_steps Gauss-Newton steps for every scene (Algorithm 2 per scene: with
 * opts.pcg_fixed exactly opts.pcg_iters iterations, else at most that many
 * with the exit tests of perf_options, a scene's device exit flag making
 * every later A p launch of the captured loop skip its rays; Algorithm 3 per
 * scene, accept per scene).  stats (HOST, may be NULL) receives
 * n_steps * n_scenes records, step-major.  Synchronises. */
perf_status perf_batch_gn_solve(perf_batch* b, float* x, const float* target, int32_t n_steps,
                                perf_gn_stats* stats, void* stream);

/* perf_render with the rendering threshold of Section "Rendering" for a
 * converged scene: a ray whose total opacity within the volume, 1 - T at
 * grid exit, is below min_opacity (the paper uses 0.7) sees the volume as
 * fully transparent and renders the shells only.  T_out (may be NULL)
 * receives T at grid exit before the threshold.  min_opacity in [0, 1]
 * (0: plain perf_render). */
perf_status perf_render_threshold(perf_ctx* ctx, const void* x, float min_opacity,
                                  float* rgb_out, float* T_out, void* stream);

/* Level change of the hierarchical formulation (Section "Hierarchical
 * formulation"): fills the parameters of the next level -- grid 2G x 2G x 2G,
 * environment maps 2 env_h x 2 env_w -- from level (G, env_h x env_w) by
 * linear interpolation at the new cell centres (fine cell i' at coarse index
 * coordinate i'/2 - 1/4): trilinear on the grid with the ray march's edge
 * clamp, bilinear on the maps with the longitude wrapped and the latitude
 * clamped.  Grid opacity is per voxel side and is halved (the optical depth
 * of every path is kept); shell opacity is kept.  x: 4 (G^3 + S env_h env_w)
 * floats, x_out: 4 (8 G^3 + 4 S env_h env_w) floats, both DEVICE, not
 * overlapping (else PERF_ERR_INVALID_ARG).  2 <= G <= 512.  env_kind
 * PERF_ENV_CUBE: the maps are cube maps (env_w = 6 env_h), each face
 * upsampled on its own with both axes clamped at its edges.  No context; the
 * work is queued on stream (cudaStream_t). */
perf_status perf_upsample(const float* x, int32_t G, int32_t n_shells, int32_t env_h,
                          int32_t env_w, int32_t env_kind, float* x_out, void* stream);

/* Residual and objective without a context and without any device
 * allocation -- the paper has no counterpart; this serves callers that cannot
 * allocate device memory when they need a residual (a device-memory budget
 * fixed at start-up, a host engine whose own pool allocator owns all device
 * memory, a latency-critical loop that must avoid cudaMalloc / cudaFree).
 * Same result as perf_create + perf_residual with the same arguments:
 * r_out[3 N_r] (may be NULL) = H^ - C and *F_out (device double, overwritten)
 * = 1/2 sum r^2.  scene, cams (HOST arrays) and opts are validated as in
 * perf_create; at most PERF_NOALLOC_MAX_CAMS cameras (more returns
 * PERF_ERR_INVALID_ARG).  The camera table is staged in one file-scope device
 * array of PERF_NOALLOC_MAX_CAMS x 64 bytes (256 KiB), held by every GPU that
 * loads the library until the process exits, and shared by every call:
 * calls that overlap on the GPU race on it, so serialise them (one stream,
 * or events).  The first call on a device looks up that array's device
 * address (cudaGetSymbolAddress) with the device current; make that first
 * call before any stream capture.  Not thread-safe: one host thread at a time.
 * Allocates nothing: no cudaMalloc, cudaFree or allocating library call.
 * The auxiliary residual (opts->aux) is not supported here
 * (PERF_ERR_UNSUPPORTED). */
#define PERF_NOALLOC_MAX_CAMS 4096
perf_status perf_residual_noalloc(const perf_scene* scene, const perf_cameras* cams,
                                  const perf_options* opts, const void* x,
                                  const void* target, void* r_out, double* F_out,
                                  void* stream);

#ifdef __cplusplus
}
#endif
#endif /* PERF_H */

// perf_kernels.h -- host launchers of the libperf kernels (internal).
#pragma once
#include <cuda_runtime.h>
#include "perf_device.cuh"

namespace perf {

// One scene of a batch: its geometry and where its parameters, rays and
// tiles start in the batch's concatenated vectors / work queue.
struct BatchItem {
    DevScene sc;
    long long x_off;      // first parameter (floats; multiple of 4)
    long long r_off;      // first ray
    long long tile_off;   // first tile in the work queue
};

// Batched ray marches over many scenes in one persistent launch: warps take
// tiles from the work queue `counter` (zeroed here); `start[n]` are the
// scenes' first tiles.  Forward: mode 0 image into res, 1 residual
// (+F[scene]), 2 F[scene] only,
// scenes with active[s] == 0 skipped (active may be null).  Scatter: mode 1
// A p (+ p^T A p into pap[scene * pap_stride]), 2 diag (+ grad with v = r).
cudaError_t launch_forward_batch(const BatchItem* items, const long long* start, int n,
                                 long long total, unsigned long long* counter, const float* x,
                                 const float* target, float* res, double* F, const int* active,
                                 int mode, int cap_per_sm, cudaStream_t st);
struct PcgScalars;
// pcg (may be null): per-scene Algorithm 2 state; scenes whose solve has
// exited (done) are skipped.
// coef / tile_off (mode 2, may be null): also store the per-sample
// coefficients, tile_off indexed by the global tile list.
cudaError_t launch_scatter_batch(const BatchItem* items, const long long* start, int n,
                                 long long total, unsigned long long* counter, const float* x,
                                 const float* p, const float* v, float* out, float* out2,
                                 double* pap, int pap_stride, int mode, int cap_per_sm,
                                 cudaStream_t st, const PcgScalars* pcg = nullptr,
                                 float* coef = nullptr, const long long* tile_off = nullptr,
                                 bool brick = false);
// Coefficient-cached A p over a batch, and the rows of every tile of the
// global tile list (see launch_tile_rows).  brick: p and A p of each scene
// are in the block order of its items[i].sc layout (else all canonical).
cudaError_t launch_apply_coef_batch(const BatchItem* items, const long long* start, int n,
                                    long long total, unsigned long long* counter, const float* p,
                                    const float* coef, const long long* tile_off, float* out,
                                    double* pap, int pap_stride, int cap_per_sm, cudaStream_t st,
                                    const PcgScalars* pcg, bool brick = false);
cudaError_t launch_tile_rows_batch(const BatchItem* items, const long long* start, int n,
                                   long long total, int* rows, cudaStream_t st);

// Device scalars of Algorithm 2 and the line search (FP64).
struct PcgScalars {
    double rz;        // r_k^T z_k
    double R0;        // r_0^T r_0
    double R_prev;    // r_{k}^T r_{k} of the previous iteration
    double R;         // latest r^T r
    double pAp;       // accumulator: p^T A p
    double acc_R;     // accumulator: r_{k+1}^T r_{k+1}
    double acc_rz;    // accumulator: r_{k+1}^T z_{k+1}
    double beta;
    double F;         // accumulator: objective
    int iter;
    int done;
    int exit_reason;
    int max_iter;
    int fixed;
    int pad;
    double eps_rel;
    double stall;
    double* hist;     // null, or R after iteration k written to hist[k - 1] (k <= hist_cap)
    long long hist_cap;
};

// Sets the parameter-vector block order of d (see LayoutKey): s = 0 the
// canonical order, s > 0 bricks of 2^s voxels per edge.  Returns false (and
// leaves d canonical) when G is not a multiple of the brick edge.
inline bool set_layout(DevScene& d, int s) {
    const long long G = d.G;
    if (s <= 0 || G % (1ll << s) != 0) {
        d.lay_s = 0;
        d.lay_ys = (int)G;
        d.lay_zs = (int)(G * G);
        return s <= 0;
    }
    const long long B = 1ll << s, nb = G / B;
    d.lay_s = s;
    d.lay_ys = (int)(nb * B * B * B);
    d.lay_zs = (int)(nb * nb * B * B * B);
    return true;
}

// Kernels launched by this library since load (instrumentation).
extern unsigned long long g_launches;
inline void count_launch(unsigned long long k = 1) { __atomic_fetch_add(&g_launches, k, __ATOMIC_RELAXED); }

// Total grid samples and shell hits over all rays (one march of the scene).
cudaError_t launch_count_samples(const DevScene& sc, unsigned long long* out, cudaStream_t st);

// mode: 0 render (out = float rgb, T_out), 1 residual (out = r, F), 2 F only.
// target and the residual are in the scene's storage type (float / bf16).
// cut (mode 0): the rendering opacity threshold (see composite in k_march.cu).
cudaError_t launch_forward(const DevScene& sc, int dtype, const void* x, const void* target,
                           void* out, float* T_out, double* F, int mode, cudaStream_t st,
                           float cut = 0.0f);
cudaError_t launch_jvp(const DevScene& sc, int dtype, const void* x, const void* p, int p_dtype,
                       float* out, cudaStream_t st);
// mode: 0 J^T v (v float32), 1 A p (+p^T A p), 2 diag(J^T J) (+ J^T r when v = r,
// in the scene's storage type, and out2 given).
// out3 (mode 2, may be null): per grid voxel the cross entries (colour k,
// opacity) of the 4x4 diagonal block of J^T J.
// coef / tile_off (mode 2, may be null): also store the per-sample
// coefficients (w_i, dH/dsigma_i) of the coefficient-cached A p.
cudaError_t launch_scatter(const DevScene& sc, int dtype, int mode, const void* x, const void* p,
                           int p_dtype, const void* v, float* out, float* out2, double* pap,
                           cudaStream_t st, float* out3 = nullptr, float* coef = nullptr,
                           const long long* tile_off = nullptr);
// Coefficient-cached A p (k_march.cu): rows[t] = rows of pixel tile t in the
// coefficient store (its largest grid sample count + shells); A p (+p^T A p)
// from p (p_dtype: 0 float, 1 bf16) and the stored coefficients.
cudaError_t launch_tile_rows(const DevScene& sc, int* rows, cudaStream_t st);
// sums[0] += sum of keff[ray], sums[1] += sum of K over the rays of tiles
// [tile_lo, n_tiles) of sc
cudaError_t launch_coef_prefix(const DevScene& sc, const int* keff, unsigned long long* sums,
                               cudaStream_t st);
cudaError_t launch_apply_coef(const DevScene& sc, const void* p, int p_dtype, const float* coef,
                              const long long* tile_off, float* out, double* pap, cudaStream_t st);
// A p (+p^T A p) of an FP32 scene from paired records xp[v] = (x[v], p[v])
// (2 n floats, 32-byte aligned).
cudaError_t launch_apply_pair(const DevScene& sc, const float* xp, float* out, double* pap,
                              cudaStream_t st);

// Shell-hit table of a scene (k_march.cu): n_rays x S float4 entries (first
// texel index, fu, fv, column step) for the shells each ray hits, equirect
// texel coordinates in FP64; a march reads it when sc.shell_tab is set.
cudaError_t launch_shell_table(const DevScene& sc, float4* tab, cudaStream_t st);

// Algorithm 2 vector work (k_pcg.cu).  Delta, rho, p: FP32 (p is also the
// array the ray march gathers); p16 (may be null): its BF16 copy for BF16
// scenes; Ap: FP32 scatter target, zeroed by begin and update; pxp (may be
// null): paired x / p records whose p half also receives p.
cudaError_t launch_pcg_begin(long long n, const float* grad, const float* diag, float* delta,
                             float* rho, float* p, __nv_bfloat16* p16, float* Ap, PcgScalars* s,
                             int max_iter, int fixed, double eps_rel, double stall,
                             const float* blocks, long long n_block, cudaStream_t st,
                             float* pxp = nullptr, double* hist = nullptr, long long hist_cap = 0);
cudaError_t launch_pcg_update(long long n, float* delta, float* rho, const float* p, float* Ap,
                              const float* diag, const float* blocks, long long n_block,
                              PcgScalars* s, cudaStream_t st);
// One thread: the exit test of Algorithm 2 and beta (after launch_pcg_update).
cudaError_t launch_pcg_finish(PcgScalars* s, cudaStream_t st);
cudaError_t launch_pcg_dir(long long n, const float* rho, const float* diag, const float* blocks,
                           long long n_block, float* p, __nv_bfloat16* p16, PcgScalars* s,
                           cudaStream_t st, float* pxp = nullptr);
// xp[v] = (x[v], p[v]) for the n / 4 parameter blocks (p null: x half only).
cudaError_t launch_pair_pack(long long n, const float* x, const float* p, float* xp,
                             cudaStream_t st);
// x_out = P(x + gamma delta) (project: sigma >= 0, 0 <= c <= 1), formed in FP64;
// optional float32 and bf16 outputs.  delta is in the block order lay
// (x = G, y = brick shift s, z = ys, w = zs of the LayoutKey; y = 0:
// canonical, the default), x and the outputs are canonical.
cudaError_t launch_trial(long long n, const float* x, const float* delta, double gamma,
                         int project, float* x_out, __nv_bfloat16* x16_out, cudaStream_t st,
                         int4 lay = int4{0, 0, 0, 0});
// The int4 block order of d for launch_trial.
inline int4 layout_of(const DevScene& d) { return int4{d.G, d.lay_s, d.lay_ys, d.lay_zs}; }
cudaError_t launch_to_bf16(long long n, const float* x, __nv_bfloat16* y, cudaStream_t st);
// One Adam step with projection (k_pcg.cu); c1, c2 the bias corrections.
cudaError_t launch_adam(long long n, float* x, const float* g, float* m, float* v, float b1,
                        float b2, float lr, float eps, float c1, float c2, int project,
                        cudaStream_t st);

// Segmented forms (a batch of independent systems, scalars s[y] for system
// y < n_seg): chunks (device, n_chunks int4) assigns CTA b the parameter
// blocks [chunks[b].y, chunks[b].z) of system chunks[b].x; null = one system.
cudaError_t launch_pcg_begin_seg(long long n, int n_seg, const int4* chunks, long long n_chunks,
                                 const float* grad, const float* diag, float* delta, float* rho,
                                 float* p, __nv_bfloat16* p16, float* Ap, PcgScalars* s,
                                 int max_iter, int fixed, double eps_rel, double stall,
                                 const float* blocks, long long n_block, cudaStream_t st,
                                 float* pxp = nullptr);
cudaError_t launch_pcg_update_seg(long long n, int n_seg, const int4* chunks, long long n_chunks,
                                  float* delta, float* rho, const float* p, float* Ap,
                                  const float* diag, const float* blocks, long long n_block,
                                  PcgScalars* s, cudaStream_t st);
cudaError_t launch_pcg_finish_seg(PcgScalars* s, int n_seg, cudaStream_t st);
cudaError_t launch_pcg_dir_seg(long long n, int n_seg, const int4* chunks, long long n_chunks,
                               const float* rho, const float* diag, const float* blocks,
                               long long n_block, float* p, __nv_bfloat16* p16, PcgScalars* s,
                               cudaStream_t st, float* pxp = nullptr);
// Segment y: x_out = P(x + gamma[y] Delta) where mask[y] (or every segment).
// lay / base (device, n_seg entries each, may be null): segment y's Delta is
// in the block order lay[y] (see launch_trial) from its first block base[y].
cudaError_t launch_trial_seg(long long n, int n_seg, const int4* chunks, long long n_chunks,
                             const float* x, const float* delta, const double* gamma,
                             const int* mask, int project, float* x_out, cudaStream_t st,
                             const int4* lay = nullptr, const long long* base = nullptr);

// Level change of the hierarchical formulation (k_hier.cu): y (level 2G,
// maps 2He x 2We) from x (level G, maps He x We).
cudaError_t launch_upsample(const float* x, int G, int S, int He, int We, int cube, float* y,
                            cudaStream_t st);

}  // namespace perf

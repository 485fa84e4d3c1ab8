#!/usr/bin/env python
"""Benchmark of the PERF Gauss-Newton step on GB300.

One step = one Gauss-Newton step of the 128^3 workload (3 shells 256x512,
100 cameras 800x800, up to 256 samples per ray): residuals and F, gradient
and exact Jacobi diagonal, 50 fixed PCG iterations (each one A p ray march
plus the fused vector kernels), and the Algorithm 3 line search.  The metric
is PCG iterations per second over whole Gauss-Newton steps (line search and
set-up included).  Inputs are synthetic (seeded scene, targets rendered from
the voxelised ground truth); the targets (768 MB) and residuals (768 MB) are
larger than L2, so every step streams them from HBM.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

The JSON line's roofline object measures the dominant kernel (A p) against
HBM (algorithmic bytes per launch / CUDA-event time, with the DRAM traffic
of an ncu capture while the sources match it) and, under "atomics", against
the 16-byte vector-atomic throughput the library's microbenchmark measures
in the same process (its lane operations counted on one extra, untimed
Gauss-Newton step).

With N > 1 (torchrun) every rank runs an independent replica of the
workload (the single-scene step has no exchange to shard without a
collective); value = all ranks' PCG iterations / max-over-ranks time.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np

WORKLOAD = "scale128"
METRIC = "PCG iters/s"

# The method's algorithmic work per ray-march sample of one A p (the fused
# J p and J^T (J p) of a PCG iteration), as the scope of the hot path counts
# it: trilinear interpolation of x and p (64 FMA), the compositing weights
# and Algorithm 1's recurrence, and the 32-element scatter products -- about
# 200 FP32 FLOP per sample (exponentials are special-function work, not
# FLOP).  The A p roofline is this work per launch over the launch's time,
# against the FP32 peak (SMs x 128 lanes x 2 FLOP x max SM clock).
FLOP_PER_SAMPLE_METHOD = 200
# What each A p implementation executes per sample (reported beside it):
# the recomputing march runs an optical-depth sweep, the J p sweep and the
# adjoint sweep (345 FLOP: four 4-channel interpolations at 56, compensated
# depth, Algorithm 1 partials twice, window accumulation); the coefficient-
# cached A p streams stored partials instead (207 FLOP: interpolation of p
# with corner weights 116, J p update 12, window weights and accumulation 44,
# v.dH/dsigma 6, flushed colour entries scaled by v 14 on average).
FLOP_PER_SAMPLE_RECOMPUTE = 345
FLOP_PER_SAMPLE_COEF = 207
# Compulsory HBM bytes of one A p: read x and p, zero and flush A p -- four
# n-vector passes of 4 bytes (16 bytes per parameter).
APPLY_COMPULSORY_BYTES_PER_PARAM = 16
# Design traffic of the coefficient-cached A p: the per-sample coefficients
# (16 bytes, stored by the step's diagonal march) streamed twice per launch,
# plus p read once and A p written once (8 bytes per parameter).
COEF_BYTES_PER_SAMPLE = 32
# PCG vector kernels per iteration: update reads p, A p, Delta, rho, d (20 B)
# and writes Delta, rho, A p = 0 (12 B); direction reads rho, d, p (12 B) and
# writes p (4 B): 48 bytes per parameter (+2 for the BF16 copy of p, +4 for
# the p half of the paired records).  The scope's count for the fused vector
# work is 11 n-vector passes of 4 bytes (44 bytes per parameter).
VEC_BYTES_PER_PARAM = 48
VEC_COMPULSORY_BYTES_PER_PARAM = 44
# The residual pass streams the targets C in and the residuals r out: 12 + 12
# bytes per ray in FP32 (6 + 6 in BF16); its ray march gathers x from L2.
RESIDUAL_BYTES_PER_RAY_F32 = 24

# DRAM traffic of one A p launch, from the ncu capture summarised in this
# file (a small case, scaled to a full launch by its sample count); it applies
# only while the kernel sources hash to the recorded value.
TRAFFIC_PROFILE = os.path.join(ROOT, "profiles", "apply_coef_traffic_scale128.md")
KERNEL_SOURCES = ("paper_2112_05598_gb300/csrc/k_march.cu",
                  "paper_2112_05598_gb300/csrc/perf_device.cuh")


def kernel_source_hash():
    """SHA-256 of the kernel sources with comments and whitespace removed
    (a comment edit does not change the kernels)."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f)) as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()


def recorded_traffic(kernel, workload, samples, rows_read=1.0):
    """DRAM bytes per launch of `kernel` on `workload` with `samples` ray-march
    samples of which the fraction `rows_read` is streamed from the store
    (each ray's non-zero prefix): the recorded capture's bytes scaled by the
    rows streamed over the capture's (the coefficient stream, which
    dominates, is proportional to them).  None when the record is missing or
    was taken on other kernel sources."""
    try:
        with open(TRAFFIC_PROFILE) as fh:
            kv = {}
            for line in fh:
                if ":" in line and line.startswith("- "):
                    k, v = line[2:].split(":", 1)
                    kv[k.strip()] = v.strip().strip("`")
    except OSError:
        return None
    if (kv.get("kernel") != kernel or kv.get("workload") != workload
            or kv.get("source_sha256") != kernel_source_hash()):
        return None
    try:
        dram = int(kv["dram_bytes_per_launch"])
        cap = int(kv["samples_per_launch"]) * float(kv.get("rows_read_fraction", "1.0"))
    except (KeyError, ValueError):
        return None
    return int(round(dram * samples * rows_read / cap)) if cap > 0 else None


def cpu_model():
    """The host CPU's model name (x86 'model name'; Arm: lscpu's model)."""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        kv = dict((a.strip(), b.strip()) for a, b in
                  (ln.split(":", 1) for ln in out.splitlines() if ":" in ln))
        name = kv.get("Model name") or ""
        vendor = kv.get("Vendor ID") or ""
        return (vendor + " " + name).strip() or None
    except Exception:
        return None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--dtype", default="f32", choices=["f32", "bf16"])
    ap.add_argument("--cams", type=int, default=None, help="first N cameras only (profiling)")
    ap.add_argument("--grid", type=int, default=None,
                    help="grid resolution G in place of the workload's (sample cap 2 G, as in the "
                         "workloads: about the grid's diagonal in steps of 2/G)")
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-cams", type=int, default=16)
    ap.add_argument("--lpc", action="store_true", help="learned vs Jacobi preconditioner study")
    ap.add_argument("--hier", action="store_true", help="hierarchical vs single-level study")
    ap.add_argument("--hier-steps", type=int, default=30)
    ap.add_argument("--hier-pcg", type=int, default=3)
    ap.add_argument("--hier-levels", type=int, default=3,
                    help="levels of the coarse-to-fine study (the first at G / 2^(levels-1))")
    ap.add_argument("--lpc-scenes", type=int, default=100)
    ap.add_argument("--lpc-steps", type=int, default=20)
    ap.add_argument("--lpc-epochs", type=int, default=2)
    ap.add_argument("--lpc-gn", type=int, default=40)
    ap.add_argument("--lpc-pcg", type=int, default=2)
    ap.add_argument("--lpc-traj", type=int, default=400)
    ap.add_argument("--no-lpc-record", action="store_true",
                    help="leave the learned-preconditioner record out of the default line")
    ap.add_argument("--brick", type=int, default=0,
                    help="fix the brick edge of the PCG vectors (1, 2, 4, 8) after autotuning")
    ap.add_argument("--coef-budget", type=int, default=-1,
                    help="bytes for the coefficient store (-1: free memory - 6 GiB; 0: off, every "
                         "A p recomputes)")
    ap.add_argument("--compare", action="store_true",
                    help="32^3 workload: Gauss-Newton vs Adam (time to held-out PSNR) and "
                         "equirectangular vs cube-map shells")
    ap.add_argument("--conv", type=int, default=0,
                    help="time the learned preconditioner's 4-layer network on a G^3 grid")
    return ap.parse_args()


def dist_setup(n_gpus):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _reduce(v, world, op):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(v, world):
    import torch.distributed as dist
    return _reduce(v, world, dist.ReduceOp.MAX if world > 1 else None)


def sum_over_ranks(v, world):
    import torch.distributed as dist
    return _reduce(v, world, dist.ReduceOp.SUM if world > 1 else None)


def replica_value(units, ms, world):
    """Whole-job throughput of independent replicas: all ranks' units over
    the slowest rank's time (each rank brackets its timed region with a
    barrier and a synchronize)."""
    return sum_over_ranks(float(units), world) / (max_over_ranks(ms, world) / 1000.0)


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [c.strip() for c in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def cpu_baseline(scene, n_cams, pcg_per_gn):
    """The FP64 oracle on a bounded sample: A p (Algorithm 1 twice per ray) on
    the first n_cams cameras, scaled to all cameras -> PCG iterations/s."""
    from oracle import Oracle
    orc = Oracle(scene.G, scene.radii, scene.env_h, scene.env_w, scene.c2w[:n_cams],
                 scene.focal[:n_cams], scene.width, scene.height,
                 max_samples=scene.cfg.max_samples)
    x = scene.x0.astype(np.float64)
    p = np.random.default_rng(0).normal(size=scene.n_params)
    t0 = time.perf_counter()
    orc.apply_A(x, p)
    dt = time.perf_counter() - t0
    full = dt * scene.n_cams / n_cams
    return {"value": 1.0 / full, "unit": METRIC, "cores": os.cpu_count(), "cpu": cpu_model(),
            "kind": "oracle",
            "sample": f"one A p (J p then J^T v, FP64, OpenMP over rays) on {n_cams} of "
                      f"{scene.n_cams} cameras ({orc.n_rays} rays, {dt:.1f} s), scaled by the "
                      f"ray count; PCG vector work (O(n)) not included"}


def run_reference(args, rank, world):
    from scenegen import make_scene
    if rank != 0:
        return
    sc = make_scene(_scene_config(args))
    vals = []
    for _ in range(args.warmup + args.steps):
        vals.append(cpu_baseline(sc, args.cpu_cams, sc.cfg.pcg_iters))
    timed = vals[args.warmup:]
    v = statistics.median([b["value"] for b in timed])
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": METRIC,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * sc.cfg.pcg_iters / v, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": _workload_desc(sc)},
            "cpu_baseline": {"value": v, "unit": METRIC, "cores": os.cpu_count(),
                             "cpu": cpu_model(), "kind": "oracle", "sample": timed[0]["sample"]},
            "e2e": {"value": v, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _scene_config(args):
    """The workload's scene configuration, at --grid G if given (sample cap
    2 G, the workloads' own ratio)."""
    import dataclasses
    from scenegen import CONFIGS
    cfg = CONFIGS[args.workload]
    if args.grid is not None:
        cfg = dataclasses.replace(cfg, G=args.grid, max_samples=2 * args.grid)
    return cfg


def _workload_desc(sc):
    c = sc.cfg
    return (f"{c.name}: {c.G}^3 RGBA grid + {len(c.radii)} shells {c.env_h}x{c.env_w} "
            f"(radii {','.join(str(r) for r in c.radii)}), {c.n_cams} cameras {c.width}x{c.height}, "
            f"<= {c.max_samples} samples/ray, {c.pcg_iters} fixed Jacobi-PCG iterations per GN step")


BATCH_PCG = 20


def _psnr_from_F(F, n_rays):
    mse = 2.0 * F / (3.0 * n_rays)
    return float("inf") if mse <= 0 else 10.0 * np.log10(1.0 / mse)


def run_conv(args, rank, world, local):
    """The learned preconditioner's network (4 layers of 3x3x3 convolution,
    16 channels, bf16 activations) on a --conv G grid of random features:
    the tcgen05 convolution's throughput against the measured bf16 tensor
    peak, and its activation traffic (32 bytes read + 32 written per voxel and
    layer) against the measured HBM bandwidth."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2112_05598_gb300 import LPC
    from paper_2112_05598_gb300._binding import launch_count
    torch.cuda.set_device(local)
    G = args.conv
    net = LPC(seed=1)
    gen = torch.Generator(device="cuda").manual_seed(0)
    feat = torch.randn(16 * G ** 3, device="cuda", generator=gen).to(torch.bfloat16)
    out = torch.empty(16 * G ** 3, dtype=torch.bfloat16, device="cuda")
    for _ in range(max(args.warmup, 3)):
        net.head_outputs(G, feat, out)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    l0 = launch_count()
    e0.record(stream)
    for _ in range(args.steps):
        net.head_outputs(G, feat, out)
    e1.record(stream)
    torch.cuda.synchronize()
    launches = launch_count() - l0
    ms = e0.elapsed_time(e1) / args.steps
    layers = 4
    flop = layers * G ** 3 * 27 * 16 * 16 * 2
    byts = layers * G ** 3 * 64
    peaks, src = measured_peaks()
    tf = flop / (ms * 1e-3) / 1e12
    line = {"metric": "conv TFLOP/s", "value": tf, "unit": "TFLOP/s", "n_gpus": 1,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms,
            "higher_is_better": True, "dtype": "bf16", "data": "synthetic (random features)",
            "config": {"workload": f"learned-preconditioner network, {G}^3 grid, 4 layers, "
                                   f"16 channels, 3x3x3 taps"},
            "gpu_launches": launches,
            "roofline": {"bound": "tensor", "achieved": tf, "peak": peaks["bf16_tflops"],
                         "unit": "TFLOP/s", "frac": tf / peaks["bf16_tflops"],
                         "peak_source": f"bf16_tflops ({src})",
                         "hbm_frac": byts / (ms * 1e-3) / 1e9 / peaks["hbm_gbs"],
                         "kernel": "k_conv_fwd_tc (tcgen05, TMA halo staging)"}}
    if rank == 0:
        print(json.dumps(line), flush=True)


def lpc_study(dev, workload, n_cams=None, train_small=100, train_steps=20, train_large=8,
              epochs=2, gn_steps=20, pcg_per_step=5, traj_iters=300, seed=7, train_pcg=5):
    """Learned block preconditioner vs Jacobi (and exact block-Jacobi).

    Training: the network learns from Gauss-Newton systems the solver logs on
    its own runs (train_pcg fixed PCG iterations per step) -- train_small
    seeded 32^3 scenes (train_steps steps each) and train_large systems of the
    128^3 workload restricted to 8 cameras -- with the library's BF16 kernels.  Evaluation on `workload`: (a) the first
    Gauss-Newton system's PCG through the solver's own path (coefficient
    store) until a relative residual of 1e-3 or traj_iters iterations: the
    residual history and the iterations to 1e-1, 1e-2, 1e-3; (b) gn_steps
    Gauss-Newton steps from the workload's start in two PCG regimes -- the
    paper's (at most 3 iterations with its residual and stall exits) and
    pcg_per_step fixed iterations -- held-out-view PSNR against device time,
    and the time each method needs to reach Jacobi's final PSNR - 0.1 dB in
    the same regime."""
    import torch
    from paper_2112_05598_gb300 import (Context, LPC, PERF_PRECOND_BLOCK4,
                                        PERF_PRECOND_BLOCK_JACOBI, PERF_PRECOND_JACOBI)
    from paper_2112_05598_gb300 import lpc_train as T
    from scenegen import make_scene
    gen = torch.Generator(device=dev).manual_seed(0)
    t0 = time.perf_counter()
    net = LPC(seed=seed)
    systems = []
    for k in range(train_small):
        sc = make_scene("small32", seed=2000 + k)
        ctx = Context.from_scene(sc, pcg_iters=train_pcg, pcg_fixed=1)
        target = torch.empty(3 * ctx.n_rays, device=dev)
        ctx.render(torch.from_numpy(sc.x_gt).to(dev), target)
        x = torch.from_numpy(sc.x0.copy()).to(dev)
        for _ in range(train_steps):
            systems.append(T.log_system(ctx, net, x, target, n_probes=1, generator=gen))
            ctx.gn_solve(x, target, 1)
        ctx.close()
    if train_large > 0:
        sc = make_scene("scale128", n_cams=8)
        ctx = Context.from_scene(sc, pcg_iters=train_pcg, pcg_fixed=1)
        target = torch.empty(3 * ctx.n_rays, device=dev)
        ctx.render(torch.from_numpy(sc.x_gt).to(dev), target)
        x = torch.from_numpy(sc.x0.copy()).to(dev)
        for _ in range(train_large):
            systems.append(T.log_system(ctx, net, x, target, n_probes=1, generator=gen))
            ctx.gn_solve(x, target, 1)
        ctx.close()
        del x, target
    t_log = time.perf_counter() - t0
    held = systems[:: max(1, len(systems) // max(1, len(systems) // 10))][: max(1, len(systems) // 10)]
    held_ids = {id(h) for h in held}
    train = [s_ for s_ in systems if id(s_) not in held_ids]
    loss0 = T.mean_loss(net, held)
    t0 = time.perf_counter()
    T.train(net, train, epochs=epochs, lr=1e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    loss1 = T.mean_loss(net, held)
    n_sys = len(systems)
    del systems, train, held
    torch.cuda.empty_cache()
    sc = make_scene(workload, n_cams=n_cams)
    ctx = Context.from_scene(sc)
    hold = Context.from_scene(sc, c2w=sc.heldout_c2w, focal=sc.heldout_focal)
    x_gt = torch.from_numpy(sc.x_gt).to(dev)
    target = torch.empty(3 * ctx.n_rays, device=dev)
    ctx.render(x_gt, target)
    htarget = torch.empty(3 * hold.n_rays, device=dev)
    hold.render(x_gt, htarget)
    del x_gt
    F = torch.zeros(1, dtype=torch.float64, device=dev)
    methods = (("jacobi", PERF_PRECOND_JACOBI), ("learned", PERF_PRECOND_BLOCK4),
               ("block_jacobi", PERF_PRECOND_BLOCK_JACOBI))
    x0 = torch.from_numpy(sc.x0.copy()).to(dev)
    first = {}
    for name, pc in methods:
        ctx.set_lpc(net if pc == PERF_PRECOND_BLOCK4 else None)
        it = T.pcg_iterations(ctx, x0, target, pc, eps=1e-3, max_iter=traj_iters)
        rel = it["rel_residual"]
        first[name] = {"iters_to": it["iters_to"], "iters": it["iters"], "exit": it["exit"],
                       "coef_coverage": ctx.coef_info()["coverage"],
                       "ms_per_iter": it["ms"] / max(it["iters"], 1),
                       "rel_residual_at": {str(k): rel[k - 1]
                                           for k in (5, 10, 20, 50, 100, 200, 300, 600, 1200)
                                           if k <= len(rel)},
                       "fallback": it["fallback"]}
    # Gauss-Newton from the workload's start in two PCG regimes: the paper's
    # (at most 3 iterations, exits on a relative residual of 1e-3 or a stall
    # ratio of 0.85) and a fixed count per step
    regimes = {"paper": dict(pcg_iters=3, pcg_fixed=0, pcg_eps_rel=1e-3, pcg_stall=0.85),
               f"fixed{pcg_per_step}": dict(pcg_iters=pcg_per_step, pcg_fixed=1)}
    gn = {}
    for reg, opts in regimes.items():
        runs = {}
        # the learned blocks under both judges of a step's PCG: the true residual
        # (the default) and the objective (the line search)
        gn_methods = methods + (("learned_objective_judge", PERF_PRECOND_BLOCK4),)
        for name, pc in gn_methods:
            x = x0.clone()
            ctx.set_options(precond=pc, precond_judge=int(name == "learned_objective_judge"), **opts)
            ctx.set_lpc(net if pc == PERF_PRECOND_BLOCK4 else None)
            hold.residual(x, htarget, None, F)
            curve = [(0.0, _psnr_from_F(float(F.item()), hold.n_rays))]
            t_acc, fb, iters = 0.0, 0, 0
            for _ in range(gn_steps):
                st = ctx.gn_solve(x, target, 1)[0]
                t_acc += st["ms"] / 1000.0
                fb += int(st["precond_fallback"])
                iters += int(st["pcg_iters"])
                hold.residual(x, htarget, None, F)
                curve.append((t_acc, _psnr_from_F(float(F.item()), hold.n_rays)))
            runs[name] = {"psnr_curve": curve, "fallbacks": fb, "pcg_iters": iters}
        target_db = runs["jacobi"]["psnr_curve"][-1][1] - 0.1

        def time_to(curve):
            return next((t for t, p_ in curve if p_ >= target_db), None)
        gn[reg] = {"steps": gn_steps, "pcg": opts, "target_psnr_db": target_db,
                   "time_to_psnr_s": {k: time_to(v["psnr_curve"]) for k, v in runs.items()},
                   "final_psnr_db": {k: v["psnr_curve"][-1][1] for k, v in runs.items()},
                   "runs": runs}
    ctx.close()
    hold.close()
    return {"workload": f"{workload}: {sc.G}^3, {sc.n_shells} shells {sc.env_h}x{sc.env_w}, "
                        f"{sc.n_cams} cameras {sc.width}x{sc.height} "
                        f"({sc.cfg.cam_layout}), background shell sigma "
                        f"{sc.cfg.background_sigma}",
            "heldout": f"{len(sc.heldout_c2w)} views"
                       + (" on the training ring, midway between training cameras"
                          if sc.cfg.cam_layout == "ring" else f" ({sc.cfg.cam_layout})"),
            "training": {"systems": n_sys, "small32_scenes": train_small,
                         "scale128_systems": train_large, "epochs": epochs, "log_s": t_log,
                         "train_s": t_train, "held_out_probe_loss_identity": loss0,
                         "held_out_probe_loss_trained": loss1},
            "first_system_pcg": first,
            "gn": gn,
            "summary": lpc_summary(gn)}


def lpc_summary(gn):
    """Per PCG regime, each preconditioner's time to Jacobi's final PSNR - 0.1 dB
    over Jacobi's own (< 1: faster than Jacobi; None: target not reached)."""
    out = {}
    for reg, g in gn.items():
        t = g["time_to_psnr_s"]
        tj = t.get("jacobi")
        out[reg] = {name: (t[name] / tj if t.get(name) is not None and tj else None)
                    for name in t if name != "jacobi"}
    return out


def run_lpc(args, rank, world, local):
    """The learned-preconditioner study (lpc_study) on --workload (default
    the full ring workload: 256^3, 4 shells, 150 cameras 960x540 on a ring)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    if rank != 0:
        return
    dev = torch.device("cuda", local)
    wl = args.workload if args.workload != WORKLOAD else "ring256"
    res = lpc_study(dev, wl, n_cams=args.cams, train_small=args.lpc_scenes,
                    train_steps=args.lpc_steps, epochs=args.lpc_epochs, gn_steps=args.lpc_gn,
                    pcg_per_step=args.lpc_pcg, traj_iters=args.lpc_traj)
    print(json.dumps(dict(metric="PCG iterations to relative residual and time-to-PSNR, "
                                 "learned vs Jacobi", **res)), flush=True)


def run_hier(args, rank, world, local):
    """Hierarchical formulation vs a single level: the coarse-to-fine driver
    (--hier-levels levels, by default 3: 32^3 -> 64^3 -> 128^3 with maps
    doubling to the workload's size, --hier-steps Gauss-Newton steps per
    level, random colours with low
    opacity at the first level) against Gauss-Newton at the final resolution
    from the workload's constant start, both with --hier-pcg fixed PCG
    iterations per step; held-out-view PSNR against wall-clock time."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2112_05598_gb300 import Context
    from paper_2112_05598_gb300.hierarchy import coarse_to_fine
    from scenegen import make_scene, random_params
    if rank != 0:
        return
    dev = torch.device("cuda", local)
    sc = make_scene(args.workload, n_cams=args.cams)
    levels = args.hier_levels
    G0, He0, We0 = sc.G >> (levels - 1), sc.env_h >> (levels - 1), sc.env_w >> (levels - 1)
    S = len(sc.radii)
    ctx = Context.from_scene(sc)
    x_gt = torch.from_numpy(sc.x_gt).to(dev)
    target = torch.empty(3 * ctx.n_rays, device=dev)
    ctx.render(x_gt, target)
    ctx.close()
    F = torch.zeros(1, dtype=torch.float64, device=dev)
    holds = {}

    def held_psnr(shape, x):
        G, He, We = shape
        if shape not in holds:
            h = Context(G, sc.radii, He, We, sc.heldout_c2w, sc.heldout_focal, sc.width,
                        sc.height, max_samples=int(np.ceil(np.sqrt(3.0) * G)) + 1)
            hold_gt = Context.from_scene(sc, c2w=sc.heldout_c2w, focal=sc.heldout_focal)
            ht = torch.empty(3 * h.n_rays, device=dev)
            hold_gt.render(x_gt, ht)
            hold_gt.close()
            holds[shape] = (h, ht)
        h, ht = holds[shape]
        h.residual(x, ht, None, F)
        return _psnr_from_F(float(F.item()), h.n_rays)

    def thresholded_psnr(x, cut=0.7):
        """Held-out PSNR of the final state rendered with the converged-scene
        opacity threshold of Section "Rendering"."""
        h, ht = holds[(sc.G, sc.env_h, sc.env_w)]
        rgb = torch.empty(3 * h.n_rays, device=dev)
        h.render_threshold(x, cut, rgb)
        mse = float(torch.mean((rgb - ht) ** 2).item())
        return 10.0 * np.log10(1.0 / mse) if mse > 0 else float("inf")

    opts = dict(pcg_iters=args.hier_pcg, pcg_fixed=1)
    # paper mode: at most --hier-pcg iterations with the relative-residual
    # (1e-3) and stall (0.85) exits, pixel and sample jitter on
    paper_opts = dict(pcg_iters=args.hier_pcg, pcg_fixed=0, pcg_eps_rel=1e-3, pcg_stall=0.85,
                      jitter=1, seed=99)
    runs = {}
    pause = [0.0]
    for name, o in (("hierarchical", opts), ("hierarchical_paper_mode", paper_opts)):
        rng = np.random.default_rng(77)
        x0 = torch.from_numpy(random_params(rng, G0, S, He0, We0, 0.0, 0.1,
                                            shell_sigma_hi=0.1)).to(dev)
        curve, steps = [], []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pause[0] = 0.0

        def on_step(l, k, shape, x, st):
            torch.cuda.synchronize()
            tp = time.perf_counter()
            curve.append((tp - t0 - pause[0], held_psnr(shape, x), l))
            steps.append({"level": l, "G": shape[0], "ms": st["ms"], "F_after": st["F_after"],
                          "gamma": st["gamma"], "pcg_iters": st["pcg_iters"]})
            pause[0] += time.perf_counter() - tp      # held-out evaluation is not solve time
        xf = coarse_to_fine(x0, G0, sc.radii, He0, We0, sc.c2w, sc.focal, sc.width, sc.height,
                            target, levels, args.hier_steps, on_step=on_step, **o)
        runs[name] = {"psnr_curve": curve, "steps": steps,
                      "levels": [[G0 << l, He0 << l, We0 << l] for l in range(levels)],
                      "final_psnr_threshold_0.7_db": thresholded_psnr(xf)}
        del xf
    curve = runs["hierarchical"]["psnr_curve"]
    # single level at the final resolution, for the same wall time or more
    budget = curve[-1][0]
    ctx = Context.from_scene(sc, **opts)
    x = torch.from_numpy(sc.x0.copy()).to(dev)
    curve2, steps2 = [], []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pause[0] = 0.0
    while True:
        st = ctx.gn_solve(x, target, 1)[0]
        torch.cuda.synchronize()
        tp = time.perf_counter()
        curve2.append((tp - t0 - pause[0], held_psnr((sc.G, sc.env_h, sc.env_w), x), levels - 1))
        steps2.append({"level": levels - 1, "G": sc.G, "ms": st["ms"], "F_after": st["F_after"],
                       "gamma": st["gamma"]})
        pause[0] += time.perf_counter() - tp
        if curve2[-1][0] >= budget or len(steps2) >= 4 * levels * args.hier_steps:
            break
    ctx.close()
    runs["single_level"] = {"psnr_curve": curve2, "steps": steps2,
                            "final_psnr_threshold_0.7_db": thresholded_psnr(x)}
    best_single = max(p for _, p, _ in curve2)
    final_h = curve[-1][1]

    def time_to(cv, target_db):
        return next((t for t, p, _ in cv if p >= target_db), None)
    target_db = min(final_h, best_single) - 0.1
    line = {"metric": "held-out PSNR vs wall time, hierarchical vs single level",
            "workload": f"{args.workload}: {sc.G}^3 grid + {S} shells {sc.env_h}x{sc.env_w}, "
                        f"{sc.n_cams} cameras {sc.width}x{sc.height}; levels "
                        f"{[G0 << l for l in range(levels)]}",
            "pcg_iters_per_step": args.hier_pcg, "gn_steps_per_level": args.hier_steps,
            "final_psnr_db": {k: v["psnr_curve"][-1][1] for k, v in runs.items()},
            "target_psnr_db": target_db,
            "time_to_psnr_s": {k: time_to(v["psnr_curve"], target_db) for k, v in runs.items()},
            "runs": runs}
    for h, _ in holds.values():
        h.close()
    print(json.dumps(line), flush=True)


def run_compare(args, rank, world, local):
    """The 32^3 workload (8 cameras 64x64, 2 shells, 5 Gauss-Newton steps x 20
    PCG iterations): (1) Gauss-Newton against Adam on the same objective and
    gradient -- the paper's Fig. 1 contrast -- with Adam's learning rate swept
    and given at least Gauss-Newton's wall time; (2) the environment shells
    as equirectangular maps (32 x 64) against cube maps (16 x 16 per face) of
    the same smooth field.  Held-out-view PSNR against device time."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2112_05598_gb300 import Context
    from scenegen import make_scene
    if rank != 0:
        return
    dev = torch.device("cuda", local)
    F = torch.zeros(1, dtype=torch.float64, device=dev)

    def setup(env):
        sc = make_scene("small32", env=env)
        ctx = Context.from_scene(sc, pcg_iters=sc.cfg.pcg_iters, pcg_fixed=1)
        hold = Context.from_scene(sc, c2w=sc.heldout_c2w, focal=sc.heldout_focal)
        gt = torch.from_numpy(sc.x_gt).to(dev)
        target = torch.empty(3 * ctx.n_rays, device=dev)
        ctx.render(gt, target)
        htarget = torch.empty(3 * hold.n_rays, device=dev)
        hold.render(gt, htarget)
        return sc, ctx, hold, target, htarget

    def psnr(hold, htarget, x):
        hold.residual(x, htarget, None, F)
        return _psnr_from_F(float(F.item()), hold.n_rays)

    def run_gn(env, steps):
        sc, ctx, hold, target, htarget = setup(env)
        x = torch.from_numpy(sc.x0.copy()).to(dev)
        curve, t = [(0.0, psnr(hold, htarget, x))], 0.0
        for _ in range(steps):
            st = ctx.gn_solve(x, target, 1)[0]
            t += st["ms"] / 1000.0
            curve.append((t, psnr(hold, htarget, x)))
        return {"psnr_curve": curve, "params": sc.n_params}

    def run_adam(lr, budget_s, max_steps=4000):
        sc, ctx, hold, target, htarget = setup("equirect")
        x = torch.from_numpy(sc.x0.copy()).to(dev)
        m = torch.zeros_like(x)
        v = torch.zeros_like(x)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        curve, t, k = [(0.0, psnr(hold, htarget, x))], 0.0, 0
        while t < budget_s and k < max_steps:
            e0.record()
            for _ in range(10):
                k += 1
                ctx.adam_step(x, target, m, v, k, lr=lr)
            e1.record()
            torch.cuda.synchronize()
            t += e0.elapsed_time(e1) / 1000.0
            curve.append((t, psnr(hold, htarget, x)))
        return {"lr": lr, "steps": k, "psnr_curve": curve}

    gn_steps = 5
    gn = run_gn("equirect", gn_steps)
    budget = max(2.0 * gn["psnr_curve"][-1][0], 1.0)
    adam = [run_adam(lr, budget) for lr in (0.003, 0.01, 0.03, 0.1)]
    best = max(adam, key=lambda a: a["psnr_curve"][-1][1])
    target_db = min(gn["psnr_curve"][-1][1], best["psnr_curve"][-1][1]) - 0.1

    def time_to(curve, db):
        return next((t for t, p in curve if p >= db), None)
    cube = run_gn("cube", gn_steps)
    target_env = min(gn["psnr_curve"][-1][1], cube["psnr_curve"][-1][1]) - 0.1
    line = {"metric": "held-out PSNR vs device time on the 32^3 workload",
            "gn_vs_adam": {"gn_steps": gn_steps, "pcg_iters_per_step": 20,
                           "adam_budget_s": budget, "target_psnr_db": target_db,
                           "time_to_target_s": {"gauss_newton": time_to(gn["psnr_curve"], target_db),
                                                "adam_best_lr": time_to(best["psnr_curve"], target_db)},
                           "final_psnr_db": {"gauss_newton": gn["psnr_curve"][-1][1],
                                             "adam": {str(a["lr"]): a["psnr_curve"][-1][1]
                                                      for a in adam}},
                           "adam_best_lr": best["lr"], "gauss_newton": gn, "adam": adam},
            "equirect_vs_cube": {"target_psnr_db": target_env,
                                 "time_to_target_s": {
                                     "equirect": time_to(gn["psnr_curve"], target_env),
                                     "cube": time_to(cube["psnr_curve"], target_env)},
                                 "final_psnr_db": {"equirect": gn["psnr_curve"][-1][1],
                                                   "cube": cube["psnr_curve"][-1][1]},
                                 "shell_texels": {"equirect": "2 x 32x64", "cube": "2 x 6x16x16"},
                                 "equirect": gn, "cube": cube}}
    print(json.dumps(line), flush=True)


def run_batch(args, rank, world, local):
    """The many-scenes form: 64 uneven scenes (grids 32^3-96^3, 8-40 cameras at
    128x128, 1-3 shells), every ray march one persistent launch, the PCG loop
    a CUDA graph, tile shape from the autotuner.  One step = one GN step of
    every scene with 20 PCG iterations; value = scene-PCG-iterations/s."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2112_05598_gb300 import Batch
    from paper_2112_05598_gb300._binding import launch_count
    from scenegen import make_batch
    scenes = make_batch()
    dev = torch.device("cuda", local)
    b = Batch(scenes, max_samples=192, pcg_iters=BATCH_PCG, pcg_fixed=1)
    x_gt = torch.from_numpy(np.concatenate([s["x_gt"] for s in scenes])).to(dev)
    target = torch.empty(3 * b.n_rays, device=dev)
    b.render(x_gt, target)
    x = torch.from_numpy(np.concatenate([s["x0"] for s in scenes])).to(dev)
    tuning = b.autotune(x)
    if args.brick:
        b.set_brick(args.brick)
        tuning = dict(tuning, brick=args.brick, brick_fixed=True)
    for _ in range(args.warmup):
        b.gn_solve(x, target, 1)
    stream = torch.cuda.current_stream()
    clocks = Clocks(local)
    barrier(world)
    torch.cuda.synchronize()
    l0 = launch_count()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    stats = []
    for _ in range(args.steps):
        stats.extend(b.gn_solve(x, target, 1))
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), world)
    iters = sum_over_ranks(float(sum(s["pcg_iters"] for st in stats for s in st)), world)
    value = iters / (ms / 1000.0)
    # end to end with host buffers
    x_host = x.detach().cpu().pin_memory()      # continue from the timed steps' state
    t_host = target.cpu().pin_memory()
    x_dev = torch.empty_like(x)
    t_dev = torch.empty_like(target)
    e2e_steps = args.e2e_steps or args.steps
    torch.cuda.synchronize()
    e0.record(stream)
    it2 = 0
    for _ in range(e2e_steps):
        x_dev.copy_(x_host, non_blocking=True)
        t_dev.copy_(t_host, non_blocking=True)
        st = b.gn_solve(x_dev, t_dev, 1)
        x_host.copy_(x_dev, non_blocking=True)
        it2 += sum(s["pcg_iters"] for s in st[0])
    e1.record(stream)
    torch.cuda.synchronize()
    ms2 = max_over_ranks(e0.elapsed_time(e1), world)
    if rank != 0:
        return
    Gs = [s["G"] for s in scenes]
    line = {"metric": METRIC + " (scene-iterations, batched)", "value": value,
            "unit": "PCG iters/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (64 seeded voxelised scenes)",
            "config": {"workload": f"batch64: {len(scenes)} scenes, grids {min(Gs)}^3-{max(Gs)}^3, "
                                   f"8-40 cameras 128x128, 1-3 shells Gx2G, {BATCH_PCG} PCG/GN step",
                       "n_params": b.n_params, "n_rays": b.n_rays, "tuning": tuning},
            "gpu_launches": int(launch_count() - l0),
            "e2e": {"value": it2 / (ms2 / 1000.0), "unit": "PCG iters/s",
                    "h2d_bytes_per_step": int(4 * (b.n_params + 3 * b.n_rays)),
                    "d2h_bytes_per_step": int(4 * b.n_params)},
            "clocks": clk,
            "accepted_fraction": float(np.mean([s["accepted"] for st in stats for s in st]))}
    print(json.dumps(line), flush=True)


def rows_read_fraction(ctx):
    """The share of the store's grid-sample rows the last Gauss-Newton step's
    A p read (perf_coef_prefix); None without a filled store."""
    from paper_2112_05598_gb300 import PerfError
    try:
        pre = ctx.coef_prefix()
    except PerfError:
        return None
    return pre["read"] / pre["total"] if pre["total"] else None


def count_lane_ops(ctx, x, target, pcg_iters):
    """Vector-atomic lane operations per A p of the Jacobian-transpose
    scatter, counted (perf_set_atomic_counter, the counting instantiation of
    the A p kernels) on one Gauss-Newton step of 2 PCG iterations from a
    copy of x.  Blocks whose contribution is exactly zero are not issued, so
    the count depends on the state."""
    import torch
    cnt = torch.zeros(1, dtype=torch.int64, device=x.device)
    ctx.set_atomic_counter(cnt)
    ctx.set_options(pcg_iters=2)
    st = ctx.gn_solve(x.clone(), target, 1)
    ctx.set_atomic_counter(None)
    ctx.set_options(pcg_iters=pcg_iters)
    return float(cnt.item()) / max(sum(s["pcg_iters"] for s in st), 1)


def run_ours(args, rank, world, local):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2112_05598_gb300 import Context
    from paper_2112_05598_gb300._binding import launch_count
    from scenegen import make_scene

    from paper_2112_05598_gb300 import PERF_BF16, PERF_F32
    sc = make_scene(_scene_config(args), n_cams=args.cams)
    cfg = sc.cfg
    dev = torch.device("cuda", local)
    bf = args.dtype == "bf16"
    sdt = torch.bfloat16 if bf else torch.float32
    ctx = Context.from_scene(sc, dtype=PERF_BF16 if bf else PERF_F32, pcg_iters=cfg.pcg_iters,
                             pcg_fixed=1)
    if args.coef_budget != -1:
        ctx.set_coef_budget(args.coef_budget)
    stream = torch.cuda.current_stream()
    x_gt = torch.from_numpy(sc.x_gt).to(dev).to(sdt)
    target = torch.empty(3 * ctx.n_rays, device=dev)
    ctx.render(x_gt, target)
    target = target.to(sdt)
    del x_gt
    samples = ctx.sample_count()
    x = torch.from_numpy(sc.x0.copy()).to(dev)

    for _ in range(args.warmup):
        ctx.gn_solve(x, target, 1)
    # (before the tuner, which rebuilds the shell hits that changing the
    # options invalidates)
    red_before = count_lane_ops(ctx, x, target, cfg.pcg_iters)
    prefix_before = rows_read_fraction(ctx)
    # tile shape / CTA cap tuned at the warmed-up state along a random direction
    gp = torch.Generator(device=dev).manual_seed(0)
    probe = torch.randn(sc.n_params, device=dev, generator=gp).to(sdt)
    tuning = ctx.autotune(x.to(sdt) if bf else x, probe)
    if args.brick:
        ctx.set_brick(args.brick)
        tuning = dict(tuning, brick=args.brick, brick_fixed=True)
    del probe
    # the end-to-end steps below repeat the timed steps from the same state
    # (a step's A p gets cheaper as more rays turn opaque and their zero row
    # tails are skipped)
    x_host = x.detach().to(dtype=torch.float32).cpu().pin_memory()
    torch.cuda.synchronize()
    ctx.enable_timing(True)
    ctx.timing(reset=True)
    clocks = Clocks(local)
    barrier(world)
    torch.cuda.synchronize()
    l0 = launch_count()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    stats = []
    for _ in range(args.steps):
        stats.extend(ctx.gn_solve(x, target, 1))
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    launches = launch_count() - l0
    ms = e0.elapsed_time(e1)
    ms = max_over_ranks(ms, world)
    pcg_total = sum_over_ranks(float(sum(s["pcg_iters"] for s in stats)), world)
    value = pcg_total / (ms / 1000.0)
    tm = ctx.timing(reset=True)
    ctx.enable_timing(False)
    coef_timed = ctx.coef_info()
    # grid-sample rows the A p reads from the store (each ray's non-zero
    # prefix) over the store's grid samples, before and after the timed steps
    prefix_after = rows_read_fraction(ctx)
    rows_read = ([prefix_before, prefix_after] if prefix_before is not None
                 and prefix_after is not None else None)

    # end to end through the public API with host buffers
    e2e_steps = args.e2e_steps or args.steps
    # from the state the timed steps started in (x_host), so that both numbers
    # measure the same Gauss-Newton steps; each step's x goes back to x_host
    t_host = target.cpu().pin_memory()
    x_dev = torch.empty_like(x)
    t_dev = torch.empty_like(target)
    barrier(world)
    torch.cuda.synchronize()
    e0.record(stream)
    e2e_pcg = 0
    for _ in range(e2e_steps):
        x_dev.copy_(x_host, non_blocking=True)
        t_dev.copy_(t_host, non_blocking=True)
        st = ctx.gn_solve(x_dev, t_dev, 1)
        x_host.copy_(x_dev, non_blocking=True)
        e2e_pcg += sum(s["pcg_iters"] for s in st)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    ms_e2e = max_over_ranks(e0.elapsed_time(e1), world)
    e2e_value = sum_over_ranks(float(e2e_pcg), world) / (ms_e2e / 1000.0)

    # the scatter's vector-atomic lane operations per A p: the mean of two
    # counts, one from the state before the timed steps and one from the
    # state they end in
    from paper_2112_05598_gb300 import measure_atomic_peak
    red_after = count_lane_ops(ctx, x, target, cfg.pcg_iters)
    red_per_apply = 0.5 * (red_before + red_after)
    red_peak = measure_atomic_peak()

    peaks, peak_src = measured_peaks()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = sm_count * 128 * 2 * sm_mhz * 1e6 / 1e12
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    apply_ms = tm["apply"]["ms"] / max(tm["apply"]["launches"], 1)
    per_step = {k: v["ms"] / args.steps for k, v in tm.items()}
    iters = max(sum(s["pcg_iters"] for s in stats), 1)
    # the store's coverage in the timed steps (a fraction of the pixel tiles;
    # the rest of each A p recomputes)
    cov = coef_timed["coverage"] if coef_timed["used"] else 0.0
    coef = cov >= 1.0
    coef_kernel = ("k_apply_coef<bf16> (A p from stored coefficients)" if bf else
                   "k_apply_coef<float> (A p from stored coefficients)")
    rec_kernel = ("k_scatter<bf16,bf16,1> (A p)" if bf else
                  "k_scatter<PairF32,PairF32,1> (A p, paired x/p records)"
                  if tuning.get("paired") else "k_scatter<float,float,1> (A p)")
    if coef:
        apply_kernel = coef_kernel
    elif cov > 0.0:
        apply_kernel = f"{coef_kernel} on {cov:.3f} of the pixel tiles + {rec_kernel} on the rest"
    else:
        apply_kernel = rec_kernel
    # per PCG iteration (a partial coefficient store splits one A p in two launches)
    apply_s = tm["apply"]["ms"] / 1000.0 / iters
    achieved = FLOP_PER_SAMPLE_METHOD * samples / apply_s / 1e12
    # (a partial store: weighted by the tiles each kernel runs)
    impl_flop = cov * FLOP_PER_SAMPLE_COEF + (1.0 - cov) * FLOP_PER_SAMPLE_RECOMPUTE
    # the mean share of the store's rows its A p reads (each ray's non-zero
    # prefix; 1 without a store): the samples the kernels actually visit
    rf = 0.5 * sum(rows_read) if rows_read else 1.0
    visited = samples * (cov * rf + (1.0 - cov))
    compulsory = APPLY_COMPULSORY_BYTES_PER_PARAM * sc.n_params
    roof = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
            "frac": achieved / fp32_peak,
            "flop_per_sample": FLOP_PER_SAMPLE_METHOD, "samples_per_launch": samples,
            "peak_source": f"{sm_count} SMs x 128 FP32 lanes x 2 FLOP x {sm_mhz:.0f} MHz "
                           f"(max SM clock, {peak_src})",
            "kernel": apply_kernel,
            "traffic": recorded_traffic(apply_kernel, args.workload, samples, rf)
            if args.cams is None and args.grid is None else None,
            "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of a 4-camera "
                              "capture, scaled by the store rows streamed: samples x the mean "
                              "of the rows-read fractions before and after the timed steps "
                              "(profiles/apply_coef_traffic_scale128.md)",
            "impl_flop_per_sample": impl_flop,
            "samples_visited_per_launch": visited,
            "impl_alu_frac": impl_flop * visited / apply_s / 1e12 / fp32_peak,
            "compulsory_bytes_per_launch": compulsory,
            "hbm_frac_compulsory": compulsory / apply_s / 1e9 / hbm_peak}
    if coef:
        design = int(COEF_BYTES_PER_SAMPLE * samples * rf) + ((2 if bf else 4) + 4) * sc.n_params
        roof["design_traffic"] = {
            "what": "coefficient store: 16 B per sample or shell hit streamed twice per A p "
                    "(the rows each ray's non-zero prefix holds: samples x the mean rows-read "
                    "fraction), plus p read and A p written once (an implementation choice "
                    "that trades HBM capacity for recomputation, not the method's compulsory "
                    "bytes)",
            "bytes_per_launch": design, "ratio_to_compulsory": design / compulsory,
            "achieved": design / apply_s / 1e9, "unit": "GB/s",
            "hbm_frac": design / apply_s / 1e9 / hbm_peak}
    # the scope's labelled "effective gather bandwidth": per sample the 8
    # corner blocks of p gathered by J p and the 8 corner contributions the
    # J^T sweep scatters (before the window merges them), over the launch
    # time -- served by L1 and L2, not HBM
    pb = 8 if bf else 16
    eff = (8 * pb + 8 * 16) * samples
    roof["effective_gather"] = {"what": "algorithmic gather + scatter bytes (8 corners of p "
                                        "and 8 corner contributions of A p per sample), served "
                                        "by L1/L2: not HBM traffic",
                                "bytes_per_launch": eff, "achieved": eff / apply_s / 1e9,
                                "unit": "GB/s"}
    # the scatter's 16-byte vector atomics, one lane operation per active lane
    red_rate = red_per_apply / apply_s
    roof["atomics"] = {"lane_ops_per_apply": red_per_apply,
                       "lane_ops_before_after": [red_before, red_after],
                       "count_source": "mean of two counts on an extra Gauss-Newton step (2 PCG "
                                       "iterations), from the states before and after the timed "
                                       "steps; blocks whose contribution is exactly zero are not "
                                       "issued, so the count falls as the reconstruction "
                                       "proceeds",
                       "achieved": red_rate,
                       "peak": red_peak, "unit": "lane-ops/s", "frac": red_rate / red_peak,
                       "peak_source": "perf_measure_atomic_peak (16-byte vector atomic "
                                      "microbenchmark on this GPU, measured in this run)"}
    vb = VEC_BYTES_PER_PARAM + (2 if bf else 0) + (4 if (not bf and not coef and tuning.get("paired")) else 0)
    vec_s = tm["vector"]["ms"] / 1000.0 / iters
    vector_roof = {"kernels": "k_pcg_update + k_pcg_finish + k_pcg_dir (per PCG iteration)",
                   "bound": "hbm", "bytes_per_iter": vb * sc.n_params,
                   "ms_per_iter": vec_s * 1000.0,
                   "achieved": vb * sc.n_params / vec_s / 1e9, "peak": hbm_peak, "unit": "GB/s",
                   "frac": vb * sc.n_params / vec_s / 1e9 / hbm_peak,
                   "compulsory_bytes_per_iter": VEC_COMPULSORY_BYTES_PER_PARAM * sc.n_params,
                   "frac_compulsory": VEC_COMPULSORY_BYTES_PER_PARAM * sc.n_params / vec_s / 1e9
                   / hbm_peak,
                   "peak_source": f"hbm_gbs ({peak_src})"}
    rb = (RESIDUAL_BYTES_PER_RAY_F32 // (2 if bf else 1)) * sc.n_rays
    res_s = tm["residual"]["ms"] / 1000.0 / max(tm["residual"]["launches"], 1)
    residual_roof = {"kernel": "k_forward<MODE 1> (residual r = H^ - C and F: one ray march)",
                     "bound": "hbm", "bytes_per_launch": rb, "ms_per_launch": res_s * 1000.0,
                     "achieved": rb / res_s / 1e9, "peak": hbm_peak, "unit": "GB/s",
                     "frac": rb / res_s / 1e9 / hbm_peak,
                     "note": "streams C in and r out, but each ray's march (interpolation of x "
                             "from L2, exponentials) bounds the launch",
                     "peak_source": f"hbm_gbs ({peak_src})"}

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16" if bf else "f32",
        "data": "synthetic (seeded voxelised primitives, targets rendered from ground truth)",
        "config": {"workload": _workload_desc(sc) + (" (BF16 storage form)" if bf else ""),
                   "n_params": sc.n_params, "n_rays": sc.n_rays,
                   "samples_per_march": samples, "tuning": tuning,
                   "coef_store_bytes": coef_timed["bytes"],
                   "coef_coverage": cov,
                   "coef_rows_read_before_after": rows_read,
                   "l2": "inputs larger than L2: targets and residuals 768 MB each per step"},
        "gpu_launches": int(launches),
        "rays_per_s": 2.0 * sc.n_rays * pcg_total / (ms / 1000.0),
        "gn_steps": [{k: s[k] for k in ("F_before", "F_after", "gamma", "ls_evals", "pcg_iters")}
                     for s in stats],
        "kernel_ms_per_step": per_step,
        "apply_ms_per_launch": apply_ms,
        "roofline": roof,
        "vector_roofline": vector_roof,
        "residual_roofline": residual_roof,
        "e2e": {"value": e2e_value, "unit": METRIC,
                "h2d_bytes_per_step": int(4 * sc.n_params + (2 if bf else 4) * 3 * sc.n_rays),
                "d2h_bytes_per_step": int(4 * sc.n_params)},
        "clocks": clk,
    }
    if not args.no_cpu_baseline and world == 1 and args.cams is None:
        line["cpu_baseline"] = cpu_baseline(sc, args.cpu_cams, cfg.pcg_iters)
    if (not args.no_lpc_record and world == 1 and args.cams is None and args.workload == WORKLOAD
            and args.grid is None and not bf):
        # the time-to-PSNR half of the metric: learned vs Jacobi on the reduced
        # ring workload (outside every timed region above)
        del ctx, target, x, x_host, t_host, x_dev, t_dev
        torch.cuda.empty_cache()
        line["lpc"] = lpc_study(dev, "ring128", train_small=100, train_steps=20, train_large=8,
                                gn_steps=40, pcg_per_step=2, traj_iters=1200, train_pcg=2)
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_setup(args.gpus)
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.conv:
        run_conv(args, rank, world, local)
    elif args.compare:
        run_compare(args, rank, world, local)
    elif args.lpc:
        run_lpc(args, rank, world, local)
    elif args.hier:
        run_hier(args, rank, world, local)
    elif args.workload == "batch64":
        run_batch(args, rank, world, local)
    else:
        run_ours(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

"""Coarse-to-fine driver of PERF's hierarchical formulation (Section
"Hierarchical formulation").

A fixed number of Gauss-Newton steps runs on each level; the next level
doubles the resolution of the voxel grid and of the environment maps and is
filled from this level's result by linear interpolation (``perf_upsample``:
grid opacity is per voxel side, so it is halved), and the solve resumes.
The targets and cameras are the same on every level.  This module is host
orchestration only -- contexts, the loop and the level change are libperf
calls; every step runs in its kernels.
"""
from __future__ import annotations

import math
from typing import Callable, List, Optional, Tuple

from ._binding import Context, upsample


def level_shapes(G0: int, env_h0: int, env_w0: int, levels: int) -> List[Tuple[int, int, int]]:
    """(G, env_h, env_w) of every level: each doubles the previous one."""
    return [(G0 << l, env_h0 << l, env_w0 << l) for l in range(levels)]


def coarse_to_fine(x0, G0: int, radii, env_h0: int, env_w0: int, c2w, focal, width: int,
                   height: int, target, levels: int, gn_per_level: int,
                   on_step: Optional[Callable] = None, env_kind: int = 0, **opts):
    """Runs the hierarchy from x0 (device tensor, level-0 parameters) and
    returns the final level's parameters.  on_step(level, step, (G, env_h,
    env_w), x, stats) is called after every Gauss-Newton step.  opts are
    Context options (pcg_iters, pcg_fixed, ...); the per-ray sample cap is
    raised where needed so that it never binds (K <= ceil(sqrt(3) G)).
    env_kind 1: the shells are cube maps (env_w0 = 6 env_h0)."""
    import torch
    S = len(radii)
    x = x0
    shapes = level_shapes(G0, env_h0, env_w0, levels)
    for l, (G, He, We) in enumerate(shapes):
        kw = dict(opts)
        kw["max_samples"] = max(int(kw.get("max_samples", 0)), math.ceil(math.sqrt(3.0) * G) + 1)
        ctx = Context(G, radii, He, We, c2w, focal, width, height, env_kind=env_kind, **kw)
        try:
            for k in range(gn_per_level):
                st = ctx.gn_solve(x, target, 1)[0]
                if on_step is not None:
                    on_step(l, k, (G, He, We), x, st)
        finally:
            ctx.close()
        if l + 1 < levels:
            y = torch.empty(4 * (8 * G ** 3 + 4 * S * He * We), dtype=x.dtype, device=x.device)
            upsample(x, G, S, He, We, y, env_kind=env_kind)
            x = y
    return x

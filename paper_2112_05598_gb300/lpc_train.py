"""Training pipeline of the learned block preconditioner.

Logs Gauss-Newton systems from the solver's own runs (features of each step's
x, J^T r, diag(J^T J) and block couplings, plus probe pairs
xi / a_hat = D^{-1/2} A D^{-1/2} xi computed with the library's A p), trains
the network with the library's BF16 kernels, and measures PCG iterations to a
relative residual.  This module only sequences library calls; every
arithmetic step runs in libperf's kernels (random probe vectors are drawn by
torch and passed in as inputs).
"""
from __future__ import annotations

import dataclasses
from typing import List

import numpy as np

from ._binding import LPC, Context, dscale


@dataclasses.dataclass
class System:
    G: int
    feat: object       # G^3 x 16 bf16 (torch)
    ahat: list         # probe pairs: D^{-1/2} A D^{-1/2} xi (G^3 x 4 float, torch)
    xi: list
    mask: object       # G^3 uint8


def log_system(ctx: Context, lpc: LPC, x, target, n_probes: int = 2, generator=None) -> System:
    """One logged system at parameters x (device float tensor)."""
    import torch
    G = ctx.G
    V = G ** 3
    n = ctx.n_params
    dev = x.device
    r = torch.empty(3 * ctx.n_rays, device=dev)
    F = torch.zeros(1, dtype=torch.float64, device=dev)
    ctx.residual(x, target, r, F)
    diag = torch.empty(n, device=dev)
    grad = torch.empty(n, device=dev)
    ctx.diag_jtj(x, diag, r, grad)
    d2 = torch.empty(n, device=dev)
    cross = torch.empty(4 * V, device=dev)
    ctx.diag_cross(x, d2, cross)
    feat = torch.empty(16 * V, dtype=torch.bfloat16, device=dev)
    lpc.features(G, x, grad, diag, cross, feat)
    mask = torch.empty(V, dtype=torch.uint8, device=dev)
    xis, ahats = [], []
    for _ in range(n_probes):
        xi = torch.randn(4 * V, device=dev, generator=generator)
        w = torch.zeros(n, device=dev)
        dscale(G, diag, xi, w, mask)        # w = D^{-1/2} xi on observed voxels
        xi_m = torch.where(mask.repeat_interleave(4).bool(), xi, torch.zeros_like(xi))
        Aw = torch.empty(n, device=dev)
        ctx.apply_normal(x, w, Aw)
        ahat = torch.empty(4 * V, device=dev)
        dscale(G, diag, Aw, ahat)           # a_hat = D^{-1/2} A w
        xis.append(xi_m)
        ahats.append(ahat)
    return System(G=G, feat=feat, ahat=ahats, xi=xis, mask=mask)


def train(lpc: LPC, systems: List[System], epochs: int = 3, lr: float = 1e-3, seed: int = 0):
    """Adam over (system, probe) pairs in shuffled order; returns the losses."""
    rng = np.random.default_rng(seed)
    pairs = [(i, k) for i, s in enumerate(systems) for k in range(len(s.xi))]
    losses = []
    for _ in range(epochs):
        for j in rng.permutation(len(pairs)):
            i, k = pairs[j]
            s = systems[i]
            losses.append(lpc.train_step(s.G, s.feat, s.ahat[k], s.xi[k], s.mask, lr))
    return losses


def mean_loss(lpc: LPC, systems: List[System]) -> float:
    vals = [lpc.loss_grad(s.G, s.feat, s.ahat[k], s.xi[k], s.mask)
            for s in systems for k in range(len(s.xi))]
    return float(np.mean(vals))


def pcg_iterations(ctx: Context, x, target, precond: int, eps: float = 1e-3,
                   max_iter: int = 200, lpc: LPC = None, thresholds=(1e-1, 1e-2, 1e-3)) -> dict:
    """One GN step's PCG at x (the solver's own path, coefficient store
    included) until |r_k| / |r_0| < eps or max_iter (paper mode without the
    stall exit); x is not modified.  Returns the iterations, the relative
    residual after each iteration and the first iteration below each
    threshold (None: not reached)."""
    ctx.set_options(pcg_iters=max_iter, pcg_fixed=0, pcg_eps_rel=eps, pcg_stall=1e30,
                    precond=precond)
    if lpc is not None:
        ctx.set_lpc(lpc)
    xx = x.clone()
    st = ctx.gn_solve(xx, target, 1)[0]
    R = ctx.pcg_history(max_iter)
    rel = np.sqrt(R / st["R0"]) if st["R0"] > 0 else np.zeros_like(R)
    first = {f"{t:g}": next((k + 1 for k, v in enumerate(rel) if v < t), None) for t in thresholds}
    return dict(iters=st["pcg_iters"], exit=st["pcg_exit"], R=st["R"], R0=st["R0"],
                fallback=st["precond_fallback"], ms=st["ms"], F_after=st["F_after"],
                rel_residual=rel.tolist(), iters_to=first)

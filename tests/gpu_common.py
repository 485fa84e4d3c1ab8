"""Shared helpers of the GPU parity tests (CUDA path vs the FP64 oracle)."""
import numpy as np

from conftest import rel_l2
from oracle import Oracle

# Tolerances: relative L2 for FP32 r, J p, J^T v (and the renders and the
# Jacobi diagonal computed from the same partials), and for the parameters
# after each Gauss-Newton step.
TOL_FP32 = 1e-5
TOL_GN = 1e-4
# Element-wise bound beside the relative L2:
#   |a_i - b_i| <= EW_REL mag_i + EW_ABS max_j mag_j,
# mag_i the sum of the absolute values of the terms entry i is made of (the
# oracle returns it for J p and J^T v; a render's terms are all positive, so
# there mag = |b|; a residual's are |H^| and |C|).  FP32 rounding scales with
# that sum, not with the entry, which can be a small difference of large
# terms (J p and J^T v along random directions, the opacity entries).  The
# absolute part (one millionth of the largest magnitude) covers entries
# whose terms are all tiny.
EW_REL = 1e-5
EW_ABS = 1e-6


def assert_elementwise(a, b, mag=None, rel=EW_REL, abs_frac=EW_ABS, what=""):
    """Every element of a within rel mag + abs_frac max(mag) of b (mag
    defaults to |b|); prints the worst ratio of error to bound, so a log shows
    the margin."""
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    m = np.abs(b) if mag is None else np.abs(np.asarray(mag, np.float64).ravel())
    assert a.shape == b.shape == m.shape, (what, a.shape, b.shape, m.shape)
    if b.size == 0:
        return
    bound = rel * m + abs_frac * float(m.max())
    ratio = np.abs(a - b) / np.where(bound > 0, bound, 1.0)
    ratio[(bound == 0) & (a == b)] = 0.0
    ratio[(bound == 0) & (a != b)] = np.inf
    i = int(np.argmax(ratio))
    print(f"[elementwise] {what}: worst |a-b|/bound = {ratio[i]:.3g} at {i} "
          f"(a={a[i]:.9g}, b={b[i]:.9g}, mag={m[i]:.3g}, n={b.size})")
    assert ratio[i] <= 1.0, (what, i, a[i], b[i], m[i], ratio[i])


# Parameters seen only through interpolation weights of order 1e-5 have
# Jacobi diagonals below ~1e-10 of the largest, and the Jacobi-scaled step
# gives them |Delta| ~ 1e5: on the 128^3 workload from the constant start,
# 35 of 2.2 M observed blocks carry 99.7 % of |Delta|^2.  Their rows of J
# must therefore agree to FP32 rounding, which is why the shells' texel
# coordinates are FP64 (a binary32 coordinate of a 1024-texel map resolves
# only ~6e-5 of a texel) and the grid's sample coordinates are binary32 on
# both sides.  The bar applies to all parameters; the split by observability
# is printed to show where the difference sits.
WEAK_DIAG = 1e-10


def assert_params(xg, xo, diag, tol=1e-4, what="x", weak=WEAK_DIAG):
    """x after a Gauss-Newton step: relative L2 below tol over all parameters,
    every value finite and inside the projection's bounds."""
    xg = np.asarray(xg, np.float64).reshape(-1, 4)
    xo = np.asarray(xo, np.float64).reshape(-1, 4)
    blk = np.asarray(diag, np.float64).reshape(-1, 4).max(1)
    w = (blk > 0) & (blk <= weak * blk.max())
    err = rel_l2(xg, xo)
    print(f"[params] {what}: rel L2 {err:.3e} (over the {int((~w).sum())} blocks with diagonal "
          f"above {weak:g} x max: {rel_l2(xg[~w], xo[~w]):.3e}; {int(w.sum())} below)")
    assert err < tol, (what, err)
    assert np.all(np.isfinite(xg))
    assert np.all(xg[:, :3] >= 0) and np.all(xg[:, :3] <= 1) and np.all(xg[:, 3] >= 0)


def cuda_tensor(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def empty(n, dtype=None):
    import torch
    return torch.zeros(int(n), dtype=dtype or torch.float32, device="cuda")


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def make_pair(G, radii, env_h, env_w, c2w, focal, width, height, max_samples=64,
              dtype=0, jitter=False, seed=0, epoch=0, env_kind=0, **opt):
    """(GPU context, oracle) on the same scene and cameras."""
    from paper_2112_05598_gb300 import Context
    ctx = Context(G, radii, env_h, env_w, c2w, focal, width, height, dtype=dtype,
                  max_samples=max_samples, jitter=int(jitter), seed=seed, epoch=epoch,
                  env_kind=env_kind, **opt)
    orc = Oracle(G, radii, env_h, env_w, c2w, focal, width, height,
                 max_samples=max_samples, jitter=jitter, seed=seed, epoch=epoch, env_kind=env_kind)
    return ctx, orc


def pair_from_scene(scene, **kw):
    kw.setdefault("max_samples", scene.cfg.max_samples)
    kw.setdefault("env_kind", getattr(scene, "env_kind", 0))
    return make_pair(scene.G, scene.radii, scene.env_h, scene.env_w, scene.c2w, scene.focal,
                     scene.width, scene.height, **kw)


def mid_state(rng, scene, spread=0.5):
    """A state between the start and the ground truth, with noise: exercises
    every derivative term (partial opacity everywhere)."""
    x = (0.5 * scene.x0 + 0.5 * scene.x_gt).reshape(-1, 4).astype(np.float64)
    x += spread * rng.uniform(-0.1, 0.1, size=x.shape)
    x[:, 0:3] = np.clip(x[:, 0:3], 0, 1)
    x[:, 3] = np.clip(x[:, 3], 0, None)
    return x.reshape(-1).astype(np.float32)

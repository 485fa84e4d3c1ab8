"""Shared helpers of the GPU parity tests (CUDA path vs the FP64 oracle)."""
import numpy as np

from oracle import Oracle

# Tolerances: relative L2 for FP32 r, J p, J^T v (and the renders and the
# Jacobi diagonal computed from the same partials), and for the parameters
# after each Gauss-Newton step.
TOL_FP32 = 1e-5
TOL_GN = 1e-4
# Element-wise bound beside the relative L2: |a - b| <= EW_REL |b| + EW_ABS max|b|.
# The relative part is the FP32 bar; the absolute part (one millionth of the
# largest entry) covers entries that are sums of terms of both signs (J^T v,
# the opacity entries of A p), whose own size says nothing about the rounding
# of the terms they cancel from.
EW_REL = 1e-5
EW_ABS = 1e-6


def assert_elementwise(a, b, rel=EW_REL, abs_frac=EW_ABS, what=""):
    """Every element of a within rel |b| + abs_frac max|b| of b; prints the
    worst ratio of error to bound, so a log shows the margin."""
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    assert a.shape == b.shape, (what, a.shape, b.shape)
    if b.size == 0:
        return
    bound = rel * np.abs(b) + abs_frac * float(np.abs(b).max())
    ratio = np.abs(a - b) / np.where(bound > 0, bound, 1.0)
    ratio[(bound == 0) & (a == b)] = 0.0
    ratio[(bound == 0) & (a != b)] = np.inf
    i = int(np.argmax(ratio))
    print(f"[elementwise] {what}: worst |a-b|/bound = {ratio[i]:.3g} at {i} "
          f"(a={a[i]:.9g}, b={b[i]:.9g}, n={b.size})")
    assert ratio[i] <= 1.0, (what, i, a[i], b[i], ratio[i])


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
              dtype=0, jitter=False, seed=0, epoch=0, **opt):
    """(GPU context, oracle) on the same scene and cameras."""
    from paper_2112_05598_gb300 import Context
    ctx = Context(G, radii, env_h, env_w, c2w, focal, width, height, dtype=dtype,
                  max_samples=max_samples, jitter=int(jitter), seed=seed, epoch=epoch, **opt)
    orc = Oracle(G, radii, env_h, env_w, c2w, focal, width, height,
                 max_samples=max_samples, jitter=jitter, seed=seed, epoch=epoch)
    return ctx, orc


def pair_from_scene(scene, **kw):
    kw.setdefault("max_samples", scene.cfg.max_samples)
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

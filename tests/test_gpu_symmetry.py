"""J p and J^T v apply one matrix and its transpose, also where Algorithm 1's
partials are small differences of nearly equal terms: behind optically deep
media in front of an opaque background shell, along directions rescaled by
the Jacobi preconditioner (1 / sqrt(diag(J^T J)), which blows up barely
observed parameters by many orders of magnitude).  CG on the preconditioned
normal equations (Algorithm 2) needs the operator symmetric there."""
import numpy as np
import pytest

from gpu_common import empty

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def deep():
    """The 256^3 ring workload's structure at 64^3 and 6 cameras: four
    shells, the outermost opaque (sigma 10), and a grid of opacity 0.9 per
    voxel side (optical depth up to ~100 through the volume)."""
    import torch
    from paper_2112_05598_gb300 import Context
    from scenegen import make_scene
    sc = make_scene("ring256", G=64, n_cams=6)
    ctx = Context.from_scene(sc)
    x = sc.x0.reshape(-1, 4).copy()
    g = sc.G ** 3
    x[:g, 3] = 0.9
    x = torch.from_numpy(x.reshape(-1)).cuda()
    d = empty(ctx.n_params)
    ctx.diag_jtj(x, d)
    torch.cuda.synchronize()
    return dict(sc=sc, ctx=ctx, x=x, d=d)


def _scaled(rng, d, floor):
    """A random direction scaled by the Jacobi preconditioner over the
    parameters whose diagonal exceeds floor (zero elsewhere)."""
    import torch
    dd = d.double()
    inv = torch.where(dd > floor, 1.0 / dd.clamp_min(1e-300).sqrt(), torch.zeros_like(dd))
    z = torch.from_numpy(rng.normal(size=d.numel())).cuda()
    return (z * inv).float()


@pytest.mark.parametrize("floor", [0.0, 1e-19, 1e-12])
def test_adjoint_identity_jacobi_scaled(deep, floor):
    import torch
    ctx, x, d = deep["ctx"], deep["x"], deep["d"]
    rng = np.random.default_rng(7)
    assert float(d.min()) < 1e-12 * float(d.max())   # the scene has barely observed parameters
    p = _scaled(rng, d, floor)
    v = torch.from_numpy(rng.normal(size=3 * ctx.n_rays).astype(np.float32)).cuda()
    jp = empty(3 * ctx.n_rays)
    jtv = empty(ctx.n_params)
    ctx.jvp(x, p, jp)
    ctx.vjp(x, v, jtv)
    a = float((jp.double() * v.double()).sum())
    b = float((p.double() * jtv.double()).sum())
    # v is random, so |a| is about the root-sum-square of the per-residual
    # products; a forward tangent sweep missed this by ~10% on such scenes
    rss = float((jp.double() * v.double()).square().sum().sqrt())
    assert abs(a - b) <= 1e-3 * rss, (a, b, rss)


def test_fused_normal_operator_symmetric(deep):
    """u.(A w) = w.(A u) for the recomputing fused A p on Jacobi-scaled u, w."""
    import torch
    ctx, x, d = deep["ctx"], deep["x"], deep["d"]
    rng = np.random.default_rng(8)
    u = _scaled(rng, d, 0.0)
    w = _scaled(rng, d, 0.0)
    au, aw = empty(ctx.n_params), empty(ctx.n_params)
    pap = torch.zeros(1, dtype=torch.float64, device="cuda")
    ctx.apply_normal(x, u, au, pap)
    ctx.apply_normal(x, w, aw, pap)
    a = float((u.double() * aw.double()).sum())
    b = float((w.double() * au.double()).sum())
    rss = float((u.double() * aw.double()).square().sum().sqrt())
    assert abs(a - b) <= 1e-3 * rss, (a, b, rss)

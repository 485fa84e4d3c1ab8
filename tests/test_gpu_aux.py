"""Auxiliary opacity residual (Section "Auxiliary terms") on the GPU against
the FP64 oracle with the same term: 4 residuals per ray, J p, J^T v, the
exact diagonal with its auxiliary row, A p, and Gauss-Newton steps from the
coefficient store and recomputed."""
import numpy as np
import pytest

from conftest import rel_l2
from gpu_common import TOL_FP32, TOL_GN, cuda_tensor, empty, host, mid_state, pair_from_scene

pytestmark = pytest.mark.gpu

LAM = 0.1


@pytest.fixture(scope="module")
def aux():
    from scenegen import make_scene
    sc = make_scene("small32")
    ctx, orc = pair_from_scene(sc, aux=1, aux_lambda=LAM)
    from oracle import Oracle
    orc = Oracle.from_scene(sc, aux=True, aux_lambda=LAM)
    target = orc.render(sc.x_gt)[0].astype(np.float32).ravel()
    rng = np.random.default_rng(200)
    x = mid_state(rng, sc)
    assert ctx.n_res == 4
    return dict(sc=sc, ctx=ctx, orc=orc, target=target, x=x, rng=rng)


def test_aux_residual_and_objective(aux):
    import torch
    ctx, orc, x, target = aux["ctx"], aux["orc"], aux["x"], aux["target"]
    r = empty(4 * ctx.n_rays)
    F = torch.zeros(1, dtype=torch.float64, device="cuda")
    ctx.residual(cuda_tensor(x), cuda_tensor(target), r, F)
    rref, Fref = orc.residual(x.astype(np.float64), target)
    assert rel_l2(host(r), rref) < TOL_FP32
    assert rel_l2(host(r).reshape(-1, 4)[:, 3], rref.reshape(-1, 4)[:, 3]) < TOL_FP32
    assert abs(host(F)[0] - Fref) <= 1e-5 * Fref


def test_aux_jvp_vjp_apply(aux):
    import torch
    ctx, orc, x, rng = aux["ctx"], aux["orc"], aux["x"], aux["rng"]
    x64 = x.astype(np.float64)
    p = rng.normal(size=x.shape[0]).astype(np.float32)
    jp = empty(4 * ctx.n_rays)
    ctx.jvp(cuda_tensor(x), cuda_tensor(p), jp)
    ref = orc.jvp(x64, p.astype(np.float64))
    assert rel_l2(host(jp), ref) < TOL_FP32
    assert rel_l2(host(jp).reshape(-1, 4)[:, 3], ref.reshape(-1, 4)[:, 3]) < TOL_FP32
    v = rng.normal(size=4 * ctx.n_rays).astype(np.float32)
    out = empty(ctx.n_params)
    ctx.vjp(cuda_tensor(x), cuda_tensor(v), out)
    assert rel_l2(host(out), orc.vjp(x64, v.astype(np.float64))) < TOL_FP32
    # the auxiliary row alone
    va = np.zeros_like(v)
    va[3::4] = v[3::4]
    ctx.vjp(cuda_tensor(x), cuda_tensor(va), out)
    assert rel_l2(host(out), orc.vjp(x64, va.astype(np.float64))) < TOL_FP32
    ap = empty(ctx.n_params)
    pap = torch.zeros(1, dtype=torch.float64, device="cuda")
    ctx.apply_normal(cuda_tensor(x), cuda_tensor(p), ap, pap)
    assert rel_l2(host(ap), orc.apply_A(x64, p.astype(np.float64))) < TOL_FP32
    assert abs(host(pap)[0] - float(ref @ ref)) <= 1e-5 * float(ref @ ref)


def test_aux_diag_and_gradient(aux):
    ctx, orc, x, target = aux["ctx"], aux["orc"], aux["x"], aux["target"]
    x64 = x.astype(np.float64)
    rref, _ = orc.residual(x64, target)
    r32 = rref.astype(np.float32)
    d = empty(ctx.n_params)
    g = empty(ctx.n_params)
    ctx.diag_jtj(cuda_tensor(x), d, cuda_tensor(r32), g)
    dref, gref = orc.diag_grad(x64, r32.astype(np.float64))
    assert rel_l2(host(d), dref) < TOL_FP32
    assert rel_l2(host(g), gref) < TOL_FP32
    # the auxiliary row raises the opacity diagonal
    from oracle import Oracle
    sc = aux["sc"]
    d0, _ = Oracle.from_scene(sc).diag_grad(x64)
    assert np.all(dref.reshape(-1, 4)[:, 3] >= d0.reshape(-1, 4)[:, 3] - 1e-12)
    assert np.any(dref.reshape(-1, 4)[:, 3] > d0.reshape(-1, 4)[:, 3] * (1 + 1e-6))


@pytest.mark.parametrize("coef", [True, False])
def test_aux_gn_steps_parity(aux, coef):
    """Three Gauss-Newton steps with the auxiliary term (3 PCG iterations),
    each against the oracle's step from the same x: parameters within the
    Gauss-Newton tolerance; the coefficient store carries the term's per-ray
    factor in an extra row."""
    from oracle import gn_step
    ctx, orc, target = aux["ctx"], aux["orc"], aux["target"]
    ctx.set_options(pcg_iters=3, pcg_fixed=1, aux=1, aux_lambda=LAM)
    ctx.set_coef_budget(-1 if coef else 0)
    xd = cuda_tensor(aux["sc"].x0.copy())
    td = cuda_tensor(target)
    checked = 0
    for step in range(3):
        x_before = host(xd)
        st = ctx.gn_solve(xd, td, 1)[0]
        assert ctx.coef_info()["used"] == coef
        ref = gn_step(orc, x_before, target.astype(np.float64), 3)
        assert abs(st["F_before"] - ref.F_before) <= TOL_FP32 * ref.F_before
        if abs(st["gamma"] - ref.gamma) < 1e-9:
            assert rel_l2(host(xd), ref.x) < TOL_GN, step
            checked += 1
        else:
            xd = cuda_tensor(ref.x.astype(np.float32))
    ctx.set_coef_budget(-1)
    assert checked >= 2


def test_aux_rejected_where_unsupported(aux):
    import torch
    from paper_2112_05598_gb300 import PerfError, default_options
    from paper_2112_05598_gb300._binding import residual_noalloc
    sc = aux["sc"]
    o = default_options(aux=1)
    with pytest.raises(PerfError):
        residual_noalloc(sc.G, sc.radii, sc.env_h, sc.env_w, sc.c2w, sc.focal, sc.width,
                         sc.height, cuda_tensor(aux["x"]), cuda_tensor(aux["target"]),
                         empty(4 * aux["ctx"].n_rays),
                         torch.zeros(1, dtype=torch.float64, device="cuda"), options=o)

"""BF16 storage form (grid, shells, p and per-ray targets / residuals in
bfloat16; FP32 arithmetic; FP64 PCG inner products and acceptance) against
the FP64 oracle evaluated on the same dequantised BF16 inputs, and against
the FP32 path.  The marches see exactly the oracle's inputs, so render,
J p, J^T v, A p, diag and gradient keep the FP32 tolerance; the residual is
stored in BF16 (error of one BF16 rounding), and a Gauss-Newton step differs
by the BF16 rounding of p in every A p gather."""
import numpy as np
import pytest

from conftest import rel_l2
from gpu_common import TOL_FP32, cuda_tensor, empty, host, mid_state

pytestmark = pytest.mark.gpu

BF16_ULP = 2.0 ** -8      # relative spacing of bfloat16 (8 significant bits)


def _bf16(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16)


def _deq(t):
    import torch
    return t.to(torch.float32).cpu().numpy().astype(np.float64)


@pytest.fixture(scope="module")
def bf():
    from oracle import Oracle
    from paper_2112_05598_gb300 import Context, PERF_BF16
    from scenegen import make_scene
    sc = make_scene("small32")
    rng = np.random.default_rng(300)
    orc = Oracle.from_scene(sc)
    ctx = Context.from_scene(sc, dtype=PERF_BF16)
    x16 = _bf16(mid_state(rng, sc))
    target16 = _bf16(orc.render(sc.x_gt)[0].ravel())
    return dict(sc=sc, orc=orc, ctx=ctx, x16=x16, xq=_deq(x16), t16=target16, tq=_deq(target16),
                rng=rng)


def test_bf16_render_jvp_vjp_apply(bf):
    ctx, orc, x16, xq, rng = bf["ctx"], bf["orc"], bf["x16"].cuda(), bf["xq"], bf["rng"]
    rgb = empty(3 * ctx.n_rays)
    ctx.render(x16, rgb)
    assert rel_l2(host(rgb), orc.render(xq)[0]) < TOL_FP32
    p = rng.normal(size=ctx.n_params).astype(np.float32)
    jp = empty(3 * ctx.n_rays)
    ctx.jvp(x16, cuda_tensor(p), jp)
    assert rel_l2(host(jp), orc.jvp(xq, p.astype(np.float64))) < TOL_FP32
    v = rng.normal(size=3 * ctx.n_rays).astype(np.float32)
    out = empty(ctx.n_params)
    ctx.vjp(x16, cuda_tensor(v), out)
    assert rel_l2(host(out), orc.vjp(xq, v.astype(np.float64))) < TOL_FP32
    ap = empty(ctx.n_params)
    ctx.apply_normal(x16, cuda_tensor(p), ap)
    assert rel_l2(host(ap), orc.apply_A(xq, p.astype(np.float64))) < TOL_FP32


def test_bf16_residual_diag_grad(bf):
    import torch
    ctx, orc, x16, xq = bf["ctx"], bf["orc"], bf["x16"].cuda(), bf["xq"]
    t16 = bf["t16"].cuda()
    r16 = torch.zeros(3 * ctx.n_rays, dtype=torch.bfloat16, device="cuda")
    F = torch.zeros(1, dtype=torch.float64, device="cuda")
    ctx.residual(x16, t16, r16, F)
    rref, Fref = orc.residual(xq, bf["tq"])
    # F accumulates the FP32 residuals in FP64 before they are stored
    assert abs(host(F)[0] - Fref) <= TOL_FP32 * Fref
    # the stored residual carries one BF16 rounding
    rq = _deq(r16)
    assert np.all(np.abs(rq - rref) <= BF16_ULP * np.abs(rref) + 1e-6)
    d = empty(ctx.n_params)
    g = empty(ctx.n_params)
    ctx.diag_jtj(x16, d, r16, g)
    dref, gref = orc.diag_grad(xq, rq)
    assert rel_l2(host(d), dref) < TOL_FP32
    assert rel_l2(host(g), gref) < TOL_FP32


def test_bf16_gn_step_against_oracle_and_fp32(bf):
    """One Gauss-Newton step (20 PCG iterations) from a BF16-exact start:
    accepted on all three paths, F before the step exact to FP32, and the
    step's objective within 1% of the oracle's and of the FP32 path's."""
    from oracle import gn_step
    from paper_2112_05598_gb300 import Context
    sc, orc, ctx = bf["sc"], bf["orc"], bf["ctx"]
    x0q = _deq(_bf16(sc.x0)).astype(np.float32)
    ctx.set_options(pcg_iters=sc.cfg.pcg_iters, pcg_fixed=1)
    xb = cuda_tensor(x0q)
    st = ctx.gn_solve(xb, bf["t16"].cuda(), 1)[0]
    ref = gn_step(orc, x0q.astype(np.float64), bf["tq"], sc.cfg.pcg_iters)
    c32 = Context.from_scene(sc, pcg_iters=sc.cfg.pcg_iters, pcg_fixed=1)
    x32 = cuda_tensor(x0q)
    st32 = c32.gn_solve(x32, cuda_tensor(bf["tq"].astype(np.float32)), 1)[0]
    assert st["accepted"] and ref.accepted and st32["accepted"]
    assert abs(st["F_before"] - ref.F_before) <= TOL_FP32 * ref.F_before
    assert abs(st["F_after"] - ref.F_after) <= 1e-2 * ref.F_after
    assert abs(st["F_after"] - st32["F_after"]) <= 1e-2 * st32["F_after"]
    xg = host(xb)
    print(f"BF16 GN step: x vs oracle {rel_l2(xg, ref.x):.3e}, vs FP32 path "
          f"{rel_l2(xg, host(x32)):.3e}; F_after {st['F_after']:.6g} / oracle "
          f"{ref.F_after:.6g} / FP32 {st32['F_after']:.6g}")

"""Cube-map environment shells (Section "Implementation") on the CUDA path
against the FP64 oracle, element by element, through the C ABI: the 32^3
workload with its shells stored as cube maps (16 x 16 texels per face),
every per-call operation, Gauss-Newton steps with the A p from the
coefficient store and recomputed, and a batch holding cube-map and
equirectangular scenes together.  The hit point, face and texel coordinates
are binary32 on both sides, so the texel decisions agree exactly; the bars
are the FP32 ones of the equirectangular tests."""
import numpy as np
import pytest

from conftest import rel_l2, tiny_problem
from gpu_common import (TOL_FP32, TOL_GN, assert_elementwise, assert_params, cuda_tensor, empty,
                        host, make_pair, mid_state, pair_from_scene)

pytestmark = pytest.mark.gpu


def _check(name, got, ref, mag=None, tol=TOL_FP32):
    err = rel_l2(got, ref)
    print(f"[cube] {name}: rel L2 {err:.3e}")
    assert err < tol, (name, err)
    assert_elementwise(got, ref, mag, what=name)


@pytest.fixture(scope="module")
def cube():
    from scenegen import make_scene
    sc = make_scene("small32", env="cube")
    assert sc.env_kind == 1 and sc.env_w == 6 * sc.env_h
    ctx, orc = pair_from_scene(sc)
    rng = np.random.default_rng(600)
    target = orc.render(sc.x_gt)[0].astype(np.float32).ravel()
    x = mid_state(rng, sc)
    return dict(sc=sc, ctx=ctx, orc=orc, target=target, x=x, x64=x.astype(np.float64), rng=rng)


def test_cube_render_residual(cube):
    import torch
    ctx, orc, x, x64, target = cube["ctx"], cube["orc"], cube["x"], cube["x64"], cube["target"]
    rgb = empty(3 * ctx.n_rays)
    T = empty(ctx.n_rays)
    ctx.render(cuda_tensor(x), rgb, T)
    ref, Tref, _ = orc.render(x64)
    _check("render", host(rgb), ref)
    _check("T", host(T), Tref)
    r = empty(3 * ctx.n_rays)
    F = torch.zeros(1, dtype=torch.float64, device="cuda")
    ctx.residual(cuda_tensor(x), cuda_tensor(target), r, F)
    rref, Fref = orc.residual(x64, target)
    _check("residual", host(r), rref, np.abs(rref + target) + np.abs(target))
    assert abs(host(F)[0] - Fref) <= TOL_FP32 * Fref


def test_cube_jvp_vjp_apply_diag(cube):
    ctx, orc, x, x64, rng = cube["ctx"], cube["orc"], cube["x"], cube["x64"], cube["rng"]
    p = rng.normal(size=ctx.n_params).astype(np.float32)
    jp = empty(3 * ctx.n_rays)
    ctx.jvp(cuda_tensor(x), cuda_tensor(p), jp)
    jref, jmag = orc.jvp(x64, p.astype(np.float64), mag=True)
    _check("J p", host(jp), jref, jmag)
    v = rng.normal(size=3 * ctx.n_rays).astype(np.float32)
    out = empty(ctx.n_params)
    ctx.vjp(cuda_tensor(x), cuda_tensor(v), out)
    vref, vmag = orc.vjp(x64, v.astype(np.float64), mag=True)
    _check("J^T v", host(out), vref, vmag)
    # the shells' share of J^T v is not negligible: the texels are exercised
    nv = 4 * ctx.G ** 3
    assert np.linalg.norm(vref[nv:]) > 1e-2 * np.linalg.norm(vref)
    ap = empty(ctx.n_params)
    ctx.apply_normal(cuda_tensor(x), cuda_tensor(p), ap)
    _check("A p", host(ap), orc.vjp(x64, jref), orc.vjp(x64, jmag, mag=True)[1])
    rref, _ = orc.residual(x64, cube["target"])
    r32 = rref.astype(np.float32)
    d = empty(ctx.n_params)
    g = empty(ctx.n_params)
    ctx.diag_jtj(cuda_tensor(x), d, cuda_tensor(r32), g)
    dref, gref = orc.diag_grad(x64, r32.astype(np.float64))
    _check("diag", host(d), dref)
    _check("grad", host(g), gref, orc.vjp(x64, r32.astype(np.float64), mag=True)[1])


@pytest.mark.parametrize("coef", [True, False])
def test_cube_gn_steps(cube, coef):
    """Three Gauss-Newton steps (3 PCG iterations each), each against one
    oracle step from the same x."""
    from oracle import gn_step
    from paper_2112_05598_gb300 import Context
    sc, orc, target = cube["sc"], cube["orc"], cube["target"]
    ctx = Context.from_scene(sc, pcg_iters=3, pcg_fixed=1)
    ctx.set_coef_budget(-1 if coef else 0)
    xd = cuda_tensor(sc.x0.copy())
    td = cuda_tensor(target)
    checked = 0
    for step in range(3):
        xb = host(xd)
        st = ctx.gn_solve(xd, td, 1)[0]
        assert ctx.coef_info()["used"] == coef
        ref = gn_step(orc, xb, target, 3)
        assert st["accepted"] == ref.accepted
        assert abs(st["F_before"] - ref.F_before) <= TOL_FP32 * ref.F_before
        if abs(st["gamma"] - ref.gamma) > 1e-9:
            mus = [m for _, m in ref.trace]
            assert any(abs(a - b) <= 1e-6 * abs(a) for a, b in zip(mus, mus[1:]))
            xd = cuda_tensor(ref.x.astype(np.float32))
            continue
        assert_params(host(xd), ref.x, ref.diag, TOL_GN, what=f"cube GN step {step} coef={coef}")
        checked += 1
    assert checked >= 2


def test_cube_tiny_edge_cases():
    """Smallest faces (2 x 2 texels), a ragged image and several shells."""
    rng = np.random.default_rng(61)
    prob = tiny_problem(rng, G=7, n_cams=3, res=11, radii=(2.2, 3.5, 6.0), env_h=2, env_w=12)
    ctx, orc = make_pair(prob["G"], prob["radii"], 2, 12, prob["c2w"], prob["focal"], 11, 11,
                         env_kind=1)
    x = prob["x"]
    rgb = empty(3 * ctx.n_rays)
    ctx.render(cuda_tensor(x), rgb)
    _check("tiny render", host(rgb), orc.render(x.astype(np.float64))[0])
    v = rng.normal(size=3 * ctx.n_rays).astype(np.float32)
    out = empty(ctx.n_params)
    ctx.vjp(cuda_tensor(x), cuda_tensor(v), out)
    _check("tiny J^T v", host(out), *orc.vjp(x.astype(np.float64), v.astype(np.float64), mag=True))


def test_cube_rejects_a_non_strip_map():
    from paper_2112_05598_gb300 import Context, PerfError
    rng = np.random.default_rng(62)
    prob = tiny_problem(rng, G=4, env_h=4, env_w=8)
    with pytest.raises(PerfError):
        Context(4, prob["radii"], 4, 8, prob["c2w"], prob["focal"], 4, 4, env_kind=1)


def test_batch_with_cube_and_equirect_scenes():
    """A batch mixing both shell kinds: each scene's residual and one
    Gauss-Newton step against the oracle."""
    import torch
    from oracle import Oracle, gn_step
    from paper_2112_05598_gb300 import Batch
    from scenegen import constant_params, make_cameras, random_params
    scenes = []
    for i, (G, kind, F) in enumerate(((14, 1, 6), (11, 0, 8), (17, 1, 4))):
        r2 = np.random.default_rng(900 + i)
        c2w, focal = make_cameras(r2, 3, 20, 3.0, "sphere", 40.0)
        eh, ew = (F, 6 * F) if kind == 1 else (F, 2 * F)
        x_gt = random_params(r2, G, 2, eh, ew, 0.0, 0.8)
        orc = Oracle(G, (2.0, 4.0), eh, ew, c2w, focal, 20, 20, max_samples=64, env_kind=kind)
        tgt = orc.render(x_gt.astype(np.float64))[0].astype(np.float32).ravel()
        x = (0.5 * x_gt + 0.5 * constant_params(G, 2, eh, ew)).astype(np.float32)
        scenes.append(dict(G=G, radii=(2.0, 4.0), env_h=eh, env_w=ew, env_kind=kind, c2w=c2w,
                           focal=focal, width=20, height=20, x=x, target=tgt, orc=orc))
    b = Batch(scenes, max_samples=64, pcg_iters=3, pcg_fixed=1)
    x = cuda_tensor(np.concatenate([s["x"] for s in scenes]))
    t = cuda_tensor(np.concatenate([s["target"] for s in scenes]))
    r = empty(3 * b.n_rays)
    F = torch.zeros(b.n, dtype=torch.float64, device="cuda")
    b.residual(x, t, r, F)
    rh = host(r)
    for i, s in enumerate(scenes):
        rref, Fref = s["orc"].residual(s["x"].astype(np.float64), s["target"])
        _check(f"batch residual {i}", rh[3 * b.ray_off[i]:3 * b.ray_off[i + 1]], rref,
               np.abs(rref + s["target"]) + np.abs(s["target"]))
    xb = host(x)
    stats = b.gn_solve(x, t, 1)[0]
    xa = host(x)
    for i, s in enumerate(scenes):
        sl = slice(b.param_off[i], b.param_off[i + 1])
        ref = gn_step(s["orc"], xb[sl], s["target"], 3)
        assert stats[i]["accepted"] == ref.accepted
        if abs(stats[i]["gamma"] - ref.gamma) <= 1e-9:
            assert_params(xa[sl], ref.x, ref.diag, TOL_GN, what=f"batch cube/equirect scene {i}")

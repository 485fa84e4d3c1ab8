"""Brick order of a Gauss-Newton step's PCG vectors (perf_set_brick,
perf_batch_set_brick) on the CUDA path, against the FP64 oracle through the
C ABI.

With a brick edge set and the A p of the step running from the coefficient
store, the diagonal march writes the Jacobi diagonal, the gradient and the
block couplings in brick order, the PCG works on p, A p, Delta and rho in
that order, and the trial point maps Delta back to the canonical x.  The
order is a permutation of the parameter blocks, so each Gauss-Newton step
must match the oracle's step to the same bar as the canonical order (the
atomic additions land in another order, nothing else changes)."""
import numpy as np
import pytest

from conftest import rel_l2
from gpu_common import TOL_FP32, TOL_GN, assert_params, cuda_tensor, host

pytestmark = pytest.mark.gpu


def _steps(sc, orc, target, edge, n_steps=3, pcg=3, coef=True):
    """n_steps Gauss-Newton steps of the GPU with brick edge `edge`, each
    checked against one oracle step from the GPU's state before it."""
    from oracle import gn_step
    from paper_2112_05598_gb300 import Context
    ctx = Context.from_scene(sc, pcg_iters=pcg, pcg_fixed=1)
    ctx.set_coef_budget(-1 if coef else 0)
    ctx.set_brick(edge)
    xd = cuda_tensor(sc.x0.copy())
    td = cuda_tensor(target)
    checked = 0
    for step in range(n_steps):
        xb = host(xd)
        st = ctx.gn_solve(xd, td, 1)[0]
        assert ctx.coef_info()["used"] == coef
        ref = gn_step(orc, xb, target, pcg)
        assert st["accepted"] == ref.accepted
        assert abs(st["F_before"] - ref.F_before) <= TOL_FP32 * ref.F_before
        if abs(st["gamma"] - ref.gamma) > 1e-9:
            mus = [m for _, m in ref.trace]
            assert any(abs(a - b) <= 1e-6 * abs(a) for a, b in zip(mus, mus[1:]))
            xd = cuda_tensor(ref.x.astype(np.float32))
            continue
        assert_params(host(xd), ref.x, ref.diag, TOL_GN, what=f"brick {edge} step {step}")
        checked += 1
    assert checked >= 2
    return host(xd)


@pytest.fixture(scope="module")
def s32():
    from oracle import Oracle
    from scenegen import make_scene
    sc = make_scene("small32")
    orc = Oracle.from_scene(sc)
    target = orc.render(sc.x_gt)[0].astype(np.float32).ravel()
    return sc, orc, target


@pytest.mark.parametrize("edge", [2, 4, 8])
def test_brick_gn_steps_against_oracle(s32, edge):
    sc, orc, target = s32
    _steps(sc, orc, target, edge)


def test_brick_equals_canonical_order(s32):
    """Three steps in 4^3 bricks and in the canonical order from the same
    start end at the same parameters (up to the order of the atomic sums)."""
    sc, orc, target = s32
    xb = _steps(sc, orc, target, 4)
    xc = _steps(sc, orc, target, 1)
    err = rel_l2(xb, xc)
    print(f"[brick] 4^3 vs canonical after 3 steps: rel L2 {err:.3e}")
    assert err < 1e-4


def test_brick_with_exact_block_jacobi(s32):
    """Exact block-Jacobi reads the diagonal and the block couplings the
    diagonal march writes in brick order (through the same key as the
    diagonal, which the Jacobi tests above check; the block inverse and its
    application are per voxel, blind to the order): a step in 4^3 bricks
    equals the canonical order's step up to rounding.  Near-singular blocks
    (Schur complement just above its 1e-4 cut) amplify the rounding of the
    atomic sums, whose order differs, by up to ~1e4: one step measured x
    4.4e-3, F after 8e-6 and the image 3.7e-4 apart, against 5e-7 on x for
    Jacobi.  The bars leave room for that and still catch a misplaced block,
    which changes the preconditioned step itself."""
    from paper_2112_05598_gb300 import PERF_PRECOND_BLOCK_JACOBI, Context
    sc, orc, target = s32
    out = {}
    for edge in (1, 4):
        ctx = Context.from_scene(sc, pcg_iters=3, pcg_fixed=1, precond=PERF_PRECOND_BLOCK_JACOBI)
        ctx.set_brick(edge)
        xd = cuda_tensor(sc.x0.copy())
        st = ctx.gn_solve(xd, cuda_tensor(target), 1)[0]
        assert st["accepted"] and not st["precond_fallback"]
        rgb = cuda_tensor(np.zeros(3 * ctx.n_rays, np.float32))
        ctx.render(xd, rgb)
        out[edge] = (host(xd), st["F_after"], host(rgb))
    dx = rel_l2(out[4][0], out[1][0])
    dF = abs(out[4][1] - out[1][1]) / out[1][1]
    dimg = rel_l2(out[4][2], out[1][2])
    print(f"[brick] block-Jacobi 4^3 vs canonical: x {dx:.3e}, F_after {dF:.3e}, image {dimg:.3e}")
    assert dF < 1e-4 and dimg < 2e-3 and dx < 3e-2


def test_brick_without_the_store_stays_canonical(s32):
    """With the coefficient store off the steps run in the canonical order
    (the recomputing A p has no brick form): same parity."""
    sc, orc, target = s32
    _steps(sc, orc, target, 8, n_steps=2, coef=False)


def test_brick_edge_must_divide_G():
    from paper_2112_05598_gb300 import Context, PerfError
    from scenegen import make_scene
    sc = make_scene("small32", G=20)
    ctx = Context.from_scene(sc)
    ctx.set_brick(4)
    with pytest.raises(PerfError):
        ctx.set_brick(8)
    with pytest.raises(PerfError):
        ctx.set_brick(3)


def test_brick_bf16_equals_canonical():
    """BF16 storage: p is gathered from its bfloat16 copy in brick order; one
    step with 4^3 bricks equals the canonical step."""
    from paper_2112_05598_gb300 import PERF_BF16, Context
    from oracle import Oracle
    from scenegen import make_scene
    sc = make_scene("small32")
    target = Oracle.from_scene(sc).render(sc.x_gt)[0].astype(np.float32)
    out = {}
    for edge in (1, 4):
        ctx = Context.from_scene(sc, dtype=PERF_BF16, pcg_iters=3, pcg_fixed=1)
        ctx.set_brick(edge)
        xd = cuda_tensor(sc.x0.copy())
        import torch
        td = cuda_tensor(target).to(torch.bfloat16)
        st = ctx.gn_solve(xd, td, 1)[0]
        assert st["accepted"] and ctx.coef_info()["used"]
        out[edge] = host(xd)
    err = rel_l2(out[4], out[1])
    print(f"[brick] bf16 4^3 vs canonical: rel L2 {err:.3e}")
    assert err < 1e-4


def test_batch_brick_against_oracle():
    """A batch whose grids are multiples of 4 (bricked) and one that is not
    (stays canonical): each scene's Gauss-Newton step against the oracle."""
    from oracle import Oracle, gn_step
    from paper_2112_05598_gb300 import Batch
    from scenegen import constant_params, make_cameras, random_params
    scenes = []
    for i, G in enumerate((16, 14, 12)):
        r2 = np.random.default_rng(950 + i)
        c2w, focal = make_cameras(r2, 3, 20, 3.0, "sphere", 40.0)
        x_gt = random_params(r2, G, 2, 8, 16, 0.0, 0.8)
        orc = Oracle(G, (2.0, 4.0), 8, 16, c2w, focal, 20, 20, max_samples=64)
        tgt = orc.render(x_gt.astype(np.float64))[0].astype(np.float32).ravel()
        x = (0.5 * x_gt + 0.5 * constant_params(G, 2, 8, 16)).astype(np.float32)
        scenes.append(dict(G=G, radii=(2.0, 4.0), env_h=8, env_w=16, c2w=c2w, focal=focal,
                           width=20, height=20, x=x, target=tgt, orc=orc))
    b = Batch(scenes, max_samples=64, pcg_iters=3, pcg_fixed=1)
    b.set_brick(4)
    x = cuda_tensor(np.concatenate([s["x"] for s in scenes]))
    t = cuda_tensor(np.concatenate([s["target"] for s in scenes]))
    xb = host(x)
    stats = b.gn_solve(x, t, 1)[0]
    assert b.coef_info()["used"]
    xa = host(x)
    checked = 0
    for i, s in enumerate(scenes):
        sl = slice(b.param_off[i], b.param_off[i + 1])
        ref = gn_step(s["orc"], xb[sl], s["target"], 3)
        assert stats[i]["accepted"] == ref.accepted
        if abs(stats[i]["gamma"] - ref.gamma) <= 1e-9:
            assert_params(xa[sl], ref.x, ref.diag, TOL_GN, what=f"batch brick scene {i} (G={s['G']})")
            checked += 1
    assert checked >= 2


@pytest.mark.parametrize("G, edge", [(2, 2), (6, 2), (8, 8)])
def test_brick_small_grids(G, edge):
    """Small grids in brick order (a single brick, a grid of three bricks per
    edge, one brick of 8^3) on a ragged image with rays that miss the grid:
    one Gauss-Newton step against the oracle."""
    from conftest import tiny_problem
    from gpu_common import make_pair
    from oracle import gn_step
    rng = np.random.default_rng(40 + G)
    # cameras at radius 6: the grid spans about 32 of the 40 degrees, so
    # the image's edge rays miss it
    prob = tiny_problem(rng, G=G, n_cams=3, res=13, radii=(2.5, 8.0), env_h=4, env_w=8,
                        cam_radius=6.0)
    ctx, orc = make_pair(prob["G"], prob["radii"], 4, 8, prob["c2w"], prob["focal"], 13, 13,
                         pcg_iters=3, pcg_fixed=1)
    ctx.set_brick(edge)
    x = prob["x"].astype(np.float32)
    target = orc.render(rng.uniform(0, 1, size=x.shape))[0].astype(np.float32).ravel()
    xd = cuda_tensor(x.copy())
    st = ctx.gn_solve(xd, cuda_tensor(target), 1)[0]
    assert ctx.coef_info()["used"]
    ref = gn_step(orc, x.astype(np.float64), target, 3)
    assert st["accepted"] == ref.accepted
    if abs(st["gamma"] - ref.gamma) <= 1e-9:
        assert_params(host(xd), ref.x, ref.diag, TOL_GN, what=f"brick {edge} on {G}^3")

"""Coefficient-cached A p: the per-sample derivatives stored by a Gauss-Newton
step's diagonal march replace the recomputation in every PCG iteration.  The
step must equal the recomputing path up to rounding (both are checked
against the oracle in test_gpu_parity.py), under jitter, with a re-tiled
context, in BF16 storage, and when the store does not fit its budget."""
import numpy as np
import pytest

from conftest import rel_l2
from gpu_common import (TOL_FP32, TOL_GN, assert_params, cuda_tensor, host, mid_state,
                        pair_from_scene)

pytestmark = pytest.mark.gpu


def _scene():
    from scenegen import make_scene
    return make_scene("small32")


def _step(sc, target, x, budget, pcg_iters=3, tune=None, **kw):
    import torch
    from paper_2112_05598_gb300 import PERF_BF16, Context
    ctx = Context.from_scene(sc, pcg_iters=pcg_iters, pcg_fixed=1, **kw)
    tdt = torch.bfloat16 if kw.get("dtype") == PERF_BF16 else None
    ctx.set_coef_budget(budget)
    xd = cuda_tensor(x)
    if tune is not None:
        ctx.set_coef_budget(0)
        ctx.autotune(xd)
        ctx.set_coef_budget(budget)
    st = ctx.gn_solve(xd, cuda_tensor(target, tdt), 2)
    return st, host(xd), ctx.coef_info()


@pytest.fixture(scope="module")
def prob():
    sc = _scene()
    ctx, orc = pair_from_scene(sc)
    target = orc.render(sc.x_gt)[0].astype(np.float32).ravel()
    x = mid_state(np.random.default_rng(5), sc)
    return sc, target, x


@pytest.mark.parametrize("kw", [{}, {"jitter": 1, "seed": 9, "epoch": 3}])
def test_coef_step_equals_recompute(prob, kw):
    sc, target, x = prob
    st_c, x_c, info_c = _step(sc, target, x, -1, **kw)
    st_r, x_r, info_r = _step(sc, target, x, 0, **kw)
    assert info_c["used"] and info_c["bytes"] > 0
    assert not info_r["used"] and info_r["bytes"] == 0
    for a, b in zip(st_c, st_r):
        assert abs(a["F_before"] - b["F_before"]) <= TOL_FP32 * b["F_before"]
        assert abs(a["F_after"] - b["F_after"]) <= TOL_FP32 * b["F_after"]
        assert a["accepted"] == b["accepted"]
    assert rel_l2(x_c, x_r) < TOL_FP32


def test_coef_store_size(prob):
    """16 bytes per (tile row, lane): rows = the tile's largest sample count
    plus one per shell, summed over the 8x4 tiles."""
    from paper_2112_05598_gb300 import Context
    sc, target, x = prob
    ctx = Context.from_scene(sc, pcg_iters=1, pcg_fixed=1)
    ctx.gn_solve(cuda_tensor(x), cuda_tensor(target), 1)
    info = ctx.coef_info()
    assert info["used"]
    from oracle import Oracle
    orc = Oracle(sc.G, sc.radii, sc.env_h, sc.env_w, sc.c2w, sc.focal, sc.width, sc.height,
                 max_samples=sc.cfg.max_samples)
    n_rays = len(sc.c2w) * sc.height * sc.width
    K = np.array([orc.ray_info(r)["K"] for r in range(n_rays)]).reshape(len(sc.c2w), sc.height,
                                                                        sc.width)
    rows = 0
    for c in range(K.shape[0]):
        for ty in range(0, sc.height, 4):
            for tx in range(0, sc.width, 8):
                rows += int(K[c, ty:ty + 4, tx:tx + 8].max()) + len(sc.radii)
    assert info["bytes"] == rows * 32 * 16


def test_coef_retiled_context(prob):
    """Tiles chosen by the autotuner without the store, then the store laid
    out for that tiling."""
    sc, target, x = prob
    st_c, x_c, info_c = _step(sc, target, x, -1, tune=True)
    st_r, x_r, _ = _step(sc, target, x, 0)
    assert info_c["used"]
    assert rel_l2(x_c, x_r) < TOL_FP32


def test_coef_over_budget_recomputes(prob):
    sc, target, x = prob
    st_s, x_s, info_s = _step(sc, target, x, 1024)
    st_r, x_r, _ = _step(sc, target, x, 0)
    assert not info_s["used"] and info_s["bytes"] == 0
    assert rel_l2(x_s, x_r) < TOL_FP32


def test_coef_bf16(prob):
    from paper_2112_05598_gb300 import PERF_BF16
    sc, target, x = prob
    st_c, x_c, info_c = _step(sc, target, x, -1, dtype=PERF_BF16)
    st_r, x_r, _ = _step(sc, target, x, 0, dtype=PERF_BF16)
    assert info_c["used"]
    for a, b in zip(st_c, st_r):
        assert abs(a["F_after"] - b["F_after"]) <= 1e-4 * b["F_after"]
    assert rel_l2(x_c, x_r) < 1e-4


def test_coef_autotune_reports_coef(prob):
    from paper_2112_05598_gb300 import Context
    sc, target, x = prob
    ctx = Context.from_scene(sc, pcg_iters=2, pcg_fixed=1)
    t = ctx.autotune(cuda_tensor(x))
    assert t["coef"] == 1 and t["tile_w"] * t["tile_h"] == 32 and t["apply_ms"] > 0
    assert ctx.coef_info()["used"]
    # a Gauss-Newton step after tuning (store laid out for the chosen tiles)
    # equals the recomputing path
    xd = cuda_tensor(x)
    st = ctx.gn_solve(xd, cuda_tensor(target), 1)
    st_r, x_r, _ = _step(sc, target, x, 0, pcg_iters=2)
    assert ctx.coef_info()["used"]
    assert abs(st[0]["F_after"] - st_r[0]["F_after"]) <= TOL_FP32 * st_r[0]["F_after"]


@pytest.mark.parametrize("aux", [0, 1])
def test_coef_ragged_tiles_and_missing_rays(aux):
    """Odd image sizes (partial 8x4 tiles at the right and bottom edges),
    cameras far enough out that some rays miss the grid (K = 0) and hit only
    shells: the store's rows and the lanes without pixels are handled, with
    and without the auxiliary row."""
    from conftest import tiny_problem
    from paper_2112_05598_gb300 import Context
    rng = np.random.default_rng(31)
    prob = tiny_problem(rng, G=12, n_cams=3, res=13, radii=(2.5, 5.0), cam_radius=4.5,
                        sigma=(0.0, 0.5))
    target = rng.uniform(0, 1, size=3 * 3 * 13 * 13).astype(np.float32)
    out = {}
    for budget in (-1, 0):
        ctx = Context(prob["G"], prob["radii"], prob["env_h"], prob["env_w"], prob["c2w"],
                      prob["focal"], 13, 13, max_samples=64, pcg_iters=1, pcg_fixed=1, aux=aux)
        ctx.set_coef_budget(budget)
        xd = cuda_tensor(prob["x"])
        st = ctx.gn_solve(xd, cuda_tensor(target), 1)
        out[budget] = (st[0], host(xd), ctx.coef_info()["used"])
        ctx.close()
    (a, xa, ua), (b, xb, ub) = out[-1], out[0]
    assert ua and not ub
    assert abs(a["F_after"] - b["F_after"]) <= TOL_FP32 * b["F_after"]
    assert rel_l2(xa, xb) < TOL_FP32


def test_coef_partial_store(prob):
    """A budget of about half the store: the longest tile prefix that fits
    reads the store, the other tiles recompute (paired records), in the same
    A p; the step equals the recomputing path."""
    sc, target, x = prob
    _, _, full = _step(sc, target, x, -1)
    assert full["coverage"] == 1.0
    st_p, x_p, part = _step(sc, target, x, full["bytes"] // 2)
    st_r, x_r, _ = _step(sc, target, x, 0)
    assert part["used"] and 0.2 < part["coverage"] < 0.8
    assert 0 < part["bytes"] <= full["bytes"] // 2
    for a, b in zip(st_p, st_r):
        assert abs(a["F_after"] - b["F_after"]) <= TOL_FP32 * b["F_after"]
    assert rel_l2(x_p, x_r) < TOL_FP32


def _opaque(sc, scale=300.0):
    """The ground truth with its opacities scaled up: past a primitive's
    first voxel a ray's transmittance underflows to 0 in binary32 (optical
    depth above about 104), so its later coefficient rows are zero."""
    x = sc.x_gt.astype(np.float64).reshape(-1, 4).copy()
    x[:sc.G ** 3, 3] *= scale
    return x.astype(np.float32).ravel()


@pytest.mark.parametrize("aux", [0, 1])
def test_zero_tail_rows_skipped_exactly(prob, aux):
    """Rows past a ray's last non-zero one are neither written nor read:
    on an opaque state the A p reads fewer rows than the rays have samples
    (perf_coef_prefix), and the step still equals the recomputing path,
    which visits every sample, and the oracle's step.  At the constant start
    nothing underflows and every row is read."""
    from oracle import Oracle, gn_step
    from paper_2112_05598_gb300 import Context
    sc, target, _ = prob
    xo = _opaque(sc)
    res = {}
    for budget in (-1, 0):
        ctx = Context.from_scene(sc, pcg_iters=3, pcg_fixed=1, aux=aux, aux_lambda=0.01)
        ctx.set_coef_budget(budget)
        xd = cuda_tensor(xo.copy())
        st = ctx.gn_solve(xd, cuda_tensor(target), 1)[0]
        res[budget] = (st, host(xd))
        if budget == -1:
            assert ctx.coef_info()["used"]
            pre = ctx.coef_prefix()
            print(f"[coef] opaque state, aux {aux}: {pre['read']} of {pre['total']} rows read")
            assert 0 < pre["read"] < pre["total"]
            x0 = cuda_tensor(sc.x0.copy())
            ctx.gn_solve(x0, cuda_tensor(target), 1)
            pre0 = ctx.coef_prefix()
            assert pre0["read"] == pre0["total"] > 0
        ctx.close()
    (a, xa), (b, xb) = res[-1], res[0]
    assert a["accepted"] == b["accepted"]
    assert abs(a["F_after"] - b["F_after"]) <= TOL_FP32 * b["F_after"]
    assert rel_l2(xa, xb) < TOL_FP32
    orc = Oracle(sc.G, sc.radii, sc.env_h, sc.env_w, sc.c2w, sc.focal, sc.width, sc.height,
                 max_samples=sc.cfg.max_samples, aux=aux, aux_lambda=0.01)
    ref = gn_step(orc, xo.astype(np.float64), target, 3)
    assert a["accepted"] == ref.accepted
    assert abs(a["F_before"] - ref.F_before) <= TOL_FP32 * ref.F_before
    if abs(a["gamma"] - ref.gamma) <= 1e-9:
        assert_params(xa, ref.x, ref.diag, TOL_GN, what=f"opaque state, aux {aux}")


def test_coef_prefix_needs_a_filled_store(prob):
    from paper_2112_05598_gb300 import Context, PerfError
    sc, target, x = prob
    ctx = Context.from_scene(sc, pcg_iters=1, pcg_fixed=1)
    with pytest.raises(PerfError):
        ctx.coef_prefix()
    ctx.set_coef_budget(0)
    ctx.gn_solve(cuda_tensor(x), cuda_tensor(target), 1)
    with pytest.raises(PerfError):
        ctx.coef_prefix()

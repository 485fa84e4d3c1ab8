"""Batched form: uneven scenes in one persistent launch with a graph-captured
PCG loop.  Every scene of the batch must match the same scene solved alone
(the single-scene path is checked against the oracle elsewhere): residuals
and objectives exactly to FP32 accumulation order, Gauss-Newton steps to
the parameter tolerance; the autotuner's choice must not change results."""
import numpy as np
import pytest

from conftest import rel_l2
from gpu_common import TOL_FP32, TOL_GN, cuda_tensor, empty, host

pytestmark = pytest.mark.gpu


def _scenes(seed=7, n=4):
    from scenegen import batch_scene_configs, make_cameras, random_params
    rng = np.random.default_rng(seed)
    cfgs = batch_scene_configs(rng, n_scenes=n, G_lo=12, G_hi=28, cams_lo=2, cams_hi=5, res=24)
    out = []
    for i, c in enumerate(cfgs):
        r2 = np.random.default_rng(c["seed"])
        c2w, focal = make_cameras(r2, c["n_cams"], c["res"], 3.0, "sphere", 40.0)
        x = random_params(r2, c["G"], len(c["radii"]), c["env_h"], c["env_w"], 0.0, 0.6)
        tgt = r2.uniform(0, 1, size=3 * c["n_cams"] * c["res"] ** 2).astype(np.float32)
        out.append(dict(G=c["G"], radii=c["radii"], env_h=c["env_h"], env_w=c["env_w"], c2w=c2w,
                        focal=focal, width=c["res"], height=c["res"], x=x, target=tgt))
    return out


def _cat(b, scenes, key):
    return np.concatenate([s[key] for s in scenes]).astype(np.float32)


def test_batch_residual_matches_single_scenes():
    import torch
    from paper_2112_05598_gb300 import Batch, Context
    scenes = _scenes()
    b = Batch(scenes, max_samples=64)
    x = cuda_tensor(_cat(b, scenes, "x"))
    t = cuda_tensor(_cat(b, scenes, "target"))
    r = empty(3 * b.n_rays)
    F = torch.zeros(b.n, dtype=torch.float64, device="cuda")
    b.residual(x, t, r, F)
    for i, s in enumerate(scenes):
        c = Context(s["G"], s["radii"], s["env_h"], s["env_w"], s["c2w"], s["focal"], s["width"],
                    s["height"], max_samples=64)
        rr = empty(3 * c.n_rays)
        FF = torch.zeros(1, dtype=torch.float64, device="cuda")
        c.residual(cuda_tensor(s["x"]), cuda_tensor(s["target"]), rr, FF)
        sl = slice(3 * b.ray_off[i], 3 * b.ray_off[i + 1])
        assert rel_l2(host(r)[sl], host(rr)) < 1e-6
        assert abs(host(F)[i] - host(FF)[0]) <= 1e-12 * host(FF)[0]


@pytest.mark.parametrize("tune", [False, True])
def test_batch_gn_steps_match_single_scenes(tune):
    from paper_2112_05598_gb300 import Batch, Context
    scenes = _scenes(seed=11)
    b = Batch(scenes, max_samples=64, pcg_iters=3, pcg_fixed=1)
    x = cuda_tensor(_cat(b, scenes, "x"))
    t = cuda_tensor(_cat(b, scenes, "target"))
    if tune:
        info = b.autotune(x)
        assert info["tile_w"] * info["tile_h"] == 32 and info["apply_ms"] > 0
    stats = b.gn_solve(x, t, 2)
    xb = host(x)
    for i, s in enumerate(scenes):
        c = Context(s["G"], s["radii"], s["env_h"], s["env_w"], s["c2w"], s["focal"], s["width"],
                    s["height"], max_samples=64, pcg_iters=3, pcg_fixed=1)
        xs = cuda_tensor(s["x"])
        st = c.gn_solve(xs, cuda_tensor(s["target"]), 2)
        for k in range(2):
            assert stats[k][i]["accepted"] == st[k]["accepted"]
            assert abs(stats[k][i]["F_before"] - st[k]["F_before"]) <= TOL_FP32 * st[k]["F_before"]
        sl = slice(b.param_off[i], b.param_off[i + 1])
        assert rel_l2(xb[sl], host(xs)) < TOL_GN, i


def test_batch_early_exit_matches_single_scenes():
    """PCG with the exit tests (pcg_fixed = 0) inside the captured loop: each
    scene's device flag stops its A p work; iteration counts and exit
    reasons equal the single-scene solves, which exit on the host.  With up
    to 12 CG iterations the order of the FP32 scatter atomics (which differs
    between the two launch forms) is amplified by CG as for any 20-iteration
    solve, so the steps agree to 1e-2 and the objectives to 1e-3."""
    from paper_2112_05598_gb300 import Batch, Context
    scenes = _scenes(seed=5)
    kw = dict(max_samples=64, pcg_iters=12, pcg_fixed=0, pcg_eps_rel=0.05, pcg_stall=0.999)
    b = Batch(scenes, **kw)
    x = cuda_tensor(_cat(b, scenes, "x"))
    t = cuda_tensor(_cat(b, scenes, "target"))
    stats = b.gn_solve(x, t, 2)
    xb = host(x)
    iters = []
    for i, s in enumerate(scenes):
        c = Context(s["G"], s["radii"], s["env_h"], s["env_w"], s["c2w"], s["focal"], s["width"],
                    s["height"], **kw)
        xs = cuda_tensor(s["x"])
        st = c.gn_solve(xs, cuda_tensor(s["target"]), 2)
        for k in range(2):
            assert stats[k][i]["pcg_iters"] == st[k]["pcg_iters"], (i, k)
            assert stats[k][i]["pcg_exit"] == st[k]["pcg_exit"], (i, k)
            assert abs(stats[k][i]["F_after"] - st[k]["F_after"]) <= 1e-3 * st[k]["F_after"]
            iters.append(st[k]["pcg_iters"])
        sl = slice(b.param_off[i], b.param_off[i + 1])
        assert rel_l2(xb[sl], host(xs)) < 1e-2, i
    # the exit tests fired before the cap for some scene
    assert min(iters) < 12


@pytest.mark.parametrize("tune", [False, True])
def test_batch_coef_store_equals_recompute(tune):
    """The batch's coefficient store (rows over the global tile list, filled by
    the diagonal march, read by the graph-captured PCG loop) gives the same
    step as recomputing every march.  One PCG iteration, so that the two A p
    forms' FP32 rounding is not amplified by CG (these
    random-target scenes drive opacities to the hundreds, where several CG
    iterations magnify 1e-7 differences in A p to 1e-4 in x)."""
    from paper_2112_05598_gb300 import Batch
    scenes = _scenes(seed=13)
    out = {}
    for budget in (-1, 0):
        b = Batch(scenes, max_samples=64, pcg_iters=1, pcg_fixed=1)
        b.set_coef_budget(budget)
        x = cuda_tensor(_cat(b, scenes, "x"))
        t = cuda_tensor(_cat(b, scenes, "target"))
        if tune:
            info = b.autotune(x)
            assert info["coef"] == (1 if budget else 0)
        stats = b.gn_solve(x, t, 1)
        out[budget] = (stats, host(x), b.coef_info())
    (sc, xc, ic), (sr, xr, ir) = out[-1], out[0]
    assert ic["used"] and ic["bytes"] > 0 and not ir["used"]
    for k in range(1):
        for a, r in zip(sc[k], sr[k]):
            assert a["accepted"] == r["accepted"]
            assert abs(a["F_before"] - r["F_before"]) <= TOL_FP32 * r["F_before"]
            assert abs(a["F_after"] - r["F_after"]) <= TOL_FP32 * r["F_after"]
    assert rel_l2(xc, xr) < TOL_FP32


def test_batch_zero_tail_rows_equal_recompute():
    """Scenes whose opacities reach the hundreds per voxel step: past a ray's
    first opaque voxel its transmittance underflows to 0 in binary32 and the
    batch's store keeps only each ray's non-zero row prefix.  One step from
    the store equals the recomputing batch, which visits every sample."""
    from paper_2112_05598_gb300 import Batch
    scenes = _scenes(seed=17)
    for s in scenes:
        x = s["x"].astype(np.float64).reshape(-1, 4)
        x[:s["G"] ** 3, 3] *= 300.0
        s["x"] = x.astype(np.float32).ravel()
    out = {}
    for budget in (-1, 0):
        b = Batch(scenes, max_samples=64, pcg_iters=1, pcg_fixed=1)
        b.set_coef_budget(budget)
        x = cuda_tensor(_cat(b, scenes, "x"))
        t = cuda_tensor(_cat(b, scenes, "target"))
        stats = b.gn_solve(x, t, 1)
        out[budget] = (stats, host(x), b.coef_info())
    (sc, xc, ic), (sr, xr, ir) = out[-1], out[0]
    assert ic["used"] and not ir["used"]
    for a, r in zip(sc[0], sr[0]):
        assert a["accepted"] == r["accepted"]
        assert abs(a["F_after"] - r["F_after"]) <= TOL_FP32 * r["F_after"]
    assert rel_l2(xc, xr) < TOL_FP32

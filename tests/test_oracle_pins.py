"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test would fail on a plausible slip in the oracle: a dropped term or a
wrong sign in Algorithm 1 (finite differences, adjoint), a wrong index in the
interpolation chain rule (finite differences), squaring before aggregating in
the Jacobi diagonal (column norms of the dense J), a wrong compositing order
(closed forms and invariants), a wrong CG update (dense solve, conjugacy) or a
wrong line-search return (1-D quadratics)."""
import json
import math
import os

import numpy as np
import pytest

from conftest import rel_l2, tiny_problem
from oracle import Oracle, jacobi_apply, line_search, pcg, project, gn_step

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _orc(prob, **kw):
    return Oracle(prob["G"], prob["radii"], prob["env_h"], prob["env_w"],
                  prob["c2w"], prob["focal"], prob["width"], prob["height"],
                  max_samples=prob["max_samples"], **kw)


def fd_jacobian(orc, x, eps=1e-6):
    """Dense J by central differences of the forward model (Eq. 3-4) only."""
    n = x.shape[0]
    J = np.zeros((3 * orc.n_rays, n))
    for j in range(n):
        xp = x.copy(); xp[j] += eps
        xm = x.copy(); xm[j] -= eps
        J[:, j] = (orc.render(xp)[0].ravel() - orc.render(xm)[0].ravel()) / (2 * eps)
    return J


@pytest.fixture(scope="module")
def tiny():
    rng = np.random.default_rng(7)
    prob = tiny_problem(rng)
    orc = _orc(prob)
    x = prob["x"].astype(np.float64)
    J = fd_jacobian(orc, x)
    return orc, x, J


def test_jvp_columns_match_finite_differences(tiny):
    orc, x, J = tiny
    n = x.shape[0]
    Jalg = np.zeros_like(J)
    for j in range(n):
        e = np.zeros(n); e[j] = 1.0
        Jalg[:, j] = orc.jvp(x, e)
    assert np.abs(J).max() > 1e-3
    assert np.abs(Jalg - J).max() <= 1e-7 * np.abs(J).max() + 1e-9


def test_vjp_rows_match_finite_differences(tiny):
    orc, x, J = tiny
    m = J.shape[0]
    for i in range(m):
        v = np.zeros(m); v[i] = 1.0
        row = orc.vjp(x, v)
        assert np.abs(row - J[i]).max() <= 1e-7 * np.abs(J).max() + 1e-9


def test_adjoint_identity(tiny):
    orc, x, _ = tiny
    rng = np.random.default_rng(3)
    p = rng.normal(size=x.shape[0])
    v = rng.normal(size=3 * orc.n_rays)
    lhs = float(orc.jvp(x, p) @ v)
    rhs = float(p @ orc.vjp(x, v))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


def test_diag_is_column_norms_of_dense_J(tiny):
    orc, x, J = tiny
    d, _ = orc.diag_grad(x)
    ref = np.sum(J * J, axis=0)
    assert rel_l2(d, ref) < 1e-7
    # squaring per sample instead of per ray would undercount: the exact
    # diagonal must differ from the per-sample sum of squares
    assert np.max(ref) > 0


def test_grad_is_JT_r(tiny):
    orc, x, J = tiny
    rng = np.random.default_rng(4)
    target = rng.uniform(0, 1, size=3 * orc.n_rays)
    r, F = orc.residual(x, target)
    assert abs(F - 0.5 * float(r @ r)) < 1e-12
    rgb = orc.render(x)[0].ravel()
    assert np.allclose(r, rgb - target, atol=1e-14)
    _, g = orc.diag_grad(x, r)
    assert rel_l2(g, J.T @ r) < 1e-7


def test_apply_A_is_JTJ(tiny):
    orc, x, J = tiny
    rng = np.random.default_rng(5)
    p = rng.normal(size=x.shape[0])
    assert rel_l2(orc.apply_A(x, p), J.T @ (J @ p)) < 1e-7


def test_compositing_invariants():
    rng = np.random.default_rng(11)
    prob = tiny_problem(rng, G=6, n_cams=2, res=6)
    orc = _orc(prob)
    x = prob["x"].astype(np.float64)
    rgb, te, tf = orc.render(x)
    checked = 0
    for ray in range(orc.n_rays):
        s = orc.ray_samples(x, ray)
        n = len(s["T"])
        if n == 0:
            continue
        T = s["T"]
        # T non-increasing (Eq. 4 with sigma >= 0)
        assert np.all(np.diff(T) <= 1e-15)
        # telescoping: sum_i T_i alpha_i = 1 - T_final
        w = T * s["alpha"]
        assert abs(w.sum() - (1.0 - tf[ray])) < 1e-13
        # the per-sample records recombine to the rendered colour
        assert np.allclose((w[:, None] * s["c"]).sum(0), rgb[ray], atol=1e-13)
        # grid transmittance at the exit is the product over grid samples
        ng = s["n_grid"]
        Te = float(np.prod(1.0 - s["alpha"][:ng])) if ng else 1.0
        assert abs(Te - te[ray]) < 1e-13
        checked += 1
    assert checked > 10


def test_opaque_first_sample_returns_its_colour():
    rng = np.random.default_rng(12)
    prob = tiny_problem(rng, G=5, n_cams=2, res=5)
    orc = _orc(prob)
    x = prob["x"].astype(np.float64).reshape(-1, 4)
    g = prob["G"] ** 3
    x[:g, 3] = 200.0     # every voxel opaque: alpha = 1 - e^-200 per step
    x = x.reshape(-1)
    rgb = orc.render(x)[0]
    hits = 0
    for ray in range(orc.n_rays):
        s = orc.ray_samples(x, ray)
        if s["n_grid"] == 0 or s["dbar"][0] < 0.5:
            continue
        assert np.allclose(rgb[ray], s["c"][0], atol=1e-12)
        hits += 1
    assert hits > 5


def test_empty_grid_is_pure_shell_composite():
    """sigma == 0 in the grid: H^ = (1 - e^-sigma_s) c_s for one constant
    shell (a single composited shell sample with delta_bar = 1)."""
    rng = np.random.default_rng(13)
    prob = tiny_problem(rng, G=4, radii=(2.5,), n_cams=2, res=5)
    orc = _orc(prob)
    x = prob["x"].astype(np.float64).reshape(-1, 4)
    g = prob["G"] ** 3
    x[:g, 3] = 0.0
    cs = np.array([0.2, 0.5, 0.9]); ss = 0.7
    x[g:, 0:3] = cs
    x[g:, 3] = ss
    rgb = orc.render(x.reshape(-1))[0]
    assert np.allclose(rgb, (1 - math.exp(-ss)) * cs, atol=1e-14)


def _axis_problem(G, W=1, H=1, pos=(0.0, 0.0, 3.0)):
    from scenegen import look_at_c2w
    c2w = look_at_c2w(np.array(pos))[None].astype(np.float32)
    return Oracle(G, [], 2, 2, c2w, np.array([1.0], np.float32), W, H,
                  max_samples=4 * G)


def test_uniform_medium_closed_form():
    """Constant colour c and opacity sigma, no shells: H^ = c (1 - e^{-sigma L/h})
    for a chord of length L (the product over K equal steps telescopes)."""
    with open(os.path.join(GOLDEN, "closed_forms.json")) as f:
        cases = json.load(f)["uniform_medium_axis"]
    for case in cases:
        orc = _axis_problem(case["G"])
        x = np.zeros(orc.n_params).reshape(-1, 4)
        x[:, 0:3] = case["c"]
        x[:, 3] = case["sigma"]
        rgb = orc.render(x.reshape(-1))[0][0]
        assert np.allclose(rgb, case["expected_rgb"], rtol=1e-12, atol=1e-14)
    # random oblique rays: same closed form with the ray's own chord
    rng = np.random.default_rng(21)
    from scenegen import make_cameras
    c2w, focal = make_cameras(rng, 3, 9, 3.0, "sphere", 40.0)
    orc = Oracle(5, [], 2, 2, c2w, focal, 9, 9, max_samples=64)
    c = np.array([0.3, 0.6, 0.1]); sig = 0.4
    x = np.zeros(orc.n_params).reshape(-1, 4)
    x[:, 0:3] = c; x[:, 3] = sig
    rgb = orc.render(x.reshape(-1))[0]
    h = 2.0 / 5
    n = 0
    for ray in range(orc.n_rays):
        info = orc.ray_info(ray)
        if info["K"] == 0:
            assert np.all(rgb[ray] == 0)
            continue
        L = float(info["delta"]) * info["K"]
        assert np.allclose(rgb[ray], c * (1 - math.exp(-sig * L / h)), rtol=1e-12)
        n += 1
    assert n > 50


def test_single_sample_closed_form():
    """A chord shorter than one voxel side gives K = 1 and
    H^ = (1 - e^{-sigma delta/h}) c."""
    rng = np.random.default_rng(22)
    from scenegen import make_cameras
    c2w, focal = make_cameras(rng, 4, 40, 3.0, "sphere", 40.0)
    orc = Oracle(2, [], 2, 2, c2w, focal, 40, 40, max_samples=8)
    x = rng.uniform(0.1, 0.9, size=orc.n_params).reshape(-1, 4)
    x[:, 0:3] = [0.25, 0.5, 0.75]
    x[:, 3] = 1.3
    rgb = orc.render(x.reshape(-1))[0]
    found = 0
    for ray in range(orc.n_rays):
        info = orc.ray_info(ray)
        if info["K"] == 1:
            a = 1 - math.exp(-1.3 * info["delta"] / 1.0)
            assert np.allclose(rgb[ray], a * np.array([0.25, 0.5, 0.75]), rtol=1e-12)
            found += 1
    assert found > 0


def test_ray_geometry():
    """The binary32 ray: unit direction, entry/exit on the box surface,
    K delta = chord, delta <= h, samples inside the box."""
    rng = np.random.default_rng(23)
    from scenegen import make_cameras
    c2w, focal = make_cameras(rng, 3, 16, 3.0, "sphere", 40.0)
    G = 8
    orc = Oracle(G, [2.0, 4.0], 4, 8, c2w, focal, 16, 16, max_samples=64)
    h = 2.0 / G
    for ray in range(0, orc.n_rays, 7):
        info = orc.ray_info(ray)
        d = info["d"].astype(np.float64); o = info["o"].astype(np.float64)
        assert abs(np.linalg.norm(d) - 1) < 1e-6
        # camera looks at the origin: every ray points inwards
        assert float(o @ d) < 0
        # both shells enclose the box and lie beyond the camera or around it
        assert info["shell_hit"] == 0b11
        if info["K"] == 0:
            continue
        for t in (info["t_in"], info["t_out"]):
            p = o + t * d
            assert abs(np.max(np.abs(p)) - 1.0) < 1e-5
        L = info["t_out"] - info["t_in"]
        assert abs(info["K"] * info["delta"] - L) < 1e-5
        assert info["delta"] <= h * (1 + 1e-6)
        assert info["K"] == math.ceil(np.float32(L) / np.float32(h) - 1e-6) or \
            info["K"] == math.ceil(np.float32(L) / np.float32(h))


def _splitmix64(z):
    M = (1 << 64) - 1
    z = (z + 0x9E3779B97F4A7C15) & M
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
    return z ^ (z >> 31)


def test_splitmix64_published_sequence_and_jitter_draws():
    # published SplitMix64 outputs for state 0 (successive states 0, g, 2g)
    g = 0x9E3779B97F4A7C15
    M = (1 << 64) - 1
    seq = [_splitmix64((k * g) & M) for k in range(3)]
    assert seq == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    rng = np.random.default_rng(24)
    prob = tiny_problem(rng)
    orc = _orc(prob, jitter=True, seed=99, epoch=3)
    for ray, stream in [(0, 0), (5, 1), (17, 2), (31, 40)]:
        h = _splitmix64(_splitmix64(_splitmix64(99 + 3) + ray) + stream)
        assert orc.jitter_uniform(ray, stream) == (h >> 40) / 16777216.0


def test_jitter_moves_samples_within_half_a_step():
    rng = np.random.default_rng(25)
    prob = tiny_problem(rng, G=6, res=6)
    o0 = _orc(prob)
    o1 = _orc(prob, jitter=True, seed=5, epoch=1)
    x = prob["x"].astype(np.float64)
    a = o0.render(x)[0]
    b = o1.render(x)[0]
    assert not np.allclose(a, b)
    # the jittered estimate stays a valid composite: colours within [0, 1]
    assert np.all(b >= 0) and np.all(b <= 1)


def test_voxelised_ground_truth_has_zero_residual():
    from scenegen import make_scene
    sc = make_scene("small32", n_cams=2)
    orc = Oracle.from_scene(sc)
    tgt = orc.render(sc.x_gt)[0]
    r, F = orc.residual(sc.x_gt, tgt)
    assert F == 0.0
    _, g = orc.diag_grad(sc.x_gt, r)
    assert np.all(g == 0)


# --------------------------------------------------------------- Algorithm 2

def test_pcg_solves_explicit_spd_system():
    rng = np.random.default_rng(31)
    n = 12
    B = rng.normal(size=(20, n))
    A = B.T @ B + 0.1 * np.eye(n)
    b = rng.normal(size=n)
    d = np.diag(A).copy()
    res = pcg(lambda p: A @ p, b, lambda r: jacobi_apply(d, r), n, fixed=True)
    assert rel_l2(res.x, np.linalg.solve(A, b)) < 1e-9


def test_pcg_conjugacy_and_orthogonality():
    rng = np.random.default_rng(32)
    n = 10
    B = rng.normal(size=(15, n))
    A = B.T @ B + 0.05 * np.eye(n)
    b = rng.normal(size=n)
    d = np.diag(A).copy()
    ps, rs = [], []

    def rec(p):
        ps.append(p.copy())
        return A @ p
    res = pcg(rec, b, lambda r: jacobi_apply(d, r), 5, fixed=True)
    # successive search directions are A-conjugate
    for i in range(len(ps)):
        for j in range(i):
            assert abs(ps[i] @ A @ ps[j]) < 1e-9 * np.linalg.norm(ps[i]) * np.linalg.norm(A @ ps[j])
    # residual after k iterations is M^-1-orthogonal to the earlier ones:
    # recompute residuals r_k = b - A x_k from the directions
    x = np.zeros(n); r = b.copy(); rlist = [r.copy()]
    for a, p in zip(res.alphas, ps):
        x = x + a * p; r = r - a * (A @ p); rlist.append(r.copy())
    for i in range(len(rlist)):
        for j in range(i):
            zi = rlist[j] / d
            assert abs(rlist[i] @ zi) < 1e-9 * np.linalg.norm(rlist[i]) * np.linalg.norm(zi)


def test_pcg_exit_tests():
    A = np.diag([1.0, 2.0, 3.0, 4.0])
    b = np.ones(4)
    d = np.diag(A).copy()
    # Jacobi on a diagonal matrix solves in one iteration: R = 0 < eps
    res = pcg(lambda p: A @ p, b, lambda r: jacobi_apply(d, r), 10, fixed=False,
              eps_rel=1e-3)
    assert res.exit == "eps" and res.iters == 1
    assert np.allclose(res.x, b / np.diag(A))
    # identity preconditioner on an ill-conditioned system stalls
    A2 = np.diag([1.0, 1e-6])
    res = pcg(lambda p: A2 @ p, np.array([1e-3, 1.0]), lambda r: r.copy(), 10,
              fixed=False, eps_rel=1e-12, stall=0.85)
    assert res.exit == "stall"
    # the iterate at the stall is still returned (x_{k+1})
    assert res.iters >= 1 and np.any(res.x != 0)


def test_pcg_zero_diagonal_is_left_alone():
    z = jacobi_apply(np.array([0.0, 2.0]), np.array([5.0, 4.0]))
    assert z.tolist() == [0.0, 2.0]
    # entries at or below the binary32-motivated floor count as unobserved
    z = jacobi_apply(np.array([1e-31, 1e-30, 2e-30]), np.array([1.0, 1.0, 1.0]))
    assert z[0] == 0.0 and z[1] == 0.0 and abs(z[2] - 0.5e30) <= 1e-15 * 0.5e30


# --------------------------------------------------------------- Algorithm 3

def test_line_search_on_quadratics():
    for k in range(0, 8):
        g0 = 0.7 ** k
        gamma, mu, trace = line_search(lambda g: (g - g0) ** 2)
        assert abs(gamma - g0) < 1e-12, (k, gamma)
        assert mu == min(m for _, m in trace)
    # error rising from the first decimation: the full step is kept
    gamma, _, _ = line_search(lambda g: (g - 1.3) ** 2)
    assert gamma == 1.0
    # error falling all the way: the cap returns the last decimated step
    gamma, _, trace = line_search(lambda g: g, max_halvings=20)
    assert len(trace) == 21 and abs(gamma - 0.7 ** 20) < 1e-15


def test_projection():
    x = np.array([-0.5, 0.5, 1.5, -2.0, 0.2, 0.3, 0.4, 3.0])
    assert project(x).tolist() == [0.0, 0.5, 1.0, 0.0, 0.2, 0.3, 0.4, 3.0]


# --------------------------------------------------------- Gauss-Newton

def test_frozen_sigma_gn_step_equals_lstsq(tiny):
    """With sigma frozen the residual is linear in the colours, so one GN step
    with a converged PCG equals the minimum-norm least-squares solution."""
    orc, x, J = tiny
    rng = np.random.default_rng(41)
    target = rng.uniform(0, 1, size=3 * orc.n_rays)
    r, F = orc.residual(x, target)
    mask = np.zeros(x.shape[0]); mask.reshape(-1, 4)[:, 0:3] = 1.0
    diag, grad = orc.diag_grad(x, r)
    b = -grad * mask
    Jc = J * mask[None, :]
    obs = np.sum(Jc * Jc, axis=0) > 0
    nobs = int(obs.sum())
    res = pcg(lambda p: mask * orc.apply_A(x, mask * p), b,
              lambda v: jacobi_apply(diag * mask, v), 3 * nobs, fixed=False,
              eps_rel=1e-12, stall=np.inf)
    ref = np.linalg.lstsq(Jc[:, obs], -r, rcond=None)[0]
    # the fitted change J Delta is unique even when the colours are not
    assert rel_l2(Jc[:, obs] @ res.x[obs], Jc[:, obs] @ ref) < 1e-6
    # Delta solves the normal equations
    assert rel_l2(Jc.T @ (Jc @ res.x), -Jc.T @ r) < 1e-6
    gamma, mu, _ = line_search(lambda g: orc.error(x + g * res.x, target))
    assert gamma == 1.0
    assert mu < F


def test_gn_decreases_objective_on_small_scene():
    from scenegen import make_scene
    sc = make_scene("small32", n_cams=3, G=12)
    orc = Oracle.from_scene(sc)
    target = orc.render(sc.x_gt)[0].ravel()
    x = sc.x0.astype(np.float64)
    Fs = [orc.error(x, target)]
    for _ in range(3):
        st = gn_step(orc, x, target, pcg_iters=8)
        assert st.accepted
        assert st.F_after < st.F_before
        x = st.x
        Fs.append(st.F_after)
    assert Fs[-1] < 0.5 * Fs[0]


def test_cg_sensitivity_of_the_oracle_itself():
    """Why parameters are compared after few PCG iterations on the first
    system: on the 32^3 workload's first Gauss-Newton system (the constant
    start), relative noise of 1e-6 on A p (the size of FP32 rounding) moves
    the oracle's own 20-iteration Delta by more than 1e-4, while the
    3-iteration Delta and the fitted change J Delta stay within 1e-5."""
    from scenegen import make_scene
    sc = make_scene("small32")
    orc = Oracle.from_scene(sc)
    target = orc.render(sc.x_gt)[0].ravel()
    x = sc.x0.astype(np.float64)
    r, _ = orc.residual(x, target)
    d, g = orc.diag_grad(x, r)
    M = lambda v: jacobi_apply(d, v)
    rng = np.random.default_rng(0)

    def noisy(p):
        a = orc.apply_A(x, p)
        return a * (1.0 + 1e-6 * rng.normal(size=a.shape))
    for k, bound_dx, bound_jdx in ((3, 1e-5, 1e-5), (20, None, None)):
        ref = pcg(lambda p: orc.apply_A(x, p), -g, M, k)
        per = pcg(noisy, -g, M, k)
        dx = rel_l2(per.x, ref.x)
        if bound_dx is not None:
            assert dx < bound_dx, (k, dx)
            assert rel_l2(orc.jvp(x, per.x), orc.jvp(x, ref.x)) < bound_jdx
        else:
            assert dx > 1e-4, (k, dx)


def test_cg_sensitivity_after_the_first_step():
    """What 20 PCG iterations determine on the 32^3 workload, the bounds the
    GPU's 5 x 20 schedule is held to: under 1e-6 relative noise on A p,
    * the first step (from the constant start) moves Delta by ~2e-2 and
      F after the line search and the rendered image by up to ~4e-3, so
      that step is held to 1e-2 on F and the image;
    * from the second step on, Delta moves by less than 1e-4 and F after the
      step and the image by less than 1e-4, so those steps are held to the
      parameter bar 1e-4 and to 1e-4 on F and the image."""
    from scenegen import make_scene
    sc = make_scene("small32")
    orc = Oracle.from_scene(sc)
    target = orc.render(sc.x_gt)[0].ravel()
    x = sc.x0.astype(np.float64)
    rng = np.random.default_rng(1)
    for step in range(3):
        r, _ = orc.residual(x, target)
        d, g = orc.diag_grad(x, r)
        M = lambda v: jacobi_apply(d, v)

        def noisy(p):
            a = orc.apply_A(x, p)
            return a * (1.0 + 1e-6 * rng.normal(size=a.shape))
        ref = pcg(lambda p: orc.apply_A(x, p), -g, M, 20)
        per = pcg(noisy, -g, M, 20)

        def after(D):
            gam, mu, _ = line_search(lambda gg: orc.error(project(x + gg * D), target))
            return mu, project(x + gam * D)
        F1, x1 = after(ref.x)
        F2, x2 = after(per.x)
        dF = abs(F2 - F1) / F1
        dimg = rel_l2(orc.render(x2)[0], orc.render(x1)[0])
        dx = rel_l2(per.x, ref.x)
        if step == 0:
            assert dx > 1e-3 and dF < 1e-2 and dimg < 1e-2, (step, dx, dF, dimg)
        else:
            assert dx < 1e-4 and dF < 1e-4 and dimg < 1e-4, (step, dx, dF, dimg)
        x = x1


# ---------------------------------------------------------------- hierarchy

def test_upsample_constant_and_sigma_rescale():
    """Section "Hierarchical formulation": a constant field stays constant on
    the doubled grid; sigma is per voxel side, so it halves, and the optical
    depth through the volume is unchanged."""
    from oracle.hierarchy import upsample
    G, S, He, We = 5, 2, 3, 6
    x = np.empty(4 * (G ** 3 + S * He * We))
    x.reshape(-1, 4)[:] = (0.2, 0.5, 0.7, 1.6)
    y = upsample(x, G, S, He, We).reshape(-1, 4)
    nv2 = (2 * G) ** 3
    assert y.shape[0] == nv2 + S * 4 * He * We
    assert np.allclose(y[:nv2], (0.2, 0.5, 0.7, 0.8), atol=1e-15)
    assert np.allclose(y[nv2:], (0.2, 0.5, 0.7, 1.6), atol=1e-15)


def test_upsample_preserves_optical_depth_through_the_ray_march():
    """The halved sigma keeps the optical depth: the oracle's ray march (Eq. 3
    with K = ceil(L / h) steps of delta-bar = delta / h) gives the same
    grid-exit transmittance on both levels for a uniform medium."""
    from oracle import Oracle
    from oracle.hierarchy import upsample
    from scenegen import make_cameras
    rng = np.random.default_rng(3)
    c2w, focal = make_cameras(rng, 3, 9, 3.2, "sphere", 40.0)
    G = 6
    x = np.empty(4 * G ** 3)
    x.reshape(-1, 4)[:] = (0.3, 0.6, 0.9, 0.35)
    T1 = Oracle(G, (), 2, 2, c2w, focal, 9, 9).render(x)[1]
    T2 = Oracle(2 * G, (), 2, 2, c2w, focal, 9, 9).render(upsample(x, G, 0, 2, 2))[1]
    hit = T1 < 1.0
    assert hit.sum() > 50
    # the ray set-up (t_in, t_out, delta) is binary32 on both levels, so T
    # agrees to binary32 geometry rounding; a sigma not halved would give
    # T2 = T1^2 (here T1 ~ 0.2-0.5)
    assert np.abs(T1 - T2).max() < 1e-6


def test_upsample_linear_field_interior():
    """Trilinear interpolation reproduces a linear field exactly wherever the
    fine centre lies inside the coarse centres' hull (u in [0, G-1]); at the
    boundary the clamp holds the edge value.  Catches half-voxel offset,
    axis order and weight errors."""
    from oracle.hierarchy import upsample_grid
    G = 6
    k, j, i = np.meshgrid(np.arange(G), np.arange(G), np.arange(G), indexing="ij")
    grid = np.stack([1 + 0.5 * i, 2 - 0.25 * j, 0.3 * k, 0.1 * i + 0.2 * j + 0.4 * k], -1)
    fine = upsample_grid(grid)
    u = (np.arange(2 * G) + 0.5) / 2 - 0.5
    uz, uy, ux = np.meshgrid(u, u, u, indexing="ij")
    inside = (uz >= 0) & (uz <= G - 1) & (uy >= 0) & (uy <= G - 1) & (ux >= 0) & (ux <= G - 1)
    ref = np.stack([1 + 0.5 * ux, 2 - 0.25 * uy, 0.3 * uz, 0.5 * (0.1 * ux + 0.2 * uy + 0.4 * uz)], -1)
    assert np.abs(fine[inside] - ref[inside]).max() < 1e-13
    # boundary: fine centre 0 sits at u = -1/4 and takes the clamped edge value
    assert np.isclose(fine[0, 0, 0, 0], grid[0, 0, 0, 0])
    assert np.isclose(fine[-1, -1, -1, 2], grid[-1, -1, -1, 2])


def test_upsample_shell_wrap_by_hand():
    """Environment map: fine column 0 lies a quarter texel west of coarse
    column 0 and wraps: 1/4 of the last column plus 3/4 of the first (and
    the last fine column 3/4 of the last plus 1/4 of the first); fine row 0
    is clamped to coarse row 0."""
    from oracle.hierarchy import upsample_shell
    He, We = 2, 4
    tex = np.zeros((He, We, 4))
    tex[:, :, 0] = np.arange(We)[None, :] * 10.0      # varies along phi only
    tex[:, :, 1] = np.arange(He)[:, None] * 1.0       # varies along theta only
    tex[:, :, 3] = 2.5
    f = upsample_shell(tex)
    assert np.isclose(f[0, 0, 0], 0.25 * 30.0 + 0.75 * 0.0)
    assert np.isclose(f[0, 1, 0], 0.75 * 0.0 + 0.25 * 10.0)
    assert np.isclose(f[0, 7, 0], 0.75 * 30.0 + 0.25 * 0.0)
    assert np.isclose(f[0, 0, 1], 0.0) and np.isclose(f[3, 0, 1], 1.0)
    assert np.isclose(f[1, 0, 1], 0.25) and np.isclose(f[2, 0, 1], 0.75)
    assert np.allclose(f[..., 3], 2.5)


def test_render_threshold_closed_form():
    """Section "Rendering": uniform medium (colour c, opacity sigma) inside a
    constant shell (colour s, opacity sigma_s).  A ray with chord L has
    volume opacity a = 1 - e^{-sigma L/h}; at or above the threshold it
    renders c a + (1 - a) s (1 - e^{-sigma_s}), below it the shell alone,
    s (1 - e^{-sigma_s}); a threshold of 0 is the plain render."""
    from scenegen import make_cameras
    rng = np.random.default_rng(23)
    c2w, focal = make_cameras(rng, 3, 11, 3.0, "sphere", 40.0)
    G = 5
    orc = Oracle(G, [2.5], 2, 4, c2w, focal, 11, 11, max_samples=64)
    c = np.array([0.9, 0.2, 0.4]); s_rgb = np.array([0.1, 0.7, 0.3]); sig, sig_s = 0.12, 0.8
    x = np.zeros(orc.n_params).reshape(-1, 4)
    x[:G ** 3, 0:3] = c; x[:G ** 3, 3] = sig
    x[G ** 3:, 0:3] = s_rgb; x[G ** 3:, 3] = sig_s
    x = x.reshape(-1)
    h = 2.0 / G
    shell = s_rgb * (1 - math.exp(-sig_s))
    assert np.array_equal(orc.render_threshold(x, 0.0)[0], orc.render(x)[0])
    thr = 0.5
    rgb, te = orc.render_threshold(x, thr)
    n_cut = n_kept = 0
    for ray in range(orc.n_rays):
        info = orc.ray_info(ray)
        L = float(info["delta"]) * info["K"]
        a = 1 - math.exp(-sig * L / h)
        assert np.isclose(1 - te[ray], a, rtol=1e-12, atol=1e-15)
        if a < thr:
            assert np.allclose(rgb[ray], shell, rtol=1e-12)
            n_cut += info["K"] > 0
        else:
            assert np.allclose(rgb[ray], c * a + (1 - a) * shell, rtol=1e-12)
            n_kept += 1
    assert n_cut > 10 and n_kept > 10


# ------------------------------------------------------ auxiliary residual

AUX_LAMBDA = 0.1


def _aux_residual_fd_model(orc, x):
    """The residual vector with the auxiliary term built from the forward
    model alone: per ray (H^_0, H^_1, H^_2, L), L = lambda (1 - 4 (T^ - 1/2)^2)
    with T^ the render's grid-exit transmittance (Section "Auxiliary terms")."""
    rgb, te, _ = orc.render(x)
    L = AUX_LAMBDA * (1.0 - 4.0 * (te - 0.5) ** 2)
    return np.concatenate([rgb, L[:, None]], axis=1).ravel()


@pytest.fixture(scope="module")
def tiny_aux():
    rng = np.random.default_rng(7)
    prob = tiny_problem(rng)
    orc = _orc(prob, aux=True, aux_lambda=AUX_LAMBDA)
    x = prob["x"].astype(np.float64)
    n, eps = x.shape[0], 1e-6
    J = np.zeros((4 * orc.n_rays, n))
    for j in range(n):
        xp = x.copy(); xp[j] += eps
        xm = x.copy(); xm[j] -= eps
        J[:, j] = (_aux_residual_fd_model(orc, xp) - _aux_residual_fd_model(orc, xm)) / (2 * eps)
    return orc, x, J


def test_aux_derivatives_match_finite_differences(tiny_aux):
    """J p, J^T v, diag(J^T J) and J^T r with the auxiliary row, against the
    dense FD Jacobian of the forward model (the aux row has sigma entries
    only; colours and shells do not move the grid-exit transmittance)."""
    orc, x, J = tiny_aux
    n, m = x.shape[0], J.shape[0]
    assert np.abs(J[3::4]).max() > 1e-3
    Jalg = np.stack([orc.jvp(x, np.eye(n)[j]) for j in range(n)], axis=1)
    assert np.abs(Jalg - J).max() <= 1e-7 * np.abs(J).max() + 1e-9
    for i in range(3, m, 4):
        assert np.abs(orc.vjp(x, np.eye(m)[i]) - J[i]).max() <= 1e-7 * np.abs(J).max() + 1e-9
    d, _ = orc.diag_grad(x)
    assert rel_l2(d, np.sum(J * J, axis=0)) < 1e-7
    rng = np.random.default_rng(4)
    target = rng.uniform(0, 1, size=3 * orc.n_rays)
    r, F = orc.residual(x, target)
    rgb, te, _ = orc.render(x)
    assert np.allclose(r.reshape(-1, 4)[:, :3], rgb - target.reshape(-1, 3), atol=1e-14)
    assert np.allclose(r.reshape(-1, 4)[:, 3], AUX_LAMBDA * (1 - 4 * (te - 0.5) ** 2), atol=1e-14)
    assert abs(F - 0.5 * float(r @ r)) < 1e-12
    _, g = orc.diag_grad(x, r)
    assert rel_l2(g, J.T @ r) < 1e-7
    p = rng.normal(size=n)
    v = rng.normal(size=m)
    assert abs(float(orc.jvp(x, p) @ v) - float(p @ orc.vjp(x, v))) <= 1e-12 * max(abs(float(orc.jvp(x, p) @ v)), 1.0)


def test_aux_closed_form_uniform_medium():
    """Uniform medium (opacity sigma, no shells): T^ = e^{-sigma L/h} for a
    chord L, so the auxiliary residual is lambda (1 - 4 (e^{-sigma L/h} - 1/2)^2):
    0 for empty and opaque rays, lambda at T^ = 1/2."""
    from scenegen import make_cameras
    rng = np.random.default_rng(24)
    c2w, focal = make_cameras(rng, 2, 9, 3.0, "sphere", 40.0)
    G = 5
    orc = Oracle(G, [], 2, 2, c2w, focal, 9, 9, max_samples=64, aux=True, aux_lambda=AUX_LAMBDA)
    sig = 0.3
    x = np.zeros(orc.n_params).reshape(-1, 4)
    x[:, 0:3] = 0.5; x[:, 3] = sig
    r, _ = orc.residual(x.reshape(-1), np.zeros(3 * orc.n_rays))
    h = 2.0 / G
    for ray in range(orc.n_rays):
        info = orc.ray_info(ray)
        T = math.exp(-sig * float(info["delta"]) * info["K"] / h)
        assert math.isclose(r[4 * ray + 3], AUX_LAMBDA * (1 - 4 * (T - 0.5) ** 2), rel_tol=1e-12,
                            abs_tol=1e-15)


# ---------------------------------------------------------------- Adam

def test_adam_update_closed_forms():
    """Adam with its bias corrections: the first step moves every parameter by
    lr g / (|g| + eps) (m_hat = g, v_hat = g^2), and under a constant gradient
    every later step does too (m_hat and v_hat stay exactly g and g^2); a
    wrong correction power or moment update breaks either."""
    from oracle import adam_update
    g = np.array([3.0, -0.5, 1e-3, 0.0, -2e-6])
    x = np.zeros(5)
    m = np.zeros(5)
    v = np.zeros(5)
    lr, eps = 0.05, 1e-8
    for t in range(1, 8):
        x_new, m, v = adam_update(x, g, m, v, t, lr=lr, eps=eps)
        assert np.allclose(x_new - x, -lr * g / (np.abs(g) + eps), rtol=1e-12, atol=1e-15), t
        x = x_new
    # a changing gradient: the bias-corrected first moment is the weighted mean
    m = np.zeros(1); v = np.zeros(1); x = np.zeros(1)
    g1, g2, b1, b2 = 2.0, -1.0, 0.9, 0.999
    x, m, v = adam_update(x, np.array([g1]), m, v, 1, lr=1.0, beta1=b1, beta2=b2, eps=0.0)
    x2, m, v = adam_update(x, np.array([g2]), m, v, 2, lr=1.0, beta1=b1, beta2=b2, eps=0.0)
    mh = (b1 * (1 - b1) * g1 + (1 - b1) * g2) / (1 - b1 ** 2)
    vh = (b2 * (1 - b2) * g1 ** 2 + (1 - b2) * g2 ** 2) / (1 - b2 ** 2)
    assert np.allclose(x2 - x, -mh / np.sqrt(vh), rtol=1e-12)


def test_adam_step_uses_the_gradient_of_F(tiny):
    """adam_step's first step is -lr g / (|g| + eps) (before projection), with
    g = J^T r from the finite-difference Jacobian."""
    from oracle import adam_step
    orc, x, J = tiny
    rng = np.random.default_rng(31)
    target = rng.uniform(0, 1, size=3 * orc.n_rays)
    n = x.shape[0]
    xn, m, v, F = adam_step(orc, x, target, np.zeros(n), np.zeros(n), 1, lr=0.01,
                            do_project=False)
    r = orc.render(x)[0].ravel() - target
    g = J.T @ r
    assert abs(F - 0.5 * float(r @ r)) < 1e-12
    big = np.abs(g) > 1e-4
    assert big.sum() > n // 2
    assert np.allclose((xn - x)[big], -0.01 * g[big] / (np.abs(g[big]) + 1e-8), rtol=1e-6)


def test_upsample_cube_faces_by_hand():
    """Cube-map level change: each face on its own.  A ramp a + b c along a
    face's columns (a different a on every face, so faces jump) upsamples to
    a + b (c'/2 - 1/4) at the interior fine columns c' and is clamped to the
    face's edge texels at c' = 0 and c' = 2F - 1; nothing leaks across a face
    boundary (an equirectangular treatment would blend neighbouring faces)."""
    from oracle.hierarchy import upsample_cube_shell
    F = 4
    tex = np.zeros((F, 6 * F, 4))
    for f in range(6):
        for c in range(F):
            tex[:, f * F + c, 0] = 10.0 * f + 0.5 * c
    tex[..., 1] = 3.0
    out = upsample_cube_shell(tex)
    assert out.shape == (2 * F, 12 * F, 4)
    assert np.allclose(out[..., 1], 3.0)
    for f in range(6):
        for cp in range(2 * F):
            u = min(max(cp / 2.0 - 0.25, 0.0), F - 1.0)
            assert np.allclose(out[:, 2 * f * F + cp, 0], 10.0 * f + 0.5 * u), (f, cp)

"""The first-order comparator (Adam on the same objective and gradient g =
J^T r) on the CUDA path against the oracle's adam_step, through the C ABI.

Each GPU step is compared with one oracle step from the GPU's own state
(x, m, v): F at the start, the moments, and x after the step.  Adam divides
each gradient component by its own running magnitude, so the first steps
move a parameter by about lr sign(g_j): where FP32 rounding can flip that
sign -- |g_j| below 1e-4 of the magnitude of the terms it sums -- the step
is not determined, and such parameters are only checked to have moved by at
most lr (plus its rounding)."""
import numpy as np
import pytest

from conftest import rel_l2
from gpu_common import TOL_FP32, cuda_tensor, host, mid_state

pytestmark = pytest.mark.gpu


def test_adam_steps_against_oracle():
    import torch
    from oracle import Oracle, adam_step
    from paper_2112_05598_gb300 import Context
    from scenegen import make_scene
    sc = make_scene("small32")
    orc = Oracle.from_scene(sc)
    target = orc.render(sc.x_gt)[0].astype(np.float32).ravel()
    ctx = Context.from_scene(sc)
    lr = 0.01
    x = cuda_tensor(mid_state(np.random.default_rng(70), sc))
    m = torch.zeros_like(x)
    v = torch.zeros_like(x)
    F = torch.zeros(1, dtype=torch.float64, device="cuda")
    td = cuda_tensor(target)
    for t in range(1, 6):
        xb, mb, vb = host(x), host(m), host(v)
        ctx.adam_step(x, td, m, v, t, lr=lr, F_out=F)
        xo, mo, vo, Fo = adam_step(orc, xb, target, mb, vb, t, lr=lr)
        assert abs(host(F)[0] - Fo) <= TOL_FP32 * Fo
        r, _ = orc.residual(xb, target)
        g, gmag = orc.vjp(xb, r, mag=True)
        det = np.abs(g) > 1e-4 * gmag
        xg = host(x)
        err = rel_l2(xg[det], xo[det])
        print(f"[adam] step {t}: F {Fo:.6g}, x rel L2 {err:.3e} over {det.sum()} determined "
              f"of {det.size}; m rel L2 {rel_l2(host(m), mo):.3e}")
        assert err < 1e-5, (t, err)
        assert rel_l2(host(m), mo) < 1e-4
        assert np.all(np.abs(xg[~det] - xb[~det]) <= lr * (1 + 1e-4))
        assert det.sum() > 0.5 * det.size


def test_adam_rejects_bad_arguments():
    import torch
    from paper_2112_05598_gb300 import Context, PerfError
    from scenegen import make_scene
    sc = make_scene("small32")
    ctx = Context.from_scene(sc)
    x = cuda_tensor(sc.x0.copy())
    m = torch.zeros_like(x)
    with pytest.raises(PerfError):
        ctx.adam_step(x, x, m, m, 0)
    with pytest.raises(PerfError):
        ctx.adam_step(x, x, m, m, 1, lr=-1.0)

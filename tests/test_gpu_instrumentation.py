"""Instrumentation of the J^T scatter: the count of its vector-atomic lane
operations and the atomic-throughput microbenchmark that A p is measured
against."""
import numpy as np
import pytest

from gpu_common import cuda_tensor, empty, mid_state

pytestmark = pytest.mark.gpu


def _step(ctx, x, target, counter=None):
    import torch
    ctx.set_atomic_counter(counter)
    st = ctx.gn_solve(x.clone(), target, 1)[0]
    ctx.set_atomic_counter(None)
    torch.cuda.synchronize()
    return st


def test_atomic_counter_counts_the_scatter_without_changing_results():
    """Both A p paths flush the same (ray, voxel) pairs, so they count the
    same lane operations; counting leaves the Gauss-Newton step unchanged."""
    import torch
    from paper_2112_05598_gb300 import Context
    from scenegen import make_scene
    sc = make_scene("small32")
    ctx = Context.from_scene(sc, pcg_iters=2, pcg_fixed=1)
    x = cuda_tensor(mid_state(np.random.default_rng(3), sc))
    target = empty(3 * ctx.n_rays)
    ctx.render(cuda_tensor(sc.x_gt), target)
    counts = {}
    for budget in (-1, 0):
        ctx.set_coef_budget(budget)
        plain = _step(ctx, x, target)
        c = torch.zeros(1, dtype=torch.int64, device="cuda")
        counted = _step(ctx, x, target, c)
        assert ctx.coef_info()["used"] == (budget != 0)
        # atomics make A p's summation order vary between runs: F to rounding
        assert counted["gamma"] == plain["gamma"]
        assert abs(counted["F_after"] - plain["F_after"]) <= 1e-5 * plain["F_after"]
        counts[budget] = int(c.item())
    ctx.set_coef_budget(-1)
    # about 3-5 lane operations per march sample, two A p per step
    samples = ctx.sample_count()
    assert 2 * samples < counts[-1] < 2 * 8 * samples
    assert abs(counts[-1] - counts[0]) <= 1e-3 * counts[-1], counts


def test_atomic_peak_microbenchmark():
    from paper_2112_05598_gb300 import measure_atomic_peak
    peak = measure_atomic_peak()
    assert 1e10 < peak < 1e13, peak

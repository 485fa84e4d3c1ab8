"""The fixed-iteration PCG loop of perf_gn_solve replayed from a CUDA graph
(perf_set_pcg_graph) on the CUDA path, against the oracle through the C ABI:
every Gauss-Newton step matches the oracle's step whether the loop is
replayed or launched kernel by kernel, and the graph is captured again when
what it captured changes (the iteration count, the coefficient store, the
preconditioner, the brick order)."""
import numpy as np
import pytest

from conftest import rel_l2
from gpu_common import TOL_FP32, TOL_GN, assert_params, cuda_tensor, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def s32():
    from oracle import Oracle
    from scenegen import make_scene
    sc = make_scene("small32")
    orc = Oracle.from_scene(sc)
    target = orc.render(sc.x_gt)[0].astype(np.float32).ravel()
    return sc, orc, target


def _check_step(ctx, orc, xd, target, pcg, what):
    from oracle import gn_step
    xb = host(xd)
    st = ctx.gn_solve(xd, cuda_tensor(target), 1)[0]
    ref = gn_step(orc, xb, target, pcg)
    assert st["pcg_iters"] == pcg
    assert st["accepted"] == ref.accepted
    assert abs(st["F_before"] - ref.F_before) <= TOL_FP32 * ref.F_before
    if abs(st["gamma"] - ref.gamma) > 1e-9:
        return cuda_tensor(ref.x.astype(np.float32)), st
    assert_params(host(xd), ref.x, ref.diag, TOL_GN, what=what)
    return xd, st


def test_graph_recaptured_when_the_step_changes(s32):
    sc, orc, target = s32
    from paper_2112_05598_gb300 import Context
    ctx = Context.from_scene(sc, pcg_iters=3, pcg_fixed=1)
    xd = cuda_tensor(sc.x0.copy())
    xd, _ = _check_step(ctx, orc, xd, target, 3, "graph, 3 iterations")
    xd, _ = _check_step(ctx, orc, xd, target, 3, "graph replayed, 3 iterations")
    ctx.set_options(pcg_iters=2)
    xd, _ = _check_step(ctx, orc, xd, target, 2, "graph recaptured, 2 iterations")
    ctx.set_coef_budget(0)          # the recomputing A p (paired records)
    xd, _ = _check_step(ctx, orc, xd, target, 2, "graph, recomputing A p")
    ctx.set_coef_budget(-1)
    ctx.set_brick(4)
    xd, _ = _check_step(ctx, orc, xd, target, 2, "graph, 4^3 bricks")


def test_graph_equals_host_launched_loop(s32):
    """Three steps of 3 PCG iterations with the loop replayed and launched
    from the host: the same objective after each step and the same
    parameters, to the bars of the oracle comparisons (3 iterations determine
    the step; at 20, CG amplifies the rounding of the atomic sums, as pinned
    on the oracle itself).  The device time per step of the 32^3
    configuration (20 iterations) is printed for both."""
    sc, orc, target = s32
    from paper_2112_05598_gb300 import Context
    out = {}
    for graph in (True, False):
        ctx = Context.from_scene(sc, pcg_iters=3, pcg_fixed=1)
        ctx.set_pcg_graph(graph)
        xd = cuda_tensor(sc.x0.copy())
        st = ctx.gn_solve(xd, cuda_tensor(target), 3)
        out[graph] = (host(xd), [s["F_after"] for s in st])
        ctx.set_options(pcg_iters=20)
        x2 = cuda_tensor(sc.x0.copy())
        ms = [s["ms"] for s in ctx.gn_solve(x2, cuda_tensor(target), 5)]
        print(f"[graph] replayed={graph}: device ms per 20-iteration step {np.median(ms):.3f}")
    for a, b in zip(out[True][1], out[False][1]):
        assert abs(a - b) <= TOL_FP32 * b
    assert rel_l2(out[True][0], out[False][0]) < TOL_GN

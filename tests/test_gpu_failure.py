"""Failure detection, exercised without faulting, trapping or hanging the GPU.

* A non-finite objective (a NaN planted from the host in the targets or in
  the parameters): perf_gn_solve returns PERF_ERR_NONFINITE, leaves x
  unchanged, and the same context solves the next, clean system.
* A bounded device-side wait that runs out: the tcgen05 convolution of the
  learned preconditioner is given a test limit of zero polling rounds for
  each CTA's first TMA wait.  Every such wait gives up at once; the kernel
  raises its flag, waits with the normal limit for the loads it has in
  flight, frees its tensor memory and returns.  The host reads the flag
  (perf_lpc_conv_status, PERF_ERR_TIMEOUT from the training entry point),
  and with the normal limit restored the same network gives results equal
  to a run before the timeout."""
import numpy as np
import pytest

from gpu_common import cuda_tensor, host

pytestmark = pytest.mark.gpu


def _ctx_and_target():
    from oracle import Oracle
    from paper_2112_05598_gb300 import Context
    from scenegen import make_scene
    sc = make_scene("small32")
    target = Oracle.from_scene(sc).render(sc.x_gt)[0].astype(np.float32).ravel()
    ctx = Context.from_scene(sc, pcg_iters=3, pcg_fixed=1)
    return sc, ctx, target


def test_nan_target_is_reported_and_x_is_kept():
    from paper_2112_05598_gb300 import PerfError
    sc, ctx, target = _ctx_and_target()
    bad = target.copy()
    bad[3 * 2080 + 1] = np.nan
    xd = cuda_tensor(sc.x0.copy())
    before = host(xd)
    with pytest.raises(PerfError) as e:
        ctx.gn_solve(xd, cuda_tensor(bad), 1)
    assert e.value.status == 3          # PERF_ERR_NONFINITE
    assert np.array_equal(host(xd), before)
    # the context stays usable: the clean system takes a normal, accepted step
    st = ctx.gn_solve(xd, cuda_tensor(target), 1)[0]
    assert st["accepted"] and np.isfinite(st["F_after"]) and st["F_after"] < st["F_before"]


def test_nan_parameter_is_reported_and_x_is_kept():
    from paper_2112_05598_gb300 import PerfError
    sc, ctx, target = _ctx_and_target()
    x = sc.x0.copy()
    G = sc.G
    v = (G // 2 * G + G // 2) * G + G // 2          # the centre voxel: every camera sees it
    x[4 * v + 3] = np.nan
    xd = cuda_tensor(x)
    with pytest.raises(PerfError) as e:
        ctx.gn_solve(xd, cuda_tensor(target), 1)
    assert e.value.status == 3
    assert np.array_equal(host(xd), x.astype(np.float64), equal_nan=True)
    st = ctx.gn_solve(cuda_tensor(sc.x0.copy()), cuda_tensor(target), 1)[0]
    assert st["accepted"]


def test_convolution_wait_timeout_is_reported_and_recovers():
    import torch
    from paper_2112_05598_gb300 import LPC, PerfError, _binding as B
    G = 20
    rng = np.random.default_rng(77)
    net = LPC(seed=5)
    feat = torch.from_numpy(rng.normal(size=(G ** 3, 16)).astype(np.float32)).to(torch.bfloat16).cuda()
    ref = torch.empty(16 * G ** 3, dtype=torch.bfloat16, device="cuda")
    net.head_outputs(G, feat, ref)
    assert B.conv_status() == 0
    xi = torch.from_numpy(rng.normal(size=4 * G ** 3).astype(np.float32)).cuda()
    ahat = torch.from_numpy(rng.normal(size=4 * G ** 3).astype(np.float32)).cuda()
    B.set_conv_wait_limit_for_test(0)
    try:
        out = torch.zeros(16 * G ** 3, dtype=torch.bfloat16, device="cuda")
        net.head_outputs(G, feat, out)
        assert B.conv_status() == 1
        with pytest.raises(PerfError) as e:
            net.loss_grad(G, feat, ahat, xi)
        assert e.value.status == 4      # PERF_ERR_TIMEOUT
        assert B.conv_status() == 0     # the entry point read and cleared the flag
    finally:
        B.set_conv_wait_limit_for_test(1 << 20)
    out2 = torch.zeros(16 * G ** 3, dtype=torch.bfloat16, device="cuda")
    net.head_outputs(G, feat, out2)
    assert B.conv_status() == 0
    assert torch.equal(out2, ref)
    loss = net.loss_grad(G, feat, ahat, xi)
    assert np.isfinite(loss)

"""perf_residual_noalloc against perf_residual.

The no-allocation entry point serves callers that cannot allocate device
memory when they need a residual (a device-memory budget fixed at start-up,
an engine whose own allocator owns all device memory, a latency-critical loop
that must avoid cudaMalloc).  It keeps its camera table in one static device
array shared by every call, so this test makes two calls in a row with
different cameras and parameters and checks each against the context-based
entry point.  The file name sorts last so that a run stopping at the first
failure has run every other test before this one."""
import numpy as np
import pytest

from conftest import rel_l2
from gpu_common import TOL_FP32, cuda_tensor, empty, host

pytestmark = pytest.mark.gpu


def test_noalloc_matches_context_residual_twice():
    import torch
    from paper_2112_05598_gb300 import Context
    from paper_2112_05598_gb300._binding import residual_noalloc
    from scenegen import make_scene
    sc = make_scene("small32")
    rng = np.random.default_rng(2024)
    target = cuda_tensor(rng.uniform(0, 1, size=3 * sc.n_rays).astype(np.float32))
    calls = [(sc.c2w, sc.x0), (sc.c2w[::-1].copy(), (0.5 * sc.x0 + 0.5 * sc.x_gt))]
    for c2w, x in calls:
        xd = cuda_tensor(np.ascontiguousarray(x, dtype=np.float32))
        ctx = Context(sc.G, sc.radii, sc.env_h, sc.env_w, c2w, sc.focal, sc.width, sc.height,
                      max_samples=sc.cfg.max_samples)
        r_ref = empty(3 * ctx.n_rays)
        F_ref = torch.zeros(1, dtype=torch.float64, device="cuda")
        ctx.residual(xd, target, r_ref, F_ref)
        r = empty(3 * ctx.n_rays) + 7.0
        F = torch.full((1,), 123.0, dtype=torch.float64, device="cuda")
        residual_noalloc(sc.G, sc.radii, sc.env_h, sc.env_w, c2w, sc.focal, sc.width, sc.height,
                         xd, target, r, F, options=ctx.options)
        assert rel_l2(host(r), host(r_ref)) < TOL_FP32
        assert abs(host(F)[0] - host(F_ref)[0]) <= TOL_FP32 * host(F_ref)[0]
        ctx.close()

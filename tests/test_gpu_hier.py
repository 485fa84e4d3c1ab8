"""Level change of the hierarchical formulation on the GPU (perf_upsample)
against the FP64 oracle: grids of odd and even size, several shells, map
widths that wrap; the weights are exact binary fractions, so the only
difference is FP32 accumulation."""
import numpy as np
import pytest

from conftest import rel_l2
from gpu_common import cuda_tensor, empty, host

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("G,S,He,We,kind", [(2, 0, 2, 2, 0), (5, 2, 3, 7, 0), (16, 3, 8, 16, 0),
                                            (33, 1, 5, 9, 0), (6, 2, 2, 12, 1), (9, 3, 5, 30, 1)])
def test_upsample_parity(G, S, He, We, kind):
    """kind 1: cube-map shells (faces of He x He texels)."""
    from oracle.hierarchy import upsample as ref_upsample
    from paper_2112_05598_gb300 import upsample
    rng = np.random.default_rng(G * 100 + S)
    n = 4 * (G ** 3 + S * He * We)
    x = rng.uniform(0, 2, size=n).astype(np.float32)
    y = empty(4 * (8 * G ** 3 + 4 * S * He * We))
    upsample(cuda_tensor(x), G, S, He, We, y, env_kind=kind)
    ref = ref_upsample(x.astype(np.float64), G, S, He, We, env_kind=kind)
    got = host(y)
    assert got.shape == ref.shape
    assert np.abs(got - ref).max() <= 1e-6 * np.abs(ref).max()


def test_upsample_rejects_overlap_and_bad_sizes():
    from paper_2112_05598_gb300 import PerfError, upsample
    x = empty(4 * 8 * 27)
    with pytest.raises(PerfError):
        upsample(x, 3, 0, 2, 2, x)          # output overlaps input
    with pytest.raises(PerfError):
        upsample(x, 1, 0, 2, 2, empty(64))  # G < 2


def test_coarse_to_fine_driver_against_oracle():
    """Three levels (8^3, 16^3, 32^3; maps 8x16 to 32x64) of 3 Gauss-Newton
    steps with 3 PCG iterations on the small workload's cameras and targets.
    The first step of every level is checked against the oracle from the
    oracle's own level change of the previous level's result (parameters
    within the Gauss-Newton tolerance), and every level lowers F."""
    from oracle import Oracle, gn_step
    from oracle.hierarchy import upsample as ref_upsample
    from paper_2112_05598_gb300.hierarchy import coarse_to_fine, level_shapes
    from scenegen import make_scene, random_params
    from gpu_common import TOL_GN
    sc = make_scene("small32")
    orc32 = Oracle.from_scene(sc)
    target = orc32.render(sc.x_gt)[0].astype(np.float32).ravel()
    rng = np.random.default_rng(8)
    S = len(sc.radii)
    x0 = random_params(rng, 8, S, 8, 16, 0.0, 0.1, shell_sigma_hi=0.1)
    seen = []

    def on_step(l, k, shape, x, st):
        seen.append((l, k, shape, host(x), st))

    coarse_to_fine(cuda_tensor(x0), 8, sc.radii, 8, 16, sc.c2w, sc.focal, sc.width, sc.height,
                   cuda_tensor(target), 3, 3, on_step=on_step, pcg_iters=3, pcg_fixed=1)
    assert [(l, k) for l, k, *_ in seen] == [(l, k) for l in range(3) for k in range(3)]
    assert [s[2] for s in seen[::3]] == level_shapes(8, 8, 16, 3)
    prev = None
    for l in range(3):
        G, He, We = seen[3 * l][2]
        x_start = x0.astype(np.float64) if l == 0 else ref_upsample(prev, G // 2, S, He // 2, We // 2)
        orc = Oracle(G, sc.radii, He, We, sc.c2w, sc.focal, sc.width, sc.height,
                     max_samples=int(np.ceil(np.sqrt(3.0) * G)) + 1)
        ref = gn_step(orc, x_start, target.astype(np.float64), 3)
        st, xg = seen[3 * l][4], seen[3 * l][3]
        assert abs(st["F_before"] - ref.F_before) <= 1e-5 * ref.F_before
        if abs(st["gamma"] - ref.gamma) < 1e-9:
            assert rel_l2(xg, ref.x) < TOL_GN, l
        assert seen[3 * l + 2][4]["F_after"] < seen[3 * l][4]["F_before"]
        prev = seen[3 * l + 2][3]

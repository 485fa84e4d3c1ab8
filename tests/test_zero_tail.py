"""The terms a ray's zero row tail drops (CPU; the FP64 oracle).

Where a ray's optical depth passes about 103.3, e^{-V} is below binary32's
smallest subnormal (2^-149, about 1.4e-45) and a binary32 march computes
T_i = 0; from there on its per-sample partials of Eq. 3, w_i = T_i alpha_i and
dH/dsigma_i = dbar_i (T_i e^{-sigma_i dbar_i} c_i - sum_{j>i} w_j c_j), are
products with T_i or with later weights and come out exactly 0, so the GPU's
coefficient store keeps only each ray's prefix before them.  In exact
arithmetic those terms are not 0 but bounded by 2 dbar_i T_i max|c|: this
checks, in FP64, that the transmittance is non-increasing along a ray (the
dropped samples form a suffix) and that every dropped term is below a few
subnormal units, far under any bar the GPU path is held to."""
import numpy as np

BINARY32_MIN_SUBNORMAL = 2.0 ** -149


def _opaque_small32(scale=300.0):
    from scenegen import make_scene
    sc = make_scene("small32")
    x = sc.x_gt.astype(np.float64).reshape(-1, 4).copy()
    x[:sc.G ** 3, 3] *= scale
    return sc, x.ravel()


def test_partials_past_binary32_underflow_are_negligible():
    from oracle import Oracle
    sc, x = _opaque_small32()
    orc = Oracle.from_scene(sc)
    n_pix = sc.width * sc.height
    dropped = 0
    worst = 0.0
    for ray in range(0, n_pix, 3):            # a third of camera 0's rays
        r = orc.ray_samples(x, ray)
        T, a, s, c, d = r["T"], r["alpha"], r["sigma"], r["c"], r["dbar"]
        if len(T) == 0:
            continue
        assert np.all(np.diff(T) <= 0.0)      # sigma >= 0: transmittance never rises
        w = T * a
        tail = np.concatenate([np.cumsum((w[:, None] * c)[::-1], axis=0)[::-1][1:],
                               np.zeros((1, 3))])
        dH = d[:, None] * (T[:, None] * np.exp(-s * d)[:, None] * c - tail)
        under = T < BINARY32_MIN_SUBNORMAL
        if not under.any():
            continue
        first = int(np.argmax(under))
        assert np.all(under[first:])          # a suffix of the ray
        dropped += int(under.sum())
        worst = max(worst, float(np.abs(w[under]).max()), float(np.abs(dH[under]).max()))
    print(f"[zero tail] {dropped} dropped samples, largest dropped term {worst:.3e}")
    assert dropped > 100                     # the opaque state has tails to drop
    assert worst <= 4 * BINARY32_MIN_SUBNORMAL

"""Pins of the FP64 oracle of the learned-preconditioner network."""
import numpy as np

from oracle import lpc as L


def _rand_problem(rng, G=4, w_scale=0.3):
    w = rng.normal(size=L.N_WEIGHTS) * w_scale
    feat = rng.normal(size=(G, G, G, L.C))
    feat[..., 12:] = 0.0
    ahat = rng.normal(size=4 * G ** 3)
    xi = rng.normal(size=4 * G ** 3)
    mask = (rng.uniform(size=G ** 3) > 0.2).astype(np.float64)
    return w, feat, ahat, xi, mask


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    w, feat, ahat, xi, mask = _rand_problem(rng)
    loss, g = L.loss_and_grad(w, feat, ahat, xi, mask)
    assert loss > 0
    idx = rng.choice(L.N_WEIGHTS, size=60, replace=False)
    # biases of every layer too
    idx = np.concatenate([idx, [l * L.LAYER + L.W_PER + c for l in range(4) for c in (0, 5)]])
    eps = 1e-6
    for i in idx:
        wp = w.copy(); wp[i] += eps
        wm = w.copy(); wm[i] -= eps
        fd = (L.loss_and_grad(wp, feat, ahat, xi, mask)[0] -
              L.loss_and_grad(wm, feat, ahat, xi, mask)[0]) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-7 * np.abs(g).max(), (i, fd, g[i])


def test_conv_is_a_3x3x3_correlation():
    """A single tap weight reproduces a shifted copy of one channel."""
    G = 5
    a = np.random.default_rng(1).normal(size=(G, G, G, L.C))
    W = np.zeros((L.TAPS, L.C, L.C))
    tap = (1 + 1) * 9 + (0 + 1) * 3 + (-1 + 1)   # dz = +1, dy = 0, dx = -1
    W[tap, 3, 7] = 2.0                          # out channel 3 <- in channel 7
    out = L.conv(a, W, np.zeros(L.C))
    ref = np.zeros((G, G, G))
    ref[:G - 1, :, 1:] = 2.0 * a[1:, :, :G - 1, 7]
    assert np.allclose(out[..., 3], ref)
    assert np.allclose(np.delete(out, 3, axis=-1), 0.0)


def test_head_is_spd_and_identity_start_is_jacobi():
    rng = np.random.default_rng(2)
    o = rng.normal(size=(50, L.C)) * 3
    Q = L.Q_blocks(o)
    for q in Q:
        np.linalg.cholesky(q)                  # SPD by construction
        assert np.allclose(q, q.T)
    # identity head (softplus(o) = 1 on the diagonal, no off-diagonal) = Jacobi
    o0 = np.zeros((1, L.C)); o0[0, :4] = np.log(np.e - 1)
    assert np.allclose(L.Q_blocks(o0)[0], (1 + L.Q_EPS) * np.eye(4))
    d = np.array([[4.0, 1.0, 0.25, 9.0]])
    w = np.zeros(L.N_WEIGHTS)
    w[3 * L.LAYER + L.W_PER:3 * L.LAYER + L.W_PER + 4] = np.log(np.e - 1)
    P = L.blocks(w, np.zeros((1, 1, 1, L.C)), d)[0]
    assert np.allclose(P, (1 + L.Q_EPS) * np.diag(1.0 / d[0]))

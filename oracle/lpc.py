"""FP64 CPU re-implementation of the learned block preconditioner network.

TEST INFRASTRUCTURE ONLY (checks the library's BF16 training and inference
kernels; never used by them).  Same architecture and weight layout as the
library: 4 layers of 3x3x3 convolution with zero padding, 16 channels,
ReLU after the first three; per layer W[27 taps][16 out][16 in] then bias[16];
tap = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1).  Head: o[0..3] -> softplus ->
diagonal of L, o[4..9] -> L10, L20, L21, L30, L31, L32; Q = L L^T + 1e-3 I;
loss = sum_v mask_v |Q_v a_v - xi_v|^2 / sum |xi|^2.  Gradients are derived
by hand below and pinned against finite differences in the tests.
"""
import numpy as np

C = 16
TAPS = 27
LAYERS = 4
W_PER = TAPS * C * C
LAYER = W_PER + C
N_WEIGHTS = LAYERS * LAYER
Q_EPS = 1e-3


def unpack(w):
    w = np.asarray(w, np.float64)
    out = []
    for l in range(LAYERS):
        blk = w[l * LAYER:(l + 1) * LAYER]
        out.append((blk[:W_PER].reshape(TAPS, C, C), blk[W_PER:]))
    return out


def _shift(a, dz, dy, dx):
    """b[z, y, x] = a[z + dz, y + dy, x + dx] (zero outside)."""
    G = a.shape[0]
    p = np.pad(a, ((1, 1), (1, 1), (1, 1), (0, 0)))
    return p[1 + dz:1 + dz + G, 1 + dy:1 + dy + G, 1 + dx:1 + dx + G]


def _taps():
    for tap in range(TAPS):
        yield tap, tap // 9 - 1, (tap // 3) % 3 - 1, tap % 3 - 1


def conv(a, W, b):
    out = np.zeros(a.shape[:3] + (C,))
    for tap, dz, dy, dx in _taps():
        out += _shift(a, dz, dy, dx) @ W[tap].T
    return out + b


def conv_back(a, W, g):
    """(d a, d W, d b) for out = conv(a, W, b) given g = d out."""
    da = np.zeros_like(a)
    dW = np.zeros_like(W)
    for tap, dz, dy, dx in _taps():
        s = _shift(a, dz, dy, dx)
        dW[tap] = np.einsum("zyxo,zyxi->oi", g, s)
        da += _shift(g @ W[tap], -dz, -dy, -dx)
    return da, dW, g.sum(axis=(0, 1, 2))


def softplus(x):
    return np.where(x > 20, x, np.log1p(np.exp(np.minimum(x, 20))))


def head_L(o):
    L = np.zeros(o.shape[:-1] + (4, 4))
    for i in range(4):
        L[..., i, i] = softplus(o[..., i])
    L[..., 1, 0] = o[..., 4]
    L[..., 2, 0] = o[..., 5]
    L[..., 2, 1] = o[..., 6]
    L[..., 3, 0] = o[..., 7]
    L[..., 3, 1] = o[..., 8]
    L[..., 3, 2] = o[..., 9]
    return L


def forward(w, feat):
    """feat: (G, G, G, 16).  Returns the list of layer outputs (post-ReLU for
    layers 0-2, raw for the head layer)."""
    acts = [np.asarray(feat, np.float64)]
    for l, (W, b) in enumerate(unpack(w)):
        z = conv(acts[-1], W, b)
        acts.append(np.maximum(z, 0.0) if l < LAYERS - 1 else z)
    return acts


def Q_blocks(o):
    L = head_L(o)
    return L @ np.swapaxes(L, -1, -2) + Q_EPS * np.eye(4)


def loss_and_grad(w, feat, ahat, xi, mask=None):
    """Relative loss and its gradient with respect to the flat weights."""
    G = feat.shape[0]
    ahat = np.asarray(ahat, np.float64).reshape(G, G, G, 4)
    xi = np.asarray(xi, np.float64).reshape(G, G, G, 4)
    m = np.ones((G, G, G)) if mask is None else np.asarray(mask, np.float64).reshape(G, G, G)
    scale = 1.0 / max(float(np.sum(xi * xi)), 1e-300)
    acts = forward(w, feat)
    o = acts[-1]
    L = head_L(o)
    Q = L @ np.swapaxes(L, -1, -2) + Q_EPS * np.eye(4)
    e = np.einsum("...ij,...j->...i", Q, ahat) - xi
    loss = scale * float(np.sum(m[..., None] * e * e))
    # d loss / d Q = 2 s e a^T ; d / d L = (dQ + dQ^T) L
    dQ = 2.0 * scale * m[..., None, None] * e[..., :, None] * ahat[..., None, :]
    dL = (dQ + np.swapaxes(dQ, -1, -2)) @ L
    go = np.zeros(o.shape)
    for i in range(4):
        go[..., i] = dL[..., i, i] / (1.0 + np.exp(-o[..., i]))
    go[..., 4] = dL[..., 1, 0]
    go[..., 5] = dL[..., 2, 0]
    go[..., 6] = dL[..., 2, 1]
    go[..., 7] = dL[..., 3, 0]
    go[..., 8] = dL[..., 3, 1]
    go[..., 9] = dL[..., 3, 2]
    layers = unpack(w)
    grads = [None] * LAYERS
    g = go
    for l in range(LAYERS - 1, -1, -1):
        W, b = layers[l]
        da, dW, db = conv_back(acts[l], W, g)
        grads[l] = np.concatenate([dW.reshape(-1), db])
        if l > 0:
            g = da * (acts[l] > 0)
    return loss, np.concatenate(grads)


def blocks(w, feat, diag, floor=1e-30):
    """P_v = D^{-1/2} Q_v D^{-1/2} for every voxel (G^3 x 4 x 4)."""
    G = feat.shape[0]
    Q = Q_blocks(forward(w, feat)[-1]).reshape(-1, 4, 4)
    d = np.asarray(diag, np.float64).reshape(-1, 4)
    s = np.where(d > floor, 1.0 / np.sqrt(np.where(d > floor, d, 1.0)), 0.0)
    return s[:, :, None] * Q * s[:, None, :]

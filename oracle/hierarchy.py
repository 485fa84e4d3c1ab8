"""FP64 oracle of the level change of PERF's hierarchical formulation.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Section "Hierarchical formulation": every level doubles the resolution of
the voxel grid and of the environment maps, and the new buffers are filled
from the previous level's result by linear interpolation.  Written here as
a plain loop-free numpy restatement; the readings it takes are:

* cell-centred samples on both levels: fine voxel i' (side h/2) has its
  centre at coarse index coordinate u = (i' + 1/2)/2 - 1/2, interpolated
  trilinearly with the ray march's clamp convention (u clamped to
  [0, G - 1], base = min(floor(u), G - 2));
* opacity is per voxel side (the sigma-delta-bar convention of Eq. 3 with
  delta-bar = delta / h), so the fine grid's sigma is halved: the optical
  depth of any path through the volume is unchanged;
* environment maps: bilinear in texel space with the same centre mapping,
  the longitude wrapped and the latitude clamped as in the shell lookup;
  a shell hit has delta-bar = 1 on every level, so shell sigma is kept;
* cube maps (F x F texels per face, an F x 6F strip): each face on its own,
  both axes clamped to the face's edge texels, as in the cube lookup.

Pins: ``tests/test_oracle_pins.py`` (constant and linear fields, the wrap
seam by hand, optical-depth preservation).
"""
from __future__ import annotations

import numpy as np


def _axis(n_coarse: int, n_fine: int):
    """Base index and fraction of every fine cell centre on one axis."""
    u = (np.arange(n_fine) + 0.5) / 2.0 - 0.5
    u = np.clip(u, 0.0, n_coarse - 1.0)
    base = np.minimum(np.floor(u), n_coarse - 2.0).astype(np.int64)
    return base, u - base


def upsample_grid(grid: np.ndarray) -> np.ndarray:
    """grid: (G, G, G, 4) indexed [z][y][x][channel] -> (2G, 2G, 2G, 4)."""
    G = grid.shape[0]
    bz, fz = _axis(G, 2 * G)
    by, fy = _axis(G, 2 * G)
    bx, fx = _axis(G, 2 * G)
    g = grid.astype(np.float64)
    out = np.zeros((2 * G, 2 * G, 2 * G, 4))
    for dz in (0, 1):
        wz = fz if dz else 1.0 - fz
        for dy in (0, 1):
            wy = fy if dy else 1.0 - fy
            for dx in (0, 1):
                wx = fx if dx else 1.0 - fx
                w = wz[:, None, None] * wy[None, :, None] * wx[None, None, :]
                out += w[..., None] * g[np.ix_(bz + dz, by + dy, bx + dx)]
    out[..., 3] *= 0.5
    return out


def upsample_shell(tex: np.ndarray) -> np.ndarray:
    """tex: (He, We, 4) indexed [row theta][col phi] -> (2He, 2We, 4)."""
    He, We = tex.shape[0], tex.shape[1]
    br, fr = _axis(He, 2 * He)
    u = (np.arange(2 * We) + 0.5) / 2.0 - 0.5
    c0 = np.floor(u)
    fc = u - c0
    c0 = c0.astype(np.int64) % We
    c1 = (c0 + 1) % We
    t = tex.astype(np.float64)
    out = np.zeros((2 * He, 2 * We, 4))
    for dr in (0, 1):
        wr = fr if dr else 1.0 - fr
        rows = br + dr
        out += (wr[:, None] * (1.0 - fc)[None, :])[..., None] * t[np.ix_(rows, c0)]
        out += (wr[:, None] * fc[None, :])[..., None] * t[np.ix_(rows, c1)]
    return out


def upsample_cube_shell(tex: np.ndarray) -> np.ndarray:
    """tex: (F, 6F, 4), face f in columns [f F, (f + 1) F) -> (2F, 12F, 4)."""
    F = tex.shape[0]
    b, f = _axis(F, 2 * F)
    t = tex.astype(np.float64)
    out = np.zeros((2 * F, 12 * F, 4))
    for face in range(6):
        src = t[:, face * F:(face + 1) * F]
        acc = np.zeros((2 * F, 2 * F, 4))
        for dr in (0, 1):
            wr = f if dr else 1.0 - f
            for dc in (0, 1):
                wc = f if dc else 1.0 - f
                acc += (wr[:, None] * wc[None, :])[..., None] * src[np.ix_(b + dr, b + dc)]
        out[:, 2 * face * F:2 * (face + 1) * F] = acc
    return out


def upsample(x: np.ndarray, G: int, n_shells: int, env_h: int, env_w: int,
             env_kind: int = 0) -> np.ndarray:
    """Parameter vector of level (G, env_h x env_w) -> level (2G, 2env_h x 2env_w)
    (env_kind 1: cube-map shells)."""
    x = np.asarray(x, dtype=np.float64)
    nv = G ** 3
    grid = x[:4 * nv].reshape(G, G, G, 4)
    parts = [upsample_grid(grid).reshape(-1)]
    tex = env_h * env_w
    up = upsample_cube_shell if env_kind == 1 else upsample_shell
    for s in range(n_shells):
        sh = x[4 * nv + 4 * s * tex: 4 * nv + 4 * (s + 1) * tex].reshape(env_h, env_w, 4)
        parts.append(up(sh).reshape(-1))
    return np.concatenate(parts)

"""Pins of the oracle's addressing conventions: where a sample sits in the
grid, which texel a shell hit reads, which way a pixel's ray points, and the
off-diagonal entries of a voxel's 4x4 block of J^T J.

The finite-difference pins differentiate the oracle's own forward model, and
the constant-field closed forms cannot see an index shift.  So a convention
mistake made consistently (a half-voxel shift of the cell centres, a mirrored
azimuth, a flipped pole, a vertically flipped image, transposed texel
indices) would pass them, and the GPU would copy it and pass parity too.
The cases below pin each convention to values worked out by hand from its
statement (Section "Volume Rendering", Eq. 3-4; Section "Preconditioner"):

* voxel (ix, iy, iz) is centred at -1 + (i + 1/2) h, h = 2 / G; stored
  [iz][iy][ix][4], x fastest; interpolation is trilinear, clamped to the
  outermost centres;
* samples sit at t_in + (k + 1/2) delta, delta = L / K, K = ceil(L / h);
* a camera is (right, up, back, position); pixel (col, row) has its centre at
  (col + 1/2, row + 1/2), rows going down the image, so pixel (0, 0) looks to
  the left (-right) and up (+up);
* shell texel (row, col) of an H_e x W_e map is stored [row][col]; row 0 is
  the +z pole; the texel coordinate of a unit direction is
  u = (phi / 2 pi + 1/2) W_e - 1/2 (phi = atan2(y, x), wrapped across the
  -pi / pi seam) and v = (theta / pi) H_e - 1/2 (theta from +z, clamped).
"""
import math

import numpy as np
import pytest

from conftest import tiny_problem
from oracle import Oracle


def _c2w(right, up, back, pos):
    m = np.zeros((1, 3, 4), np.float32)
    m[0, :, 0], m[0, :, 1], m[0, :, 2], m[0, :, 3] = right, up, back, pos
    return m


def _linear_field(G, S=0, env_h=2, env_w=2, a=(0.5, 0.5, 0.5), b=(0.4, 0.4, 0.4), sigma=0.5):
    """Colour linear in position: r = a0 + b0 x, g = a1 + b1 y, b = a2 + b2 z at
    the voxel centres; uniform opacity sigma (per voxel side)."""
    h = 2.0 / G
    cen = -1.0 + (np.arange(G) + 0.5) * h
    x = np.zeros((G, G, G, 4))
    zz, yy, xx = np.meshgrid(cen, cen, cen, indexing="ij")
    x[..., 0] = a[0] + b[0] * xx
    x[..., 1] = a[1] + b[1] * yy
    x[..., 2] = a[2] + b[2] * zz
    x[..., 3] = sigma
    shells = np.zeros((S * env_h * env_w, 4))
    return np.concatenate([x.reshape(-1), shells.reshape(-1)])


# ------------------------------------------------------------ trilinear


@pytest.mark.parametrize("axis", ["z", "x", "y"])
def test_axis_ray_through_linear_field(axis):
    """One pixel, its ray along -z (or -x, -y) through (0.3125, -0.4375) (exact in binary32): G = 8,
    h = 1/4, chord 2 = 8 voxel sides, so K = 8, delta = h (delta_bar = 1) and
    the samples sit exactly on the voxel centres +-0.875, +-0.625, +-0.375,
    +-0.125 along the ray.  The interpolated colour at a sample is the linear
    field at the sample (no clamp: every coordinate is within the outermost
    centres), so with T_k = e^{-0.5 k} and alpha = 1 - e^{-0.5}:
      lateral channel:  (0.5 + 0.4 * offset) (1 - e^{-4})
      along-ray channel: sum_k T_k alpha (0.5 + 0.4 * coordinate of sample k).
    A half-voxel shift of the centres changes every interior sample's value by
    0.4 * h / 2 = 0.05, and swapping two axes of the [z][y][x] layout reads the
    wrong channel's slope."""
    G = 8
    x = _linear_field(G)
    lat = {"z": ((1, 0, 0), (0, 1, 0), (0, 0, 1), (0.3125, -0.4375, 3.0)),
           "x": ((0, 1, 0), (0, 0, 1), (1, 0, 0), (3.0, 0.3125, -0.4375)),
           "y": ((0, 0, 1), (1, 0, 0), (0, 1, 0), (-0.4375, 3.0, 0.3125))}[axis]
    orc = Oracle(G, [], 2, 2, _c2w(*lat), np.array([1.0], np.float32), 1, 1, max_samples=64)
    info = orc.ray_info(0)
    assert info["K"] == 8 and info["delta"] == 0.25 and info["t_in"] == 2.0
    rgb = orc.render(x)[0][0]
    # coordinates of the 8 samples along the ray, entering at +1
    along = [0.875, 0.625, 0.375, 0.125, -0.125, -0.375, -0.625, -0.875]
    alpha = 1.0 - math.exp(-0.5)
    along_sum = sum(math.exp(-0.5 * k) * alpha * (0.5 + 0.4 * c) for k, c in enumerate(along))
    full = 1.0 - math.exp(-4.0)
    ch_along = {"x": 0, "y": 1, "z": 2}[axis]
    # the ray's fixed coordinates per channel
    fixed = {"z": {0: 0.3125, 1: -0.4375}, "x": {1: 0.3125, 2: -0.4375},
             "y": {2: 0.3125, 0: -0.4375}}[axis]
    expected = np.zeros(3)
    expected[ch_along] = along_sum
    for ch, off in fixed.items():
        expected[ch] = (0.5 + 0.4 * off) * full
    assert np.allclose(rgb, expected, rtol=1e-12, atol=1e-14), (rgb, expected)


def test_clamp_to_outermost_centres():
    """A sample between the last centre and the face reads the last voxel
    (clamp address mode): a ray along -z at x = 0.95 (beyond the last x-centre
    0.875 at G = 8) sees r = 0.5 + 0.4 * 0.875 on every sample."""
    G = 8
    x = _linear_field(G)
    orc = Oracle(G, [], 2, 2, _c2w((1, 0, 0), (0, 1, 0), (0, 0, 1), (0.95, 0.0, 3.0)),
                 np.array([1.0], np.float32), 1, 1, max_samples=64)
    rgb = orc.render(x)[0][0]
    assert abs(rgb[0] - (0.5 + 0.4 * 0.875) * (1 - math.exp(-4.0))) < 1e-13


# ------------------------------------------------------------- pixel -> ray


def test_pixel_to_ray_by_hand():
    """Camera at (0, 0, 3) with right = +x, up = +y, back = +z, 4x4 pixels,
    focal 8 px, G = 4 (h = 1/2).  Pixel centre (col + 1/2, row + 1/2) is
    (x_c, y_c) = ((col + 1/2 - 2) / 8, -(row + 1/2 - 2) / 8) in the image
    plane at unit depth, so
      pixel (col 0, row 0), ray 0:   direction ~ (-0.1875, +0.1875, -1)
      pixel (col 3, row 0), ray 3:   direction ~ (+0.1875, +0.1875, -1)
      pixel (col 0, row 3), ray 12:  direction ~ (-0.1875, -0.1875, -1)
    (ray index = row * 4 + col).  Normalised by sqrt(1 + 2 * 0.1875^2) =
    1.0345590848: (-+0.18123663, +-0.18123663, -0.96659535).  The ray enters
    the box through z = 1 at t = 2 / 0.96659535 = 2.0691182 and leaves through
    z = -1 at t = 4.1382363 (|x|, |y| stay below 0.75); L = 2.0691182 =
    4.138 h, so K = 5 and delta = 0.41382363.  Sample k sits at depth
    z_k = 1 - 0.4 (k + 1/2) = 0.8, 0.4, 0, -0.4, -0.8 with lateral offsets
    0.1875 (3 - z_k) = 0.4125, 0.4875, 0.5625, 0.6375, 0.7125."""
    c2w = _c2w((1, 0, 0), (0, 1, 0), (0, 0, 1), (0, 0, 3))
    orc = Oracle(4, [], 2, 2, c2w, np.array([8.0], np.float32), 4, 4, max_samples=64)
    dd = 0.18123663
    for ray, sx, sy in ((0, -1, 1), (3, 1, 1), (12, -1, -1), (15, 1, -1)):
        info = orc.ray_info(ray)
        assert np.allclose(info["d"], [sx * dd, sy * dd, -0.96659535], atol=2e-7), (ray, info["d"])
        assert np.allclose(info["o"], [0, 0, 3])
        assert abs(info["t_in"] - 2.0691182) < 2e-6 and abs(info["t_out"] - 4.1382363) < 2e-6
        assert info["K"] == 5 and abs(info["delta"] - 0.41382363) < 1e-6
    # render through the linear field: colour (0.5 + 0.4 x, 0.5 + 0.4 y, 0.5 + 0.4 z)
    # at the samples; z is clamped to +-0.75 (the outermost centres at G = 4)
    x = _linear_field(4, sigma=0.5)
    rgb = orc.render(x)[0]
    dbar = 0.41382363 / 0.5
    alpha = 1.0 - math.exp(-0.5 * dbar)
    zs = [0.8, 0.4, 0.0, -0.4, -0.8]
    lat = [0.4125, 0.4875, 0.5625, 0.6375, 0.7125]
    for ray, sx, sy in ((0, -1, 1), (3, 1, 1), (12, -1, -1), (15, 1, -1)):
        exp_rgb = np.zeros(3)
        for k in range(5):
            w = math.exp(-0.5 * dbar * k) * alpha
            exp_rgb += w * np.array([0.5 + 0.4 * sx * lat[k], 0.5 + 0.4 * sy * lat[k],
                                     0.5 + 0.4 * max(-0.75, min(0.75, zs[k]))])
        assert np.allclose(rgb[ray], exp_rgb, rtol=2e-6), (ray, rgb[ray], exp_rgb)


# ---------------------------------------------------------- equirect texels

# Hand-worked texel coordinates on a 4 x 8 map (H_e = 4 rows, W_e = 8 columns)
# for a camera at the origin: the hit point of the far root lies along the
# ray's direction.  Each entry: direction, (row value, column value) read back
# from a map whose texel (row, col) holds colour (row, col, 0).
#   +x: phi = 0, theta = pi/2:  u = 0.5*8 - 0.5 = 3.5, v = 0.5*4 - 0.5 = 1.5
#   +y: phi = pi/2:             u = 0.75*8 - 0.5 = 5.5, v = 1.5
#   -y: phi = -pi/2:            u = 0.25*8 - 0.5 = 1.5, v = 1.5
#   (1,1,1)/sqrt 3: phi = pi/4: u = 0.625*8 - 0.5 = 4.5;
#       theta = acos(1/sqrt 3) = 0.95531662, v = 0.30408672*4 - 0.5 = 0.71634690
#   near +z (0.01, 0, 1): theta = 0.0099997, v = -0.4873 -> clamped to row 0;
#       phi = 0: u = 3.5
#   near -z (0.01, 0, -1): theta = pi - 0.0099997, v = 3.4873 -> clamped to row 3
#   seam, (-1, +0.001, 0): phi = pi - 0.001, u = 7.5 - 8*0.001/(2 pi) = 7.49872676:
#       columns 7 and 0 (wrapped), weight of column 0 = 0.49872676, so the
#       column value = 7 * 0.50127324 = 3.50891268
#   seam, (-1, -0.001, 0): phi = -pi + 0.001, u = -0.49872676: columns 7
#       (wrapped from -1) and 0, weight of column 0 = 0.50127324, so the
#       column value = 7 * 0.49872676 = 3.49108732
EQUIRECT_CASES = [
    ((1.0, 0.0, 0.0), 1.5, 3.5),
    ((0.0, 1.0, 0.0), 1.5, 5.5),
    ((0.0, -1.0, 0.0), 1.5, 1.5),
    ((1.0, 1.0, 1.0), 0.71634690, 4.5),
    ((0.01, 0.0, 1.0), 0.0, 3.5),
    ((0.01, 0.0, -1.0), 3.0, 3.5),
    ((-1.0, 0.001, 0.0), 1.5, 3.50891268),
    ((-1.0, -0.001, 0.0), 1.5, 3.49108732),
]


def _camera_looking(direction):
    d = np.asarray(direction, np.float64)
    d /= np.linalg.norm(d)
    helper = np.array([0.0, 0.0, 1.0]) if abs(d[2]) < 0.9 else np.array([1.0, 0.0, 0.0])
    right = np.cross(d, helper); right /= np.linalg.norm(right)
    up = np.cross(right, d)
    return _c2w(right, up, -d, (0.0, 0.0, 0.0))[0]


def test_equirect_texel_map_by_hand():
    He, We, sig = 4, 8, 2.0
    c2w = np.stack([_camera_looking(c[0]) for c in EQUIRECT_CASES]).astype(np.float32)
    focal = np.ones(len(EQUIRECT_CASES), np.float32)
    orc = Oracle(2, [2.5], He, We, c2w, focal, 1, 1, max_samples=64)
    x = np.zeros(orc.n_params).reshape(-1, 4)
    g = 8                                      # 2^3 voxels, sigma = 0: transparent
    rows, cols = np.meshgrid(np.arange(He), np.arange(We), indexing="ij")
    x[g:, 0] = rows.reshape(-1)
    x[g:, 1] = cols.reshape(-1)
    x[g:, 2] = 0.0
    x[g:, 3] = sig
    rgb = orc.render(x.reshape(-1))[0]
    a = 1.0 - math.exp(-sig)
    for i, (d, row_v, col_v) in enumerate(EQUIRECT_CASES):
        assert abs(rgb[i, 0] - a * row_v) < 2e-6, (d, rgb[i] / a)
        assert abs(rgb[i, 1] - a * col_v) < 2e-6, (d, rgb[i] / a)


# ---------------------------------------------------------- block couplings


def test_block_cross_is_column_products_of_dense_J():
    """cross[4v + k] = sum_rows (dr/dc_{v,k})(dr/dsigma_v), the off-diagonal
    entries of voxel v's 4x4 block of J^T J, against the same products of the
    columns of J by central differences of the forward model; the colour
    channels' mutual entries vanish (colour k enters residual k only)."""
    from test_oracle_pins import fd_jacobian, _orc
    rng = np.random.default_rng(7)
    prob = tiny_problem(rng)
    orc = _orc(prob)
    x = prob["x"].astype(np.float64)
    J = fd_jacobian(orc, x)
    diag, cross = orc.block_cross(x)
    nv = prob["G"] ** 3
    ref = np.zeros(4 * nv)
    for v in range(nv):
        for k in range(3):
            ref[4 * v + k] = float(J[:, 4 * v + k] @ J[:, 4 * v + 3])
        # colour-colour entries of the block are zero
        for k in range(3):
            for l in range(k + 1, 3):
                assert abs(float(J[:, 4 * v + k] @ J[:, 4 * v + l])) < 1e-12
    assert np.abs(ref).max() > 1e-3
    assert np.abs(cross - ref).max() <= 1e-7 * np.abs(ref).max()
    assert np.abs(diag - np.sum(J * J, axis=0)).max() <= 1e-7 * np.abs(diag).max()


# ---------------------------------------------------------- cube-map texels

# Hand-worked texels of a cube map with F = 4 texels per face edge (a 4 x 24
# strip; face f = +x, -x, +y, -y, +z, -z in columns [4 f, 4 f + 4)), read
# along directions from a camera at the origin.  On the face of the largest
# |q_a| (ties to the lower axis), with (b, c) the other axes in increasing
# order, s = q_b / |q_a|, t = q_c / |q_a|, column coordinate u = 2 s + 1.5 and
# row coordinate v = 2 t + 1.5 (texel i centred at i), clamped to [0, 3].
# Each entry: direction, (row value, strip-column value) of a map whose texel
# (row, column) holds colour (row, column, 0).
#   +x: face 0, s = t = 0: u = v = 1.5 -> (1.5, 0 + 1.5)
#   -x: face 1 -> (1.5, 4 + 1.5); +y: face 2 -> (1.5, 8 + 1.5); -y: face 3 ->
#   (1.5, 12 + 1.5); +z: face 4 -> (1.5, 16 + 1.5); -z: face 5 -> (1.5, 20 + 1.5)
#   (0.5, 1, 0.25): face 2 (+y), s = 0.5, t = 0.25: u = 2.5, v = 2.0 -> (2.0, 10.5)
#   (1, 1, 0): |x| = |y|, the tie goes to x: face 0, s = 1: u = 3.5 -> clamped
#       to the edge texel 3; t = 0: v = 1.5 -> (1.5, 3.0)
#   (-1, -0.5, 0.5): face 1 (-x), s = -0.5, t = 0.5: u = 0.5, v = 2.5 -> (2.5, 4.5)
#   (0.2, -0.99, -0.95): face 3 (-y), s = 0.2 / 0.99 = 0.2020202,
#       t = -0.95 / 0.99 = -0.9595960: u = 1.9040404, v = -0.419 -> row 0
#       -> (0.0, 12 + 1.9040404)
CUBE_CASES = [
    ((1.0, 0.0, 0.0), 1.5, 1.5),
    ((-1.0, 0.0, 0.0), 1.5, 5.5),
    ((0.0, 1.0, 0.0), 1.5, 9.5),
    ((0.0, -1.0, 0.0), 1.5, 13.5),
    ((0.0, 0.0, 1.0), 1.5, 17.5),
    ((0.0, 0.0, -1.0), 1.5, 21.5),
    ((0.5, 1.0, 0.25), 2.0, 10.5),
    ((1.0, 1.0, 0.0), 1.5, 3.0),
    ((-1.0, -0.5, 0.5), 2.5, 4.5),
    ((0.2, -0.99, -0.95), 0.0, 13.9040404),
]


def test_cube_map_texels_by_hand():
    F, sig = 4, 2.0
    c2w = np.stack([_camera_looking(c[0]) for c in CUBE_CASES]).astype(np.float32)
    orc = Oracle(2, [2.5], F, 6 * F, c2w, np.ones(len(CUBE_CASES), np.float32), 1, 1,
                 max_samples=64, env_kind=1)
    x = np.zeros(orc.n_params).reshape(-1, 4)
    rows, cols = np.meshgrid(np.arange(F), np.arange(6 * F), indexing="ij")
    x[8:, 0] = rows.reshape(-1)
    x[8:, 1] = cols.reshape(-1)
    x[8:, 3] = sig
    rgb = orc.render(x.reshape(-1))[0]
    a = 1.0 - math.exp(-sig)
    for i, (d, row_v, col_v) in enumerate(CUBE_CASES):
        assert abs(rgb[i, 0] - a * row_v) < 2e-6, (d, rgb[i] / a)
        assert abs(rgb[i, 1] - a * col_v) < 2e-6, (d, rgb[i] / a)


def test_cube_map_derivatives_match_finite_differences():
    """J with cube-map shells: columns of J p and rows of J^T v against central
    differences of the forward model, and the diagonal against column norms."""
    from test_oracle_pins import fd_jacobian, _orc
    rng = np.random.default_rng(71)
    prob = tiny_problem(rng, env_h=2, env_w=12, n_cams=3)
    orc = _orc(prob, env_kind=1)
    x = prob["x"].astype(np.float64)
    J = fd_jacobian(orc, x)
    nv = 4 * prob["G"] ** 3
    assert np.abs(J[:, nv:]).max() > 1e-3          # the cube-map texels are seen
    n = x.shape[0]
    for j in range(0, n, 3):
        e = np.zeros(n); e[j] = 1.0
        assert np.abs(orc.jvp(x, e) - J[:, j]).max() <= 1e-7 * np.abs(J).max() + 1e-9
    v = rng.normal(size=J.shape[0])
    assert np.abs(orc.vjp(x, v) - J.T @ v).max() <= 1e-7 * np.abs(J.T @ v).max()
    d, _ = orc.diag_grad(x)
    assert np.abs(d - np.sum(J * J, axis=0)).max() <= 1e-7 * d.max()

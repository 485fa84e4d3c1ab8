"""FP64 CPU oracle for the PERF Gauss-Newton path.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg
of the benchmark use it to check the CUDA library; the library never imports,
links or calls it.  It shares no code with the CUDA path -- only the seeded
inputs of ``scenegen`` serve both.

The per-ray work (Eq. 3-4 ray march, the partial derivatives of Eq. 3, J p,
J^T v, exact diag(J^T J)) is plain C in ``oracle.c``; this module adds

* Algorithm 2 (Jacobi-preconditioned conjugate gradients) on
  A = J^T J with b = -J^T r (Section "Update step"),
* Algorithm 3 (backtracking line search, alpha = 0.7) and
* the Gauss-Newton update of Eq. 7 with the projection
  sigma >= 0, 0 <= c <= 1 applied to every trial point,

written in numpy FP64 in the paper's order and notation.

Parity pins for every function are in ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
from typing import Callable, List, Optional

import numpy as np

from . import build as _build

_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        _LIB = ctypes.CDLL(_build.build())
        _LIB.oc_jitter_uniform.restype = ctypes.c_float
    return _LIB


class _Problem(ctypes.Structure):
    _fields_ = [
        ("G", ctypes.c_int), ("S", ctypes.c_int),
        ("env_h", ctypes.c_int), ("env_w", ctypes.c_int),
        ("radii", ctypes.c_float * 8),
        ("n_cams", ctypes.c_int), ("width", ctypes.c_int),
        ("height", ctypes.c_int),
        ("c2w", ctypes.c_void_p), ("focal", ctypes.c_void_p),
        ("max_samples", ctypes.c_int), ("jitter", ctypes.c_int),
        ("seed", ctypes.c_uint64), ("epoch", ctypes.c_uint32),
        ("n_threads", ctypes.c_int),
        ("aux", ctypes.c_int), ("aux_lambda", ctypes.c_double),
        ("env_kind", ctypes.c_int),
    ]


def _dptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class Oracle:
    """One scene (grid size, shells, cameras) for the FP64 oracle."""

    def __init__(self, G, radii, env_h, env_w, c2w, focal, width, height,
                 max_samples=512, jitter=False, seed=0, epoch=0, n_threads=0, aux=False,
                 aux_lambda=0.1, env_kind=0):
        radii = [float(r) for r in radii]
        if len(radii) > 8:
            raise ValueError("at most 8 shells")
        self.c2w = np.ascontiguousarray(c2w, dtype=np.float32).reshape(-1, 12)
        self.focal = np.ascontiguousarray(focal, dtype=np.float32).reshape(-1)
        self.G, self.S = int(G), len(radii)
        self.env_h, self.env_w = int(env_h), int(env_w)
        self.width, self.height = int(width), int(height)
        self.n_cams = int(self.c2w.shape[0])
        self.p = _Problem()
        self.p.G, self.p.S = self.G, self.S
        self.p.env_h, self.p.env_w = self.env_h, self.env_w
        for i, r in enumerate(radii):
            self.p.radii[i] = r
        self.p.n_cams, self.p.width, self.p.height = self.n_cams, self.width, self.height
        self.p.c2w = _dptr(self.c2w)
        self.p.focal = _dptr(self.focal)
        self.p.max_samples = int(max_samples)
        self.p.jitter = int(bool(jitter))
        self.p.seed = int(seed)
        self.p.epoch = int(epoch)
        self.p.n_threads = int(n_threads)
        # Section "Auxiliary terms": a 4th residual per ray penalising
        # grid-exit transmittance away from 0 and 1
        self.p.aux = int(bool(aux))
        self.p.aux_lambda = float(aux_lambda)
        # Section "Implementation": cube-map shells (env_w = 6 env_h, face f in
        # columns [f env_h, (f + 1) env_h)) instead of equirectangular ones
        if env_kind not in (0, 1):
            raise ValueError("env_kind is 0 (equirect) or 1 (cube map)")
        if env_kind == 1 and self.S > 0 and self.env_w != 6 * self.env_h:
            raise ValueError("a cube-map shell is env_h x 6 env_h texels")
        self.p.env_kind = int(env_kind)
        self.env_kind = int(env_kind)
        self.n_res = 4 if aux else 3
        self.n_params = 4 * (self.G ** 3 + self.S * self.env_h * self.env_w)
        self.n_rays = self.n_cams * self.width * self.height

    @classmethod
    def from_scene(cls, scene, **kw):
        kw.setdefault("max_samples", scene.cfg.max_samples)
        kw.setdefault("env_kind", getattr(scene, "env_kind", 0))
        return cls(scene.G, scene.radii, scene.env_h, scene.env_w, scene.c2w,
                   scene.focal, scene.width, scene.height, **kw)

    def set_epoch(self, epoch):
        self.p.epoch = int(epoch)

    # -- helpers
    def _x(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
        if x.shape[0] != self.n_params:
            raise ValueError(f"expected {self.n_params} parameters, got {x.shape[0]}")
        return x

    def _ids(self, ids):
        if ids is None:
            return None, self.n_rays
        ids = np.ascontiguousarray(ids, dtype=np.int64)
        return ids, int(ids.shape[0])

    # -- forward model (Eq. 3-4)
    def render(self, x, ids=None):
        """Returns (rgb [N,3], T at grid exit [N], T after the shells [N])."""
        x = self._x(x)
        ids, N = self._ids(ids)
        rgb = np.zeros((N, 3)); te = np.zeros(N); tf = np.zeros(N)
        _lib().oc_render(ctypes.byref(self.p), _dptr(x),
                         _dptr(ids) if ids is not None else None,
                         ctypes.c_int64(N), _dptr(rgb), _dptr(te), _dptr(tf))
        return rgb, te, tf

    def render_threshold(self, x, min_opacity):
        """Section "Rendering": for a converged scene, a ray whose total
        opacity within the volume (1 - T at grid exit) is below min_opacity
        sees the volume as fully transparent.  Written as its definition:
        such rays take the render of the same scene with every grid opacity
        set to zero (the shells alone); the others the plain render."""
        x = self._x(x)
        rgb, te, _ = self.render(x)
        clear = x.copy()
        clear[:4 * self.G ** 3].reshape(-1, 4)[:, 3] = 0.0
        rgb0 = self.render(clear)[0]
        cut = (1.0 - te) < min_opacity
        rgb[cut] = rgb0[cut]
        return rgb, te

    def residual(self, x, target, ids=None):
        """r = H^ - C per ray and channel, F = 1/2 sum r^2 (Eq. 5-6); with the
        auxiliary term, 4 residuals per ray (the 4th L, its target 0)."""
        x = self._x(x)
        ids, N = self._ids(ids)
        target = np.ascontiguousarray(target, dtype=np.float64).reshape(-1)
        if target.shape[0] != 3 * N:
            raise ValueError("target size")
        r = np.zeros(self.n_res * N)
        F = ctypes.c_double(0.0)
        _lib().oc_residual(ctypes.byref(self.p), _dptr(x), _dptr(target),
                           _dptr(ids) if ids is not None else None,
                           ctypes.c_int64(N), _dptr(r), ctypes.byref(F))
        return r, F.value

    def error(self, x, target):
        return self.residual(x, target)[1]

    # -- derivatives of Eq. 3 (Section "Computation of partial derivatives")
    def jvp(self, x, p, ids=None, mag=False):
        """J p; with mag=True also |J| |p| (per entry, the sum of the absolute
        values of its terms: the scale of its rounding error)."""
        x = self._x(x)
        p = self._x(p)
        ids, N = self._ids(ids)
        out = np.zeros(self.n_res * N)
        m = np.zeros(self.n_res * N) if mag else None
        _lib().oc_jvp_mag(ctypes.byref(self.p), _dptr(x), _dptr(p),
                          _dptr(ids) if ids is not None else None,
                          ctypes.c_int64(N), _dptr(out), _dptr(m) if mag else None)
        return (out, m) if mag else out

    def vjp(self, x, v, mag=False):
        """J^T v; with mag=True also |J|^T |v|."""
        x = self._x(x)
        v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1)
        if v.shape[0] != self.n_res * self.n_rays:
            raise ValueError("v size")
        out = np.zeros(self.n_params)
        m = np.zeros(self.n_params) if mag else None
        _lib().oc_vjp_mag(ctypes.byref(self.p), _dptr(x), _dptr(v), _dptr(out), 0,
                          _dptr(m) if mag else None)
        return (out, m) if mag else out

    def apply_A(self, x, p):
        """A p = J^T (J p), the product the PCG of Section "Update step" needs."""
        return self.vjp(x, self.jvp(x, p))

    def diag_grad(self, x, r=None):
        """(diag(J^T J), J^T r) -- the Jacobi preconditioner and the gradient."""
        x = self._x(x)
        diag = np.zeros(self.n_params)
        grad = np.zeros(self.n_params)
        rr = None
        if r is not None:
            rr = np.ascontiguousarray(r, dtype=np.float64).reshape(-1)
        _lib().oc_diag_grad(ctypes.byref(self.p), _dptr(x),
                            _dptr(rr) if rr is not None else None,
                            _dptr(diag), _dptr(grad))
        return diag, (grad if r is not None else None)

    def block_cross(self, x):
        """(diag(J^T J), cross) with cross[4v + k] = sum_rows dr/dc_{v,k} dr/dsigma_v
        for grid voxel v (the off-diagonal entries of its 4x4 block of J^T J)."""
        x = self._x(x)
        diag = np.zeros(self.n_params)
        cross = np.zeros(4 * self.G ** 3)
        _lib().oc_block_cross(ctypes.byref(self.p), _dptr(x), _dptr(diag), _dptr(cross))
        return diag, cross

    def ray_samples(self, x, ray, cap=1024):
        x = self._x(x)
        T = np.zeros(cap); a = np.zeros(cap); s = np.zeros(cap)
        c = np.zeros(3 * cap); d = np.zeros(cap)
        ng = ctypes.c_int(0)
        n = _lib().oc_ray_samples(ctypes.byref(self.p), _dptr(x), ctypes.c_int64(ray),
                                  ctypes.c_int(cap), _dptr(T), _dptr(a), _dptr(s),
                                  _dptr(c), _dptr(d), ctypes.byref(ng))
        n = min(n, cap)
        return dict(T=T[:n], alpha=a[:n], sigma=s[:n], c=c[:3 * n].reshape(n, 3),
                    dbar=d[:n], n_grid=ng.value)

    def ray_info(self, ray):
        o = (ctypes.c_float * 3)(); d = (ctypes.c_float * 3)()
        ti = ctypes.c_float(); to = ctypes.c_float(); de = ctypes.c_float()
        K = ctypes.c_int(); sh = ctypes.c_uint()
        _lib().oc_ray_info(ctypes.byref(self.p), ctypes.c_int64(ray), o, d,
                           ctypes.byref(ti), ctypes.byref(to), ctypes.byref(de),
                           ctypes.byref(K), ctypes.byref(sh))
        return dict(o=np.array(o[:], np.float32), d=np.array(d[:], np.float32),
                    t_in=ti.value, t_out=to.value, delta=de.value, K=K.value,
                    shell_hit=sh.value)

    def jitter_uniform(self, ray, stream):
        return float(_lib().oc_jitter_uniform(ctypes.byref(self.p),
                                              ctypes.c_int64(ray),
                                              ctypes.c_uint32(stream)))


# ------------------------------------------------------------ Algorithm 2

@dataclasses.dataclass
class PCGResult:
    x: np.ndarray
    iters: int
    R: List[float]          # r_k^T r_k after each iteration
    alphas: List[float]
    betas: List[float]
    exit: str               # "fixed" | "eps" | "stall" | "breakdown"


# Jacobi diagonal entries at or below this count as unobserved (z_j = 0).
# The paper's implementation keeps the diagonal in binary32, where the square
# of a row entry below ~1e-19 is not a normal number; parameters that deep
# behind opaque matter are indistinguishable from ones no ray sees (Section
# "Preconditioner").  1e-30 leaves binary32 full relative precision above it.
JACOBI_FLOOR = 1e-30


def jacobi_apply(diag: np.ndarray, r: np.ndarray) -> np.ndarray:
    """z = M^{-1} r with M = diag(J^T J); parameters that no residual depends
    on (d_j = 0), or only through entries squaring to at most JACOBI_FLOOR,
    get z_j = 0."""
    z = np.zeros_like(r)
    nz = diag > JACOBI_FLOOR
    z[nz] = r[nz] / diag[nz]
    return z


def pcg(apply_A: Callable[[np.ndarray], np.ndarray], b: np.ndarray,
        Minv: Callable[[np.ndarray], np.ndarray], max_iter: int,
        fixed: bool = True, eps_rel: float = 0.0, stall: float = 0.85,
        x0: Optional[np.ndarray] = None) -> PCGResult:
    """Algorithm 2.  ``fixed``: run exactly ``max_iter`` iterations (no exit
    test); otherwise exit when R < eps_rel^2 R_0 or R / R_prev > stall."""
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - apply_A(x) if x0 is not None else b.copy()
    R_prev = float(r @ r)
    R0 = R_prev
    z = Minv(r)
    p = z.copy()
    rz = float(r @ z)
    Rs, al, be = [], [], []
    exit_reason = "fixed"
    k = 0
    while k < max_iter:
        Ap = apply_A(p)
        pAp = float(p @ Ap)
        if not (pAp > 0.0) or not np.isfinite(pAp):
            exit_reason = "breakdown"
            break
        alpha = rz / pAp
        x = x + alpha * p
        r = r - alpha * Ap
        R = float(r @ r)
        Rs.append(R)
        al.append(alpha)
        k += 1
        if not fixed:
            if R < eps_rel * eps_rel * R0:
                exit_reason = "eps"
                break
            if R / R_prev > stall:
                exit_reason = "stall"
                break
        R_prev = R
        z = Minv(r)
        rz_new = float(r @ z)
        beta = rz_new / rz if rz != 0.0 else 0.0
        be.append(beta)
        p = z + beta * p
        rz = rz_new
    return PCGResult(x=x, iters=k, R=Rs, alphas=al, betas=be, exit=exit_reason)


# ------------------------------------------------------------ Algorithm 3

def line_search(error: Callable[[float], float], alpha: float = 0.7,
                max_halvings: int = 20):
    """Algorithm 3: gamma = 1, decimate by alpha while Error(gamma) keeps
    falling; return the last gamma before it rose (gamma / alpha).  The
    number of decimations is capped (the printed loop has no bound).
    Returns (gamma, mu(gamma), list of (gamma, mu))."""
    gamma = 1.0
    mu_prev = float(np.finfo(np.float32).max)
    trace = []
    for _ in range(max_halvings + 1):
        mu = float(error(gamma))
        trace.append((gamma, mu))
        if mu > mu_prev:
            return gamma / alpha, mu_prev, trace
        gamma = alpha * gamma
        mu_prev = mu
    return gamma / alpha, mu_prev, trace


def project(x: np.ndarray) -> np.ndarray:
    """P: sigma >= 0 and colours in [0, 1] for every voxel and texel."""
    y = np.array(x, dtype=np.float64).reshape(-1, 4)
    y[:, 0:3] = np.clip(y[:, 0:3], 0.0, 1.0)
    y[:, 3] = np.maximum(y[:, 3], 0.0)
    return y.reshape(-1)


@dataclasses.dataclass
class GNStep:
    x: np.ndarray
    F_before: float
    F_after: float
    gamma: float
    accepted: bool
    pcg: PCGResult
    trace: list
    delta: np.ndarray
    diag: np.ndarray = None     # the Jacobi diagonal of the step's system


def gn_step(orc: Oracle, x, target, pcg_iters: int, fixed: bool = True,
            eps_rel: float = 0.0, stall: float = 0.85, ls_alpha: float = 0.7,
            ls_max: int = 20, do_project: bool = True) -> GNStep:
    """One Gauss-Newton step (Eq. 7): solve J^T J Delta = -J^T r by
    Algorithm 2 with the Jacobi preconditioner, pick gamma by Algorithm 3,
    and accept x <- P(x + gamma Delta) only if it lowers F."""
    x = np.asarray(x, dtype=np.float64)
    r, F = orc.residual(x, target)
    diag, grad = orc.diag_grad(x, r)
    b = -grad
    res = pcg(lambda p: orc.apply_A(x, p), b, lambda v: jacobi_apply(diag, v),
              pcg_iters, fixed=fixed, eps_rel=eps_rel, stall=stall)
    delta = res.x
    P = project if do_project else (lambda y: y)
    gamma, mu, trace = line_search(lambda g: orc.error(P(x + g * delta), target),
                                   ls_alpha, ls_max)
    accepted = mu < F
    x_new = P(x + gamma * delta) if accepted else x.copy()
    return GNStep(x=x_new, F_before=F, F_after=mu if accepted else F, gamma=gamma,
                  accepted=accepted, pcg=res, trace=trace, delta=delta, diag=diag)


def psnr(rgb: np.ndarray, target: np.ndarray) -> float:
    mse = float(np.mean((np.asarray(rgb, np.float64) - np.asarray(target, np.float64)) ** 2))
    return float("inf") if mse == 0.0 else 10.0 * np.log10(1.0 / mse)


# ------------------------------------------------------------ Adam comparator

def adam_update(x, g, m, v, t, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) from gradient g at step t >= 1:
    first and second moment estimates with their bias corrections
    1 - beta^t, then x - lr m_hat / (sqrt(v_hat) + eps).  Returns (x, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** t)
    v_hat = v / (1.0 - beta2 ** t)
    return x - lr * m_hat / (np.sqrt(v_hat) + eps), m, v


def adam_step(orc: Oracle, x, target, m, v, t, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8,
              do_project=True):
    """The first-order comparator of the Gauss-Newton step (the paper's Fig. 1):
    one Adam update on F (Eq. 5-6) with the gradient g = J^T r, then the
    projection.  Returns (x, m, v, F at the starting x)."""
    x = np.asarray(x, dtype=np.float64)
    r, F = orc.residual(x, target)
    g = orc.vjp(x, r)
    x, m, v = adam_update(x, g, m, v, t, lr, beta1, beta2, eps)
    return (project(x) if do_project else x), m, v, F

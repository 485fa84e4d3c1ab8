"""ctypes binding of libperf (include/perf.h): argument marshalling only.

Every step of the Gauss-Newton path runs in the CUDA library; this module
turns torch tensors into device pointers and the current torch stream into a
cudaStream_t.  It raises if the library is missing -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("PERF_LIB_PATH") or os.path.join(HERE, "libperf.so")

PERF_F32, PERF_BF16 = 0, 1
PERF_PRECOND_JACOBI, PERF_PRECOND_BLOCK4, PERF_PRECOND_BLOCK_JACOBI = 0, 1, 2
PERF_JUDGE_RESIDUAL, PERF_JUDGE_OBJECTIVE = 0, 1
PERF_ENV_EQUIRECT, PERF_ENV_CUBE = 0, 1
STATUS = {0: "PERF_OK", 1: "PERF_ERR_INVALID_ARG", 2: "PERF_ERR_CUDA",
          3: "PERF_ERR_NONFINITE", 4: "PERF_ERR_TIMEOUT", 5: "PERF_ERR_NOT_SPD",
          6: "PERF_ERR_UNSUPPORTED"}
EXIT = {0: "fixed", 1: "eps", 2: "stall", 3: "breakdown", 4: "nonfinite"}


class PerfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Scene(ctypes.Structure):
    _fields_ = [("grid_res", ctypes.c_int32), ("n_shells", ctypes.c_int32),
                ("shell_radii", ctypes.c_float * 8),
                ("env_h", ctypes.c_int32), ("env_w", ctypes.c_int32),
                ("dtype", ctypes.c_int32), ("env_kind", ctypes.c_int32)]


class Cameras(ctypes.Structure):
    _fields_ = [("n_cams", ctypes.c_int32), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32), ("c2w", ctypes.c_void_p),
                ("focal", ctypes.c_void_p)]


class Options(ctypes.Structure):
    _fields_ = [("max_samples", ctypes.c_int32), ("jitter", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("epoch", ctypes.c_uint32),
                ("pcg_iters", ctypes.c_int32), ("pcg_fixed", ctypes.c_int32),
                ("pcg_eps_rel", ctypes.c_double), ("pcg_stall", ctypes.c_double),
                ("ls_alpha", ctypes.c_double), ("ls_max", ctypes.c_int32),
                ("project", ctypes.c_int32), ("precond", ctypes.c_int32),
                ("aux", ctypes.c_int32), ("aux_lambda", ctypes.c_double),
                ("precond_judge", ctypes.c_int32)]


class PcgInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("exit_reason", ctypes.c_int32),
                ("R0", ctypes.c_double), ("R", ctypes.c_double), ("rz", ctypes.c_double)]


class Timing(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 6), ("launches", ctypes.c_int64 * 6)]


TIMING_KINDS = ("apply", "forward", "diag", "vector", "precond", "residual")


class Tuning(ctypes.Structure):
    _fields_ = [("tile_w", ctypes.c_int32), ("tile_h", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("apply_ms", ctypes.c_float),
                ("paired", ctypes.c_int32), ("coef", ctypes.c_int32),
                ("brick", ctypes.c_int32)]


class GNStats(ctypes.Structure):
    _fields_ = [("F_before", ctypes.c_double), ("F_after", ctypes.c_double),
                ("gamma", ctypes.c_double), ("accepted", ctypes.c_int32),
                ("ls_evals", ctypes.c_int32), ("pcg", PcgInfo), ("ms", ctypes.c_float),
                ("precond_fallback", ctypes.c_int32)]


_VP = ctypes.c_void_p
_SIGS = {
    "perf_default_options": [ctypes.POINTER(Options)],
    "perf_create": [ctypes.POINTER(_VP), ctypes.POINTER(Scene), ctypes.POINTER(Cameras),
                    ctypes.POINTER(Options)],
    "perf_destroy": [_VP],
    "perf_set_options": [_VP, ctypes.POINTER(Options)],
    "perf_render": [_VP, _VP, _VP, _VP, _VP],
    "perf_residual": [_VP, _VP, _VP, _VP, _VP, _VP],
    "perf_jvp": [_VP, _VP, _VP, _VP, _VP],
    "perf_vjp": [_VP, _VP, _VP, _VP, ctypes.c_int32, _VP],
    "perf_diag_jtj": [_VP, _VP, _VP, _VP, _VP, _VP],
    "perf_apply_normal": [_VP, _VP, _VP, _VP, _VP, _VP],
    "perf_pcg_begin": [_VP, _VP, _VP, _VP],
    "perf_pcg_step": [_VP, _VP, ctypes.POINTER(ctypes.c_int32), _VP],
    "perf_pcg_result": [_VP, _VP, ctypes.POINTER(PcgInfo), _VP],
    "perf_gn_solve": [_VP, _VP, _VP, ctypes.c_int32, ctypes.POINTER(GNStats), _VP],
    "perf_enable_timing": [_VP, ctypes.c_int32],
    "perf_get_timing": [_VP, ctypes.POINTER(Timing), ctypes.c_int32],
    "perf_sample_count": [_VP, ctypes.POINTER(ctypes.c_uint64), _VP],
    "perf_set_atomic_counter": [_VP, _VP],
    "perf_measure_atomic_peak": [ctypes.POINTER(ctypes.c_double)],
    "perf_pcg_set_blocks": [_VP, _VP, ctypes.c_int64],
    "perf_autotune": [_VP, _VP, _VP, ctypes.POINTER(Tuning), _VP],
    "perf_set_coef_budget": [_VP, ctypes.c_int64],
    "perf_set_brick": [_VP, ctypes.c_int32],
    "perf_set_pcg_graph": [_VP, ctypes.c_int32],
    "perf_pcg_history": [_VP, _VP, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)],
    "perf_adam_step": [_VP, _VP, _VP, _VP, _VP, ctypes.c_int32, ctypes.c_float, ctypes.c_float,
                       ctypes.c_float, ctypes.c_float, _VP, _VP],
    "perf_upsample": [_VP, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                      ctypes.c_int32, _VP, _VP],
    "perf_render_threshold": [_VP, _VP, ctypes.c_float, _VP, _VP, _VP],
    "perf_coef_info": [_VP, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32),
                       ctypes.POINTER(ctypes.c_double)],
    "perf_coef_prefix": [_VP, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64), _VP],
    "perf_set_lpc": [_VP, _VP],
    "perf_diag_cross": [_VP, _VP, _VP, _VP, _VP],
    "perf_lpc_create": [ctypes.POINTER(_VP), ctypes.c_uint64],
    "perf_lpc_destroy": [_VP],
    "perf_lpc_get_weights": [_VP, _VP],
    "perf_lpc_set_weights": [_VP, _VP],
    "perf_lpc_features": [_VP, ctypes.c_int32, _VP, _VP, _VP, _VP, _VP, _VP],
    "perf_lpc_loss_grad": [_VP, ctypes.c_int32, _VP, _VP, _VP, _VP, ctypes.POINTER(ctypes.c_double),
                           _VP, _VP],
    "perf_lpc_train_step": [_VP, ctypes.c_int32, _VP, _VP, _VP, _VP, ctypes.c_float,
                            ctypes.POINTER(ctypes.c_double), _VP],
    "perf_lpc_head_outputs": [_VP, ctypes.c_int32, _VP, _VP, _VP],
    "perf_lpc_infer": [_VP, ctypes.c_int32, _VP, _VP, _VP, _VP],
    "perf_block_jacobi": [ctypes.c_int32, _VP, _VP, _VP, _VP],
    "perf_lpc_conv_status": [ctypes.POINTER(ctypes.c_int32)],
    "perf_lpc_test_conv_wait_limit": [ctypes.c_uint32],
    "perf_lpc_dscale": [ctypes.c_int32, _VP, _VP, _VP, _VP, _VP],
    "perf_batch_create": [ctypes.POINTER(_VP), ctypes.c_int32, _VP, _VP, ctypes.POINTER(Options)],
    "perf_batch_destroy": [_VP],
    "perf_batch_render": [_VP, _VP, _VP, _VP],
    "perf_batch_residual": [_VP, _VP, _VP, _VP, _VP, _VP],
    "perf_batch_autotune": [_VP, _VP, ctypes.POINTER(Tuning), _VP],
    "perf_batch_set_coef_budget": [_VP, ctypes.c_int64],
    "perf_batch_set_brick": [_VP, ctypes.c_int32],
    "perf_batch_coef_info": [_VP, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32)],
    "perf_batch_gn_solve": [_VP, _VP, _VP, ctypes.c_int32, ctypes.POINTER(GNStats), _VP],
}
_OPTIONAL_SIGS = {
    "perf_residual_noalloc": [ctypes.POINTER(Scene), ctypes.POINTER(Cameras),
                              ctypes.POINTER(Options), _VP, _VP, _VP, _VP, _VP],
}

_lib = None


def load_library(path: Optional[str] = None):
    """Load libperf.so (raises if it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"libperf.so not built at {p}: run paper_2112_05598_gb300/build.py")
    lib = ctypes.CDLL(p)
    for name, args in _SIGS.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    for name, args in _OPTIONAL_SIGS.items():
        if hasattr(lib, name):
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = ctypes.c_int
    lib.perf_param_count.argtypes = [_VP]
    lib.perf_param_count.restype = ctypes.c_int64
    lib.perf_ray_count.argtypes = [_VP]
    lib.perf_ray_count.restype = ctypes.c_int64
    lib.perf_launch_count.argtypes = []
    lib.perf_launch_count.restype = ctypes.c_uint64
    for name in ("perf_batch_param_offset", "perf_batch_ray_offset"):
        getattr(lib, name).argtypes = [_VP, ctypes.c_int32]
        getattr(lib, name).restype = ctypes.c_int64
    lib.perf_lpc_weight_count.argtypes = []
    lib.perf_lpc_weight_count.restype = ctypes.c_int64
    lib.perf_lpc_last_error.argtypes = [_VP]
    lib.perf_lpc_last_error.restype = ctypes.c_char_p
    lib.perf_batch_last_error.argtypes = [_VP]
    lib.perf_batch_last_error.restype = ctypes.c_char_p
    lib.perf_last_error.argtypes = [_VP]
    lib.perf_last_error.restype = ctypes.c_char_p
    if path is None:
        _lib = lib
    return lib


def upsample(x, G, n_shells, env_h, env_w, x_out, stream=None, env_kind=0):
    """perf_upsample: the next hierarchical level's parameters (grid 2G, maps
    2 env_h x 2 env_w) from level (G, env_h x env_w), into x_out."""
    lib = load_library()
    st = lib.perf_upsample(_ptr(x), int(G), int(n_shells), int(env_h), int(env_w), int(env_kind),
                           _ptr(x_out),
                           _stream(stream))
    if st != 0:
        raise PerfError(st, "upsample")


def residual_noalloc(G, radii, env_h, env_w, c2w, focal, width, height, x, target, r_out,
                     F_out, dtype=PERF_F32, options: Optional[Options] = None, stream=None):
    """perf_residual_noalloc: the residual / objective march with no context and
    no device allocation (for callers that cannot allocate device memory)."""
    lib = load_library()
    sc = Scene()
    sc.grid_res = int(G)
    radii = [float(r) for r in radii]
    sc.n_shells = len(radii)
    for i, r in enumerate(radii):
        sc.shell_radii[i] = r
    sc.env_h, sc.env_w = int(env_h), int(env_w)
    sc.dtype = int(dtype)
    c2w = np.ascontiguousarray(c2w, dtype=np.float32).reshape(-1, 12)
    focal = np.ascontiguousarray(focal, dtype=np.float32).reshape(-1)
    cams = Cameras()
    cams.n_cams = int(c2w.shape[0])
    cams.width, cams.height = int(width), int(height)
    cams.c2w = c2w.ctypes.data_as(ctypes.c_void_p)
    cams.focal = focal.ctypes.data_as(ctypes.c_void_p)
    o = options if options is not None else default_options()
    st = lib.perf_residual_noalloc(ctypes.byref(sc), ctypes.byref(cams), ctypes.byref(o),
                                   _ptr(x), _ptr(target), _ptr(r_out), _ptr(F_out),
                                   _stream(stream))
    if st != 0:
        raise PerfError(st, "perf_residual_noalloc rejected its arguments or failed")


def launch_count() -> int:
    """Kernels launched by libperf in this process so far."""
    return int(load_library().perf_launch_count())


def measure_atomic_peak() -> float:
    """Best rate (lane operations/s) of 16-byte global vector atomic adds on
    the current device, from the library's microbenchmark (synchronises)."""
    v = ctypes.c_double(0.0)
    st = load_library().perf_measure_atomic_peak(ctypes.byref(v))
    if st != 0:
        raise PerfError(st, "perf_measure_atomic_peak failed")
    return float(v.value)


def default_options(**kw) -> Options:
    o = Options()
    load_library().perf_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Context:
    """One scene + camera set (``perf_create``).  Methods take torch CUDA
    tensors and run on the current torch stream unless one is given."""

    def __init__(self, G, radii, env_h, env_w, c2w, focal, width, height,
                 dtype=PERF_F32, options: Optional[Options] = None, env_kind=0, **opt_kw):
        self.lib = load_library()
        sc = Scene()
        sc.grid_res = int(G)
        radii = [float(r) for r in radii]
        sc.n_shells = len(radii)
        for i, r in enumerate(radii):
            sc.shell_radii[i] = r
        sc.env_h, sc.env_w = int(env_h), int(env_w)
        sc.dtype = int(dtype)
        sc.env_kind = int(env_kind)
        self.env_kind = int(env_kind)
        self._c2w = np.ascontiguousarray(c2w, dtype=np.float32).reshape(-1, 12)
        self._focal = np.ascontiguousarray(focal, dtype=np.float32).reshape(-1)
        cams = Cameras()
        cams.n_cams = int(self._c2w.shape[0])
        cams.width, cams.height = int(width), int(height)
        cams.c2w = self._c2w.ctypes.data_as(ctypes.c_void_p)
        cams.focal = self._focal.ctypes.data_as(ctypes.c_void_p)
        self.options = options if options is not None else default_options()
        for k, v in opt_kw.items():
            setattr(self.options, k, v)
        h = ctypes.c_void_p()
        st = self.lib.perf_create(ctypes.byref(h), ctypes.byref(sc), ctypes.byref(cams),
                                  ctypes.byref(self.options))
        if st != 0:
            raise PerfError(st, "perf_create rejected the scene, cameras or options")
        self.h = h
        self.dtype = dtype
        self.G, self.n_shells, self.env_h, self.env_w = int(G), len(radii), int(env_h), int(env_w)
        self.width, self.height, self.n_cams = int(width), int(height), cams.n_cams
        self.n_params = int(self.lib.perf_param_count(h))
        self.n_rays = int(self.lib.perf_ray_count(h))

    @property
    def n_res(self):
        """Residuals per ray: 3, or 4 with the auxiliary opacity term."""
        return 4 if self.options.aux else 3

    @classmethod
    def from_scene(cls, scene, dtype=PERF_F32, c2w=None, focal=None, **opt_kw):
        opt_kw.setdefault("max_samples", scene.cfg.max_samples)
        opt_kw.setdefault("env_kind", getattr(scene, "env_kind", 0))
        return cls(scene.G, scene.radii, scene.env_h, scene.env_w,
                   scene.c2w if c2w is None else c2w,
                   scene.focal if focal is None else focal,
                   scene.width, scene.height, dtype=dtype, **opt_kw)

    def close(self):
        if getattr(self, "h", None):
            self.lib.perf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        if st != 0:
            msg = self.lib.perf_last_error(self.h)
            raise PerfError(st, f"{what}: {msg.decode() if msg else ''}")

    def set_options(self, **kw):
        for k, v in kw.items():
            setattr(self.options, k, v)
        self._check(self.lib.perf_set_options(self.h, ctypes.byref(self.options)), "set_options")

    # --- per-call entry points (device tensors)
    def render_threshold(self, x, min_opacity, rgb_out, T_out=None, stream=None):
        """Rendering with the converged-scene opacity threshold (rays whose
        volume opacity 1 - T is below min_opacity see only the shells)."""
        self._check(self.lib.perf_render_threshold(self.h, _ptr(x), float(min_opacity),
                                                   _ptr(rgb_out), _ptr(T_out), _stream(stream)),
                    "render_threshold")

    def render(self, x, rgb_out, T_out=None, stream=None):
        self._check(self.lib.perf_render(self.h, _ptr(x), _ptr(rgb_out), _ptr(T_out),
                                         _stream(stream)), "render")

    def residual(self, x, target, r_out, F_out, stream=None):
        self._check(self.lib.perf_residual(self.h, _ptr(x), _ptr(target), _ptr(r_out),
                                           _ptr(F_out), _stream(stream)), "residual")

    def jvp(self, x, p, out, stream=None):
        self._check(self.lib.perf_jvp(self.h, _ptr(x), _ptr(p), _ptr(out), _stream(stream)), "jvp")

    def vjp(self, x, v, out, accumulate=False, stream=None):
        self._check(self.lib.perf_vjp(self.h, _ptr(x), _ptr(v), _ptr(out), int(accumulate),
                                      _stream(stream)), "vjp")

    def diag_jtj(self, x, diag_out, r=None, grad_out=None, stream=None):
        self._check(self.lib.perf_diag_jtj(self.h, _ptr(x), _ptr(r), _ptr(diag_out),
                                           _ptr(grad_out), _stream(stream)), "diag_jtj")

    def apply_normal(self, x, p, ap_out, pap_out=None, stream=None):
        self._check(self.lib.perf_apply_normal(self.h, _ptr(x), _ptr(p), _ptr(ap_out),
                                               _ptr(pap_out), _stream(stream)), "apply_normal")

    def pcg_begin(self, grad, diag, stream=None):
        self._check(self.lib.perf_pcg_begin(self.h, _ptr(grad), _ptr(diag), _stream(stream)),
                    "pcg_begin")

    def pcg_step(self, x, want_done=False, stream=None):
        done = ctypes.c_int32(0)
        self._check(self.lib.perf_pcg_step(self.h, _ptr(x), ctypes.byref(done) if want_done else None,
                                           _stream(stream)), "pcg_step")
        return bool(done.value) if want_done else None

    def pcg_result(self, delta_out=None, stream=None):
        info = PcgInfo()
        self._check(self.lib.perf_pcg_result(self.h, _ptr(delta_out), ctypes.byref(info),
                                             _stream(stream)), "pcg_result")
        return dict(iters=info.iters, exit=EXIT.get(info.exit_reason, info.exit_reason),
                    R0=info.R0, R=info.R, rz=info.rz)

    def set_blocks(self, blocks, n_block):
        self._check(self.lib.perf_pcg_set_blocks(self.h, _ptr(blocks), int(n_block)), "set_blocks")

    def autotune(self, x, p=None, stream=None):
        t = Tuning()
        self._check(self.lib.perf_autotune(self.h, _ptr(x), _ptr(p), ctypes.byref(t),
                                           _stream(stream)), "autotune")
        return dict(tile_w=t.tile_w, tile_h=t.tile_h, ctas_per_sm=t.ctas_per_sm, apply_ms=t.apply_ms,
                    paired=t.paired, coef=t.coef, brick=t.brick)

    def adam_step(self, x, target, m, v, t, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8,
                  F_out=None, stream=None):
        """One Adam step on F with g = J^T r (in place on x, m, v); F_out gets F(x)."""
        self._check(self.lib.perf_adam_step(self.h, _ptr(x), _ptr(target), _ptr(m), _ptr(v),
                                            int(t), float(lr), float(beta1), float(beta2),
                                            float(eps), _ptr(F_out), _stream(stream)), "adam_step")

    def pcg_history(self, cap=100000):
        """R = r_k^T r_k after each iteration of the last PCG solve (numpy)."""
        out = np.zeros(max(int(cap), 1))
        k = ctypes.c_int32(0)
        self._check(self.lib.perf_pcg_history(self.h, out.ctypes.data_as(ctypes.c_void_p), int(cap),
                                              ctypes.byref(k)), "pcg_history")
        return out[:k.value].copy()

    def set_coef_budget(self, nbytes):
        """Budget of the coefficient store: -1 automatic, 0 off, > 0 bytes."""
        self._check(self.lib.perf_set_coef_budget(self.h, int(nbytes)), "set_coef_budget")

    def set_brick(self, edge):
        """Block order of a Gauss-Newton step's PCG vectors: 1 canonical, 2, 4
        or 8 voxels per brick edge (perf_set_brick)."""
        self._check(self.lib.perf_set_brick(self.h, int(edge)), "set_brick")

    def set_pcg_graph(self, on=True):
        """Replay a fixed-iteration PCG loop from a CUDA graph (default on)."""
        self._check(self.lib.perf_set_pcg_graph(self.h, int(bool(on))), "set_pcg_graph")

    def coef_info(self):
        b = ctypes.c_int64(0)
        u = ctypes.c_int32(0)
        c = ctypes.c_double(0.0)
        self._check(self.lib.perf_coef_info(self.h, ctypes.byref(b), ctypes.byref(u), ctypes.byref(c)),
                    "coef_info")
        return dict(bytes=int(b.value), used=bool(u.value), coverage=float(c.value))

    def coef_prefix(self, stream=None):
        """perf_coef_prefix: after a Gauss-Newton step that used the store,
        the grid-sample rows its A p reads (each ray's non-zero prefix) and
        the grid samples of the store's rays."""
        r = ctypes.c_int64(0)
        t = ctypes.c_int64(0)
        self._check(self.lib.perf_coef_prefix(self.h, ctypes.byref(r), ctypes.byref(t),
                                              _stream(stream)), "coef_prefix")
        return dict(read=int(r.value), total=int(t.value))

    def set_lpc(self, lpc):
        self._lpc = lpc
        self._check(self.lib.perf_set_lpc(self.h, lpc.h if lpc is not None else None), "set_lpc")

    def diag_cross(self, x, diag_out, cross_out, stream=None):
        self._check(self.lib.perf_diag_cross(self.h, _ptr(x), _ptr(diag_out), _ptr(cross_out),
                                             _stream(stream)), "diag_cross")

    def set_atomic_counter(self, counter=None):
        """Count the J^T scatter's vector-atomic lane operations into a
        zeroed int64 device tensor of one element (None: stop counting)."""
        if counter is not None:
            assert counter.is_cuda and counter.numel() >= 1 and counter.element_size() == 8
        self._check(self.lib.perf_set_atomic_counter(self.h, _ptr(counter) if counter is not None
                                                     else None), "set_atomic_counter")

    def sample_count(self, stream=None):
        n = ctypes.c_uint64(0)
        self._check(self.lib.perf_sample_count(self.h, ctypes.byref(n), _stream(stream)), "sample_count")
        return int(n.value)

    def enable_timing(self, on=True):
        self._check(self.lib.perf_enable_timing(self.h, int(bool(on))), "enable_timing")

    def timing(self, reset=False):
        t = Timing()
        self._check(self.lib.perf_get_timing(self.h, ctypes.byref(t), int(bool(reset))), "timing")
        return {k: dict(ms=t.ms[i], launches=int(t.launches[i])) for i, k in enumerate(TIMING_KINDS)}

    def gn_solve(self, x, target, n_steps, stream=None):
        stats = (GNStats * max(int(n_steps), 1))()
        self._check(self.lib.perf_gn_solve(self.h, _ptr(x), _ptr(target), int(n_steps), stats,
                                           _stream(stream)), "gn_solve")
        out = []
        for i in range(int(n_steps)):
            s = stats[i]
            out.append(dict(F_before=s.F_before, F_after=s.F_after, gamma=s.gamma,
                            accepted=bool(s.accepted), ls_evals=s.ls_evals,
                            pcg_iters=s.pcg.iters, pcg_exit=EXIT.get(s.pcg.exit_reason),
                            R0=s.pcg.R0, R=s.pcg.R, ms=s.ms,
                            precond_fallback=bool(s.precond_fallback)))
        return out


class Batch:
    """Many independent scenes solved together (``perf_batch_*``).  ``scenes``
    is a list of dicts with G, radii, env_h, env_w, c2w, focal, width, height."""

    def __init__(self, scenes, options: Optional[Options] = None, **opt_kw):
        self.lib = load_library()
        n = len(scenes)
        sc_arr = (Scene * n)()
        cam_arr = (Cameras * n)()
        self._keep = []
        for i, d in enumerate(scenes):
            radii = [float(r) for r in d["radii"]]
            sc_arr[i].grid_res = int(d["G"])
            sc_arr[i].n_shells = len(radii)
            for j, r in enumerate(radii):
                sc_arr[i].shell_radii[j] = r
            sc_arr[i].env_h, sc_arr[i].env_w = int(d["env_h"]), int(d["env_w"])
            sc_arr[i].dtype = PERF_F32
            sc_arr[i].env_kind = int(d.get("env_kind", 0))
            c2w = np.ascontiguousarray(d["c2w"], dtype=np.float32).reshape(-1, 12)
            focal = np.ascontiguousarray(d["focal"], dtype=np.float32).reshape(-1)
            self._keep += [c2w, focal]
            cam_arr[i].n_cams = int(c2w.shape[0])
            cam_arr[i].width, cam_arr[i].height = int(d["width"]), int(d["height"])
            cam_arr[i].c2w = c2w.ctypes.data_as(ctypes.c_void_p)
            cam_arr[i].focal = focal.ctypes.data_as(ctypes.c_void_p)
        self.options = options if options is not None else default_options()
        for k, v in opt_kw.items():
            setattr(self.options, k, v)
        h = ctypes.c_void_p()
        st = self.lib.perf_batch_create(ctypes.byref(h), n, ctypes.cast(sc_arr, ctypes.c_void_p),
                                        ctypes.cast(cam_arr, ctypes.c_void_p),
                                        ctypes.byref(self.options))
        if st != 0:
            raise PerfError(st, "perf_batch_create rejected the scenes or options")
        self.h = h
        self.n = n
        self.param_off = [int(self.lib.perf_batch_param_offset(h, i)) for i in range(n + 1)]
        self.ray_off = [int(self.lib.perf_batch_ray_offset(h, i)) for i in range(n + 1)]
        self.n_params = self.param_off[-1]
        self.n_rays = self.ray_off[-1]

    def close(self):
        if getattr(self, "h", None):
            self.lib.perf_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        if st != 0:
            msg = self.lib.perf_batch_last_error(self.h)
            raise PerfError(st, f"{what}: {msg.decode() if msg else ''}")

    def render(self, x, rgb_out, stream=None):
        self._check(self.lib.perf_batch_render(self.h, _ptr(x), _ptr(rgb_out), _stream(stream)),
                    "batch render")

    def residual(self, x, target, r_out, F_out, stream=None):
        self._check(self.lib.perf_batch_residual(self.h, _ptr(x), _ptr(target), _ptr(r_out),
                                                 _ptr(F_out), _stream(stream)), "batch residual")

    def autotune(self, x, stream=None):
        t = Tuning()
        self._check(self.lib.perf_batch_autotune(self.h, _ptr(x), ctypes.byref(t), _stream(stream)),
                    "batch autotune")
        return dict(tile_w=t.tile_w, tile_h=t.tile_h, ctas_per_sm=t.ctas_per_sm, apply_ms=t.apply_ms,
                    coef=t.coef, brick=t.brick)

    def set_coef_budget(self, nbytes):
        """Budget of the coefficient store: -1 automatic, 0 off, > 0 bytes."""
        self._check(self.lib.perf_batch_set_coef_budget(self.h, int(nbytes)), "batch set_coef_budget")

    def set_brick(self, edge):
        """perf_batch_set_brick: brick edge 1, 2, 4 or 8 for the scenes whose G
        allows it."""
        self._check(self.lib.perf_batch_set_brick(self.h, int(edge)), "batch set_brick")

    def coef_info(self):
        b = ctypes.c_int64(0)
        u = ctypes.c_int32(0)
        self._check(self.lib.perf_batch_coef_info(self.h, ctypes.byref(b), ctypes.byref(u)),
                    "batch coef_info")
        return dict(bytes=int(b.value), used=bool(u.value))

    def gn_solve(self, x, target, n_steps, stream=None):
        stats = (GNStats * max(int(n_steps) * self.n, 1))()
        self._check(self.lib.perf_batch_gn_solve(self.h, _ptr(x), _ptr(target), int(n_steps), stats,
                                                 _stream(stream)), "batch gn_solve")
        out = []
        for k in range(int(n_steps)):
            out.append([dict(F_before=s.F_before, F_after=s.F_after, gamma=s.gamma,
                             accepted=bool(s.accepted), ls_evals=s.ls_evals,
                             pcg_iters=s.pcg.iters, pcg_exit=EXIT.get(s.pcg.exit_reason),
                             ms=s.ms)
                        for s in stats[k * self.n:(k + 1) * self.n]])
        return out


class LPC:
    """Learned block preconditioner (``perf_lpc_*``): a 4-layer 3x3x3 conv net
    trained and run by the library's own BF16 kernels."""

    def __init__(self, seed=0):
        self.lib = load_library()
        h = ctypes.c_void_p()
        st = self.lib.perf_lpc_create(ctypes.byref(h), ctypes.c_uint64(int(seed)))
        if st != 0:
            raise PerfError(st, "perf_lpc_create failed")
        self.h = h
        self.n_weights = int(self.lib.perf_lpc_weight_count())

    def close(self):
        if getattr(self, "h", None):
            self.lib.perf_lpc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        if st != 0:
            msg = self.lib.perf_lpc_last_error(self.h)
            raise PerfError(st, f"{what}: {msg.decode() if msg else ''}")

    def get_weights(self):
        w = np.zeros(self.n_weights, np.float32)
        self._check(self.lib.perf_lpc_get_weights(self.h, w.ctypes.data_as(ctypes.c_void_p)),
                    "get_weights")
        return w

    def set_weights(self, w):
        w = np.ascontiguousarray(w, dtype=np.float32)
        assert w.shape[0] == self.n_weights
        self._check(self.lib.perf_lpc_set_weights(self.h, w.ctypes.data_as(ctypes.c_void_p)),
                    "set_weights")

    def features(self, G, x, grad, diag, cross, feat_out, stream=None):
        self._check(self.lib.perf_lpc_features(self.h, int(G), _ptr(x), _ptr(grad), _ptr(diag),
                                               _ptr(cross), _ptr(feat_out), _stream(stream)),
                    "features")

    def loss_grad(self, G, feat, ahat, xi, mask=None, grad_out=None, stream=None):
        loss = ctypes.c_double(0.0)
        self._check(self.lib.perf_lpc_loss_grad(self.h, int(G), _ptr(feat), _ptr(ahat), _ptr(xi),
                                                _ptr(mask), ctypes.byref(loss), _ptr(grad_out),
                                                _stream(stream)), "loss_grad")
        return loss.value

    def train_step(self, G, feat, ahat, xi, mask=None, lr=1e-3, stream=None):
        loss = ctypes.c_double(0.0)
        self._check(self.lib.perf_lpc_train_step(self.h, int(G), _ptr(feat), _ptr(ahat), _ptr(xi),
                                                 _ptr(mask), ctypes.c_float(lr), ctypes.byref(loss),
                                                 _stream(stream)), "train_step")
        return loss.value

    def head_outputs(self, G, feat, out, stream=None):
        self._check(self.lib.perf_lpc_head_outputs(self.h, int(G), _ptr(feat), _ptr(out),
                                                   _stream(stream)), "head_outputs")

    def infer(self, G, feat, diag, blocks_out, stream=None):
        self._check(self.lib.perf_lpc_infer(self.h, int(G), _ptr(feat), _ptr(diag),
                                            _ptr(blocks_out), _stream(stream)), "infer")


def conv_status() -> int:
    """1 if a convolution of the preconditioner network gave up a bounded wait
    since the last call (its outputs are incomplete), else 0; clears the flag."""
    v = ctypes.c_int32(0)
    st = load_library().perf_lpc_conv_status(ctypes.byref(v))
    if st != 0:
        raise PerfError(st, "perf_lpc_conv_status failed")
    return int(v.value)


def set_conv_wait_limit_for_test(rounds: int):
    """Test hook: polling rounds of each convolution CTA's first TMA wait in
    later launches (0 makes it give up at once; 1 << 20 is the default)."""
    load_library().perf_lpc_test_conv_wait_limit(ctypes.c_uint32(int(rounds)))


def dscale(G, diag, inp, out, mask_out=None, stream=None):
    st = load_library().perf_lpc_dscale(int(G), _ptr(diag), _ptr(inp), _ptr(out), _ptr(mask_out),
                                        _stream(stream))
    if st != 0:
        raise PerfError(st, "perf_lpc_dscale failed")


def block_jacobi(G, diag, cross, blocks_out, stream=None):
    st = load_library().perf_block_jacobi(int(G), _ptr(diag), _ptr(cross), _ptr(blocks_out),
                                          _stream(stream))
    if st != 0:
        raise PerfError(st, "perf_block_jacobi failed")

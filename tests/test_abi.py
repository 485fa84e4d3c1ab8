"""The C ABI without a GPU: libperf.so loads, exports every entry point that
include/perf.h declares, and rejects invalid arguments before any launch."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def _declared():
    names = set()
    for h in HEADERS:
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(perf_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2112_05598_gb300 import _binding
    return _binding.load_library()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "perf_gn_solve" in names and len(names) >= 15
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_default_options(lib):
    from paper_2112_05598_gb300 import default_options
    o = default_options()
    assert o.ls_alpha == 0.7 and o.pcg_stall == 0.85 and o.ls_max == 20 and o.project == 1


def _create(lib, G=8, radii=(2.0,), env=(4, 8), n_cams=1, res=8, focal=10.0, dtype=0, **opt):
    from paper_2112_05598_gb300 import _binding as B
    sc = B.Scene()
    sc.grid_res = G
    sc.n_shells = len(radii)
    for i, r in enumerate(radii):
        sc.shell_radii[i] = r
    sc.env_h, sc.env_w = env
    sc.dtype = dtype
    c2w = np.zeros((max(n_cams, 1), 12), np.float32)
    fo = np.full(max(n_cams, 1), focal, np.float32)
    cams = B.Cameras()
    cams.n_cams, cams.width, cams.height = n_cams, res, res
    cams.c2w = c2w.ctypes.data_as(ctypes.c_void_p)
    cams.focal = fo.ctypes.data_as(ctypes.c_void_p)
    o = B.default_options(**opt)
    h = ctypes.c_void_p()
    st = lib.perf_create(ctypes.byref(h), ctypes.byref(sc), ctypes.byref(cams), ctypes.byref(o))
    if st == 0:
        lib.perf_destroy(h)
    return st


@pytest.mark.parametrize("kw", [
    dict(G=1), dict(G=0), dict(radii=(1.5,)), dict(radii=(3.0, 2.5)), dict(env=(1, 8)),
    dict(n_cams=-1), dict(focal=0.0), dict(focal=float("nan")), dict(dtype=7),
    dict(max_samples=0), dict(ls_alpha=1.0), dict(precond=9), dict(pcg_iters=-2),
    dict(radii=(2.0,) * 9),
])
def test_create_rejects_invalid_arguments(lib, kw):
    if "radii" in kw and len(kw["radii"]) > 8:
        from paper_2112_05598_gb300 import _binding as B
        sc = B.Scene()
        sc.grid_res = 4
        sc.n_shells = 9
        st = lib.perf_create(ctypes.byref(ctypes.c_void_p()), ctypes.byref(sc),
                             ctypes.byref(B.Cameras()), ctypes.byref(B.default_options()))
        assert st == 1
        return
    assert _create(lib, **kw) == 1


def test_null_arguments_rejected(lib):
    assert lib.perf_create(None, None, None, None) == 1
    assert lib.perf_destroy(None) == 1
    assert lib.perf_render(None, None, None, None, None) == 1
    assert lib.perf_gn_solve(None, None, None, 1, None, None) == 1
    assert lib.perf_param_count(None) == -1


def test_package_fails_loudly_without_library(tmp_path):
    from paper_2112_05598_gb300 import _binding
    with pytest.raises(ImportError):
        _binding.load_library(str(tmp_path / "missing.so"))

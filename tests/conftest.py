import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")


def has_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def pytest_collection_modifyitems(config, items):
    if has_gpu():
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


def tiny_problem(rng, G=3, radii=(2.5,), env_h=4, env_w=8, n_cams=2, res=4,
                 cam_radius=3.2, sigma=(0.2, 2.0), shell_sigma=(0.2, 1.5),
                 max_samples=64):
    """A tiny seeded problem: random parameters, cameras on a sphere."""
    from scenegen import make_cameras, random_params
    c2w, focal = make_cameras(rng, n_cams, res, cam_radius, "sphere", 40.0)
    x = random_params(rng, G, len(radii), env_h, env_w, sigma[0], sigma[1],
                      shell_sigma_hi=shell_sigma[1])
    return dict(G=G, radii=radii, env_h=env_h, env_w=env_w, c2w=c2w,
                focal=focal, width=res, height=res, max_samples=max_samples,
                x=x)


def rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (den if den > 0 else 1.0))


def pytest_sessionstart(session):
    """Build the CUDA library and the oracle before collection imports them."""
    import __graft_entry__
    __graft_entry__.build()

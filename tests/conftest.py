import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a GB300 (CUDA) device")


def pytest_collection_modifyitems(config, items):
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)


def crit_distance(a, lam, eta, samples=2001):
    """Distance of photons with constants (lam, eta) from the Kerr critical curve (Bardeen 1973):
    min over the spherical-photon-orbit radii r of |R(r)| / r^4, where
    R(r) = (r^2 + a^2 - a lam)^2 - (r^2 - 2 r + a^2) (eta + (lam - a)^2) is the radial potential
    (M = E = 1).  A critical photon has a double root of R there, so the distance is 0 on the curve."""
    import numpy as np
    lam = np.asarray(lam, dtype=np.float64)[:, None]
    eta = np.asarray(eta, dtype=np.float64)[:, None]
    aa = abs(a)
    r_pro = 2 * (1 + np.cos(2 / 3 * np.arccos(-aa)))
    r_ret = 2 * (1 + np.cos(2 / 3 * np.arccos(aa)))
    r = np.linspace(r_pro, r_ret, samples)[None, :]
    R = (r * r + a * a - a * lam) ** 2 - (r * r - 2 * r + a * a) * (eta + (lam - a) ** 2)
    return np.min(np.abs(R) / r ** 4, axis=1)


@pytest.fixture
def near_critical():
    """near_critical(a, info) -> bool per ray: the oracle's constants of motion lie within 0.03
    (the library's near-critical band width) of the critical curve."""
    def flag(a, info, width=0.03):
        return crit_distance(a, info["lam"], info["eta"]) < width
    return flag

"""Shared test helpers: one problem spec feeds both the oracle and the library binding."""
from __future__ import annotations

import numpy as np

from paper_2309_12019_gb300 import inputs as I


def spec(dim, p, n, ny=None, flux="advect", stab="weno", bc="periodic", **kw):
    """A problem description with square cells of size 1/n (box grows with nx, ny)."""
    ny = ny if ny is not None else n
    h = 1.0 / n
    s = dict(dim=dim, nx=n, p=p, ny=ny if dim == 2 else 1, box=(0.0, n * h, 0.0, ny * h),
             bc=(bc,) * 4, flux=flux, stab=stab)
    if flux == "advect":
        s["a"] = (0.9, -0.6)
    elif flux == "burgers":
        s["a"] = (1.0, 1.0) if dim == 2 else (1.0, 0.0)
    elif flux == "rotation":
        s["center"] = (0.5 * n * h, 0.5 * ny * h)
        s["omega"] = 1.0
    elif flux == "kpp":
        s["lambda_nu"] = 2.0
    s.update(kw)
    return s


def state_for(s, seed, smooth=True):
    """Seeded random modal state suited to the flux (KPP values spread over [0, 11])."""
    E = s["nx"] * (s["ny"] if s["dim"] == 2 else 1)
    if s["flux"] == "kpp":
        return I.random_state(s["dim"], s["p"], E, seed, smooth=smooth, scale=3.0, offset=5.0)
    return I.random_state(s["dim"], s["p"], E, seed, smooth=smooth, scale=1.0, offset=0.2)


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))

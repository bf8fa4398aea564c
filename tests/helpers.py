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


def cell_err(got, ref):
    """Largest per-cell error: max over cells e of ||got[:, e] - ref[:, e]||_2, over the
    root-mean-square cell norm of ref.  A single wrong cell shows at its own size here,
    where a global relative L2 would divide it by sqrt(E)."""
    a = np.asarray(got, dtype=np.float64)
    b = np.asarray(ref, dtype=np.float64)
    scale = max(float(np.sqrt(np.mean(np.sum(b * b, axis=0)))), 1e-300)
    return float(np.max(np.linalg.norm(a - b, axis=0)) / scale)


# Float error bound of the sensor ratio r = ||U - U*||_e / ||U||_e in the float kernels:
# the sensor tests hold |gamma_fp32 - gamma_oracle| <= 1e-4 wherever gamma = min(1, r).
R_FLOAT_ERR = 1e-4


def near_threshold(O, s, U, delta=R_FLOAT_ERR):
    """Cells where the oracle's sensor ratio lies within delta of the threshold b of
    Eq. (gensensor): there the float kernel may take the other side of r < b (gamma 0
    against gamma ~ b).  All False unless the problem's sensor is WENO with b > 0."""
    P = O.Problem(**s)
    if P.stab != "weno" or not P.b > 0:
        return np.zeros(P.E, dtype=bool)
    _, r, _ = O.sensor(P, U)
    return np.abs(r - P.b) < delta

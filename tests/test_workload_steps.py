"""The time steps of the synthetic workloads against the explicit stability bound of the
stabilization term (Sec. 3, Eq. astab), which dominates at gamma = 1.

In physical units the term gamma nu_e M^{-1} K, nu_e = lambda h / (2p), has per direction
the eigenvalues 2 gamma lambda mu / (p h), mu those of the reference pencil (int P_i' P_j',
int P_i P_j) on [-1, 1]; in 2D the directions add.  SSP-RK3 is stable on the negative real
axis up to the root x* of |1 - x + x^2/2 - x^3/6| = 1.  Nothing here comes from the library
or the oracle: Legendre polynomials and Gauss rules are NumPy's.
"""
import numpy as np
import pytest

import bench
from paper_2309_12019_gb300 import inputs as I


def _mu_max(p):
    """Largest eigenvalue of M^{-1} A on the Legendre basis of degree p."""
    x, w = np.polynomial.legendre.leggauss(p + 2)
    P = np.array([np.polynomial.legendre.legval(x, np.eye(p + 1)[i]) for i in range(p + 1)])
    D = np.array([np.polynomial.legendre.legval(x, np.polynomial.legendre.legder(np.eye(p + 1)[i]))
                  for i in range(p + 1)])
    A = (D * w) @ D.T
    M = (P * w) @ P.T
    return float(np.max(np.linalg.eigvals(np.linalg.solve(M, A)).real))


def _rk3_axis_bound():
    R = lambda z: 1 + z + z * z / 2 + z ** 3 / 6
    lo, hi = 2.0, 3.0               # |R(-2)| < 1 < |R(-3)|
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if abs(R(-mid)) <= 1 else (lo, mid)
    return lo


def test_stabilization_radii_match_the_stated_values():
    """2 mu_max / p = 6, 15, 28.3 for p = 1, 2, 3 (the per-direction radii, in units of
    gamma lambda / h, that the workload steps are chosen against), and x* = 2.5127."""
    for p, want in ((1, 6.0), (2, 15.0), (3, 28.3)):
        assert abs(2 * _mu_max(p) / p - want) < 0.05 * want, p
    assert abs(_rk3_axis_bound() - 2.5127) < 1e-3


def _lambda_bound(w):
    if w.get("lambda_nu", 0.0) > 0:
        return w["lambda_nu"]
    if w["flux"] == "rotation":       # |omega (cy - y, x - cx)| over the box
        x0, x1, y0, y1 = w["box"]
        cx, cy = w["center"]
        return w["omega"] * max(np.hypot(x - cx, y - cy) for x in (x0, x1) for y in (y0, y1))
    return max(w["speeds"])


@pytest.mark.parametrize("name", sorted(bench.WORKLOADS))
def test_bench_workload_steps_are_stable(name):
    w = bench.WORKLOADS[name]
    if w["stab"] == "dg":
        pytest.skip("no stabilization term")
    h = (w["box"][1] - w["box"][0]) / w["nx"]
    radius = w["dim"] * 2 * _mu_max(w["p"]) / w["p"] * _lambda_bound(w) * bench.dt_of(w) / h
    assert radius < _rk3_axis_bound(), (name, radius)


def test_ensemble_instance_steps_are_stable():
    for d in I.ensemble_instances(512):
        h = 1.0 / d["nx"]
        lam = max(abs(d["a"][0]), abs(d["a"][1])) if d["flux"] == "advect" else \
            float(np.sum(d["init"]["amp"])) + len(d["init"]["lo"])
        radius = d["dim"] * 2 * _mu_max(d["p"]) / d["p"] * lam * d["dt"] / h
        assert radius < _rk3_axis_bound(), (d["dim"], d["p"], d["nx"], radius)

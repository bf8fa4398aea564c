"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

No GPU.  Each test names the passage it pins.  The pins are chosen so that a plausible
slip anywhere in the oracle (a dropped term, a wrong sign or index, a transposed
operand) breaks at least one of them:

* closed forms: Legendre values, Gauss rules, the seminorm Gram matrix, the stiffness
  and mass matrices, the p = 0 upwind scheme, the SSP-RK3 stability polynomial;
* invariants stated in the paper: LLF consistency and conservation (Sec. 2), gamma in
  [0, 1] (Sec. 3), b = 0 recovering Eq. (sensor) (Sec. 4), mass conservation;
* invariants of the definitions: polynomial reproduction (gamma = 0), shift invariance,
  mirror symmetry;
* an independent brute-force evaluation (tests/bruteforce.py) on 4-cell meshes;
* the paper's printed L1 errors (Tables 1 and 2, DG and LO columns) and EOCs.
"""
import functools
import math
import os

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

import bruteforce
from paper_2309_12019_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------------------
# closed forms
# ---------------------------------------------------------------------------------------

def test_legendre_matches_numpy(oracle_mod):
    O = oracle_mod
    for n in range(6):
        for a in range(4):
            c = np.zeros(n + 1)
            c[n] = 1
            ref = npleg.legval(0.37, npleg.legder(c, a) if a else c)
            assert abs(O.legendre(n, a, 0.37) - ref) < 1e-13


def test_gauss_rule_matches_numpy(oracle_mod):
    for n in (1, 2, 3, 5, 8, 24):
        x, w = oracle_mod.gauss_legendre(n)
        xr, wr = npleg.leggauss(n)
        assert np.max(np.abs(x - xr)) < 1e-14 and np.max(np.abs(w - wr)) < 1e-14


def _A(p, a):
    """A^(a)_mn = int_{-1}^{1} P_m^(a) P_n^(a): closed form for a <= 1, NumPy otherwise."""
    A = np.zeros((p + 1, p + 1))
    for m in range(p + 1):
        for n in range(p + 1):
            if a == 0:
                A[m, n] = 2.0 / (2 * m + 1) if m == n else 0.0
            elif a == 1:
                k = min(m, n)
                A[m, n] = k * (k + 1) if (m + n) % 2 == 0 else 0.0
            else:
                cm = np.zeros(m + 1); cm[m] = 1
                cn = np.zeros(n + 1); cn[n] = 1
                prod = npleg.legmul(npleg.legder(cm, a) if m >= a else [0], npleg.legder(cn, a) if n >= a else [0])
                integ = npleg.legint(prod)
                A[m, n] = npleg.legval(1.0, integ) - npleg.legval(-1.0, integ)
    return A


def _gram(dim, p):
    """G = sum_{1<=|k|<=p} 2^{2|k|-d} (x)_i A^(k_i): the scaled seminorm on square cells."""
    if dim == 1:
        return sum(2.0 ** (2 * k - 1) * _A(p, k) for k in range(1, p + 1))
    G = np.zeros(((p + 1) ** 2,) * 2)
    for ky in range(p + 1):
        for kx in range(p + 1):
            if 1 <= kx + ky <= p:
                # mode k = i + (p+1) j  ->  kron(A_y, A_x)
                G += 2.0 ** (2 * (kx + ky) - 2) * np.kron(_A(p, ky), _A(p, kx))
    return G


@pytest.mark.parametrize("dim,p", [(1, 1), (1, 2), (1, 3), (2, 1), (2, 2), (2, 3)])
def test_seminorm_closed_form(oracle_mod, dim, p):
    """Sec. 4 scaled Sobolev seminorm equals c^T G c and does not depend on h."""
    O = oracle_mod
    rng = np.random.default_rng(1 + p + 10 * dim)
    G = _gram(dim, p)
    for n in (4, 7):
        P = O.Problem(dim=dim, nx=n, ny=n, p=p, box=(0, 3.0, 0, 3.0))
        for _ in range(3):
            c = rng.standard_normal(P.K)
            assert abs(O.seminorm2(P, c) - c @ G @ c) < 1e-11 * max(1.0, c @ G @ c)


def test_seminorm_1d_linear(oracle_mod):
    """|| a + b xi ||_e = 2|b| for p = 1 in 1D (h^{1} * int (2b/h)^2 dx = 4 b^2)."""
    P = oracle_mod.Problem(dim=1, nx=5, p=1)
    assert abs(oracle_mod.seminorm2(P, np.array([0.7, -1.3])) - 4 * 1.69) < 1e-13


@pytest.mark.parametrize("dim,p", [(1, 1), (1, 2), (1, 3), (2, 1), (2, 2), (2, 3)])
def test_stiffness_and_mass_closed_form(oracle_mod, dim, p):
    """Eq. (lostab) with F = 0 and a fixed lambda: L = -nu M^{-1} K c, nu = lambda h/(2p)
    (Eq. visc), K = (2/h) A1 in 1D and A1(x)A0 + A0(x)A1 in 2D, M = (h/2)^d diag(2/(2i+1))."""
    O = oracle_mod
    n, lam = 6, 1.7
    P = O.Problem(dim=dim, nx=n, ny=n, p=p, box=(0, 2.0, 0, 2.0), flux="advect", a=(0.0, 0.0),
                  stab="lo", lambda_nu=lam)
    h = 2.0 / n
    U = I.random_state(dim, p, P.E, seed=5)
    L = O.residual(P, U)
    A0, A1 = _A(p, 0), _A(p, 1)
    if dim == 1:
        K = (2.0 / h) * A1
        M = (h / 2) * A0
    else:
        K = np.kron(A0, A1) + np.kron(A1, A0)
        M = (h / 2) ** 2 * np.kron(A0, A0)
    nu = lam * h / (2 * p)
    ref = -nu * np.linalg.solve(M, K @ U)
    assert np.max(np.abs(L - ref)) < 1e-10 * np.max(np.abs(ref))
    assert np.max(np.abs(L[0])) < 1e-12  # row 0 of K vanishes: no mass is created


@pytest.mark.parametrize("a", [1.3, -0.7])
def test_p0_is_upwind_finite_volume(oracle_mod, a):
    """DG with p = 0 and the LLF flux is the first-order upwind finite-volume scheme."""
    O = oracle_mod
    P = O.Problem(dim=1, nx=9, p=0, a=(a, 0.0), stab="dg")
    u = np.random.default_rng(3).standard_normal(9)
    L = O.residual(P, u[None, :])[0]
    h = 1.0 / 9
    ref = -a * (u - np.roll(u, 1)) / h if a > 0 else -a * (np.roll(u, -1) - u) / h
    assert np.max(np.abs(L - ref)) < 1e-12 * np.max(np.abs(ref))


def test_rk3_stability_polynomial(oracle_mod):
    """Eq. (ssp) applied to a linear operator L equals I + dt L + dt^2 L^2/2 + dt^3 L^3/6."""
    O = oracle_mod
    P = O.Problem(dim=2, nx=5, ny=5, p=2, flux="advect", a=(0.6, -0.3), stab="lo")
    U = I.random_state(2, 2, P.E, seed=11)
    dt = 0.013
    L1 = O.residual(P, U)
    L2 = O.residual(P, L1)
    L3 = O.residual(P, L2)
    ref = U + dt * L1 + dt ** 2 / 2 * L2 + dt ** 3 / 6 * L3
    out = O.rk3(P, U, dt, 1)
    assert np.max(np.abs(out - ref)) < 1e-12 * np.max(np.abs(ref))


# ---------------------------------------------------------------------------------------
# numerical flux (Sec. 2)
# ---------------------------------------------------------------------------------------

FLUXES = [dict(flux="advect", a=(0.8, -1.1)), dict(flux="rotation", omega=1.0),
          dict(flux="burgers", a=(1.0, 1.0)), dict(flux="kpp")]


@pytest.mark.parametrize("fl", FLUXES, ids=lambda f: f["flux"])
def test_llf_consistency_and_conservation(oracle_mod, fl):
    O = oracle_mod
    P = O.Problem(dim=2, nx=2, ny=2, p=1, **fl)
    rng = np.random.default_rng(7)
    for _ in range(200):
        u, v = rng.uniform(-12, 12, 2)
        x, y = rng.uniform(0, 1, 2)
        for n in [(1.0, 0.0), (0.0, 1.0), (-1.0, 0.0), (0.0, -1.0)]:
            if fl["flux"] == "advect":
                F = (fl["a"][0] * u, fl["a"][1] * u)
            elif fl["flux"] == "rotation":
                F = ((0.5 - y) * u, (x - 0.5) * u)
            elif fl["flux"] == "burgers":
                F = (0.5 * u * u, 0.5 * u * u)
            else:
                F = (math.sin(u), math.cos(u))
            assert abs(O.llf(P, u, u, x, y, *n) - (F[0] * n[0] + F[1] * n[1])) < 1e-12 * (1 + abs(u) ** 2)
            assert abs(O.llf(P, u, v, x, y, *n) + O.llf(P, v, u, x, y, -n[0], -n[1])) < 1e-11 * (1 + u * u + v * v)


def test_kpp_wave_speed_is_segment_maximum(oracle_mod):
    """s+ = max over the segment of |F'(w).n| (Sec. 2): compare with a dense sample."""
    O = oracle_mod
    P = O.Problem(dim=2, nx=2, ny=2, p=1, flux="kpp")
    rng = np.random.default_rng(9)
    for _ in range(300):
        u, v = rng.uniform(-12, 12, 2) * rng.choice([1.0, 0.05])
        w = np.linspace(0, 1, 20001)
        s = w * u + (1 - w) * v
        for n, g in [((1.0, 0.0), np.abs(np.cos(s))), ((0.0, 1.0), np.abs(np.sin(s)))]:
            exact = O.wave_speed(P, u, v, 0.3, 0.3, *n)
            assert exact >= g.max() - 1e-15
            assert exact <= g.max() + 2e-7


# ---------------------------------------------------------------------------------------
# sensor (Sec. 4)
# ---------------------------------------------------------------------------------------

def test_sensor_worked_example_1d_p1(oracle_mod):
    """1D, p = 1: candidates of a + b xi are a + b_L xi and a + b_R xi (continuation of a
    linear function keeps its slope), beta = 4 b^2, linear weights 0.98 / 0.01 / 0.01
    (Sec. 5).  Slopes (0.9, 1, 1.1) give w = (0.977974, 0.015210, 0.006816) and
    gamma = 2|1 - b*| / 2 = 8.394052e-4; a step cell (0, 0.5, 0) gives gamma = 1 - 4.9e-11."""
    O = oracle_mod
    P = O.Problem(dim=1, nx=3, p=1, stab="weno", b=0.0)
    g, r, w = O.sensor(P, np.array([[0.0, 0.0, 0.0], [0.9, 1.0, 1.1]]))
    assert np.allclose(w[1, :3], [0.977974, 0.015210, 0.006816], atol=2e-6)
    assert abs(g[1] - 8.394052e-4) < 1e-9
    g, r, w = O.sensor(P, np.array([[0.0, 0.3, 0.0], [0.0, 0.5, 0.0]]))
    assert abs((1 - g[1]) - 4.9e-11) < 0.1e-11


def test_zhao_sensor_worked_values_1d_p1(oracle_mod):
    """The comparison sensor of Zhao et al. restated in Sec. 5.6 (theta = 1), by hand on
    1D p = 1 cells.  (i) Slopes (0.9, 1, 1.1): weights (0.977974, 0.015210, 0.006816)
    against linear weights (0.98, 0.01, 0.01) give (0.0020673 + 0.5210 + 0.3184) / (99 + 2)
    = 8.33136e-3.  (ii) A step cell between two constant cells: both neighbour candidates
    are flat, each takes half of the weight: (1 + 49 + 49) / 101 = 99/101.  (iii) Flat
    left neighbour, steep right one: all weight on the left candidate, the one of smallest
    linear weight: (1 + 99 + 1) / 101 = 1."""
    O = oracle_mod
    P = O.Problem(dim=1, nx=3, p=1, stab="zhao")
    g, _, _ = O.sensor(P, np.array([[0.0, 0.0, 0.0], [0.9, 1.0, 1.1]]))
    assert abs(g[1] - 8.33136e-3) < 3e-6
    g, _, _ = O.sensor(P, np.array([[0.0, 0.3, 0.0], [0.0, 0.5, 0.0]]))
    assert abs(g[1] - 99.0 / 101.0) < 1e-9
    g, _, _ = O.sensor(P, np.array([[0.0, 0.3, 0.0], [0.0, 0.5, 3.0]]))
    assert abs(g[1] - 1.0) < 1e-9


@pytest.mark.parametrize("dim,p", [(1, 2), (2, 1), (2, 3)])
def test_zhao_sensor_range_invariance_and_polynomials(oracle_mod, dim, p):
    """gamma^Z lies in [0, 1] (the denominator is the value for all weight on the candidate
    of smallest linear weight), ignores constants, and vanishes up to round-off on global
    polynomials (equal indicators make the weights the linear ones)."""
    O = oracle_mod
    n = 6
    P = O.Problem(dim=dim, nx=n, ny=n, p=p, stab="zhao")
    U = I.random_state(dim, p, P.E, seed=23, smooth=True)
    g, _, _ = O.sensor(P, U)
    U2 = U.copy()
    U2[0] += 2.9
    g2, _, _ = O.sensor(P, U2)
    assert np.all((g >= 0) & (g <= 1)) and np.any(g > 1e-2)
    assert np.max(np.abs(g - g2)) < 1e-12
    Pp = O.Problem(dim=dim, nx=n, ny=n, p=p, box=(-1.0, 1.5, -1.0, 1.5), bc=("outflow",) * 4, stab="zhao")
    X, Y = I.sample_points(dim, n, n, Pp.box, 8)
    f = 0.3 + X - 0.7 * X ** p + (0.5 * Y ** p if dim == 2 else 0.0)
    gp, _, _ = O.sensor(Pp, O.project(Pp, f))
    assert np.max(np.abs(gp)) < 1e-13


@pytest.mark.parametrize("dim,p", [(1, 1), (1, 2), (1, 3), (2, 1), (2, 2), (2, 3)])
def test_polynomial_reproduction(oracle_mod, dim, p):
    """Any global polynomial of V_p is reproduced by every Hermite candidate, so U* = U_h,
    gamma = 0 and the WENO residual equals the plain DG residual."""
    O = oracle_mod
    n = 5
    P = O.Problem(dim=dim, nx=n, ny=n, p=p, box=(-1.0, 1.5, -1.0, 1.5), bc=("outflow",) * 4,
                  flux="advect", a=(0.7, 0.4), stab="weno")
    X, Y = I.sample_points(dim, n, n, P.box, 8)
    rng = np.random.default_rng(p)
    cf = rng.standard_normal((p + 1, p + 1))
    f = sum(cf[i, j] * X ** i * (Y ** j if dim == 2 else (j == 0)) for i in range(p + 1) for j in range(p + 1))
    U = O.project(P, f)
    g, r, _ = O.sensor(P, U)
    assert np.all(g == 0.0), (g.max(), r.max())
    for e in range(P.E):
        for face in range(2 * dim):
            cl = O.candidate(P, U, e, face)
            if cl is not None:
                assert np.max(np.abs(cl - U[:, e])) < 1e-11 * (1 + np.max(np.abs(U)))
    Pd = O.Problem(**{**P.__dict__, "stab": "dg"})
    assert np.max(np.abs(O.residual(P, U) - O.residual(Pd, U))) < 1e-12 * np.max(np.abs(O.residual(Pd, U)))


@pytest.mark.parametrize("dim,p", [(1, 2), (2, 1), (2, 3)])
def test_sensor_shift_invariance_and_range(oracle_mod, dim, p):
    """gamma(U + c) = gamma(U) (the seminorm ignores constants, candidates keep the mean)
    and gamma in [0, 1] (Sec. 3)."""
    O = oracle_mod
    n = 6
    P = O.Problem(dim=dim, nx=n, ny=n, p=p, b=0.0)
    U = I.random_state(dim, p, P.E, seed=21, smooth=True)
    g, r, w = O.sensor(P, U)
    U2 = U.copy()
    U2[0] += 3.7
    g2, _, _ = O.sensor(P, U2)
    assert np.max(np.abs(g - g2)) < 1e-12
    assert np.all((g >= 0) & (g <= 1))
    assert np.allclose(w.sum(axis=1), 1.0)
    assert np.any(g > 1e-3) and np.any(g < 1)


def test_threshold_b_zero_recovers_sensor(oracle_mod):
    """Eq. (gensensor): b = 0 gives Eq. (sensor); b > 0 zeroes exactly the ratios below b."""
    O = oracle_mod
    P = O.Problem(dim=2, nx=6, ny=6, p=2, b=0.0)
    U = I.random_state(2, 2, P.E, seed=4, smooth=True)
    g0, r0, _ = O.sensor(P, U)
    Pb = O.Problem(**{**P.__dict__, "b": 0.3})
    gb, rb, _ = O.sensor(Pb, U)
    assert np.array_equal(r0, rb)
    assert np.array_equal(gb, np.where(r0 < 0.3, 0.0, g0))
    assert np.array_equal(g0, np.minimum(1.0, r0))


def _reflect_x(U, dim, p, nx, ny):
    K = (p + 1) ** dim
    i = np.arange(K) % (p + 1)
    V = U * ((-1.0) ** i)[:, None]
    if dim == 1:
        return V[:, ::-1]
    return V.reshape(K, ny, nx)[:, :, ::-1].reshape(K, -1)


@pytest.mark.parametrize("dim,flux,stab", [(1, "burgers", "weno"), (2, "advect", "weno"), (2, "advect", "lo")])
def test_mirror_symmetry(oracle_mod, dim, flux, stab):
    """Reflecting x -> -x (and the x-velocity) reflects gamma and the residual."""
    O = oracle_mod
    n, p = 6, 2
    P = O.Problem(dim=dim, nx=n, ny=n, p=p, box=(-1, 1, -1, 1), flux=flux, a=(0.8, 0.5), stab=stab)
    Pm = O.Problem(**{**P.__dict__, "a": (-0.8, 0.5)})
    U = I.random_state(dim, p, P.E, seed=8, smooth=True)
    Ur = _reflect_x(U, dim, p, n, n)
    g, _, _ = O.sensor(P, U)
    gr, _, _ = O.sensor(P, Ur)
    gr_back = _reflect_x(gr[None, :], dim, 0, n, n)[0]
    assert np.max(np.abs(g - gr_back)) < 1e-12
    if flux == "burgers":
        # Burgers is odd under u -> -u together with x -> -x
        L = O.residual(P, U)
        Lr = O.residual(P, -Ur)
        assert np.max(np.abs(-_reflect_x(Lr, dim, p, n, n) - L)) < 1e-10 * np.max(np.abs(L))
    else:
        L = O.residual(P, U)
        Lr = O.residual(Pm, Ur)
        assert np.max(np.abs(_reflect_x(Lr, dim, p, n, n) - L)) < 1e-10 * np.max(np.abs(L))


# ---------------------------------------------------------------------------------------
# conservation and brute force
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("dim,flux,stab", [(1, "burgers", "weno"), (1, "advect", "lo"),
                                           (2, "advect", "weno"), (2, "burgers", "weno"),
                                           (2, "kpp", "weno"), (2, "rotation", "dg")])
def test_mass_conservation_periodic(oracle_mod, dim, flux, stab):
    """On periodic meshes the LLF flux is conservative and row 0 of the stabilization
    vanishes (grad phi_0 = 0), so the total mass is constant to round-off."""
    O = oracle_mod
    n, p = 7, 2
    P = O.Problem(dim=dim, nx=n, ny=n, p=p, flux=flux, a=(1.0, 0.5), stab=stab,
                  lambda_nu=2.0 if flux == "kpp" else 0.0)
    U = I.random_state(dim, p, P.E, seed=13, smooth=True, offset=1.0)
    m0 = O.mass(P, U)
    U1 = O.rk3(P, U, 0.002, 5)
    assert abs(O.mass(P, U1) - m0) < 1e-13 * (1 + abs(m0)) * P.E


BF_CASES = [
    (1, p, fl, st, bc) for p in (1, 2, 3) for fl in ("advect", "burgers") for st in ("dg", "lo", "weno")
    for bc in ("periodic", "outflow")
] + [(1, 2, "advect", "weno", "inflow_zero"), (1, 2, "burgers", "zhao", "outflow"), (1, 3, "advect", "zhao", "periodic"),
       (2, 2, "advect", "zhao", "periodic"), (2, 3, "rotation", "zhao", "inflow_zero")] + [
    (2, p, fl, st, bc) for p in (1, 2, 3) for fl in ("advect", "rotation") for st in ("lo", "weno")
    for bc in ("periodic", "inflow_zero")
]


@pytest.mark.parametrize("dim,p,flux,stab,bc", BF_CASES)
def test_bruteforce_agreement(oracle_mod, dim, p, flux, stab, bc):
    """Independent evaluation from the definitions (24-point Gauss, NumPy Legendre) on
    4-cell / 4x4 meshes agrees to round-off for polynomial fluxes (exact quadrature)."""
    O = oracle_mod
    P = O.Problem(dim=dim, nx=4, ny=4, p=p, bc=(bc,) * 4, flux=flux, a=(0.9, -0.6), stab=stab)
    U = I.random_state(dim, p, P.E, seed=31 + p, smooth=True, scale=0.8, offset=0.3)
    L = O.residual(P, U)
    Lb = bruteforce.residual(P, U)
    assert np.max(np.abs(L - Lb)) < 1e-12 * np.max(np.abs(Lb))
    if stab in ("weno", "zhao"):
        g, _, _ = O.sensor(P, U)
        assert np.max(np.abs(g - bruteforce.sensor(P, U))) < 1e-12


# ---------------------------------------------------------------------------------------
# paper tables (Sec. 5.1, 5.2)
# ---------------------------------------------------------------------------------------

def _load_tables():
    rows = []
    with open(os.path.join(GOLDEN, "paper_tables_l1.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                t, p, E, dg, lo, weno = line.split()
                rows.append((t, int(p), int(E), float(dg), float(lo), float(weno)))
    return rows


def exact_burgers(x, t):
    """sin(2 pi x) under Burgers before the shock: solve u = sin(2 pi (x - u t)) by Newton."""
    u = np.sin(2 * np.pi * x)
    for _ in range(60):
        g = u - np.sin(2 * np.pi * (x - u * t))
        dg = 1 + 2 * np.pi * t * np.cos(2 * np.pi * (x - u * t))
        u = u - g / dg
    return u


@functools.lru_cache(maxsize=None)
def run_1d(O, test, p, E, stab, lambda_nu=0.0, cfl=0.05, b=None):
    """L1 error at t_end of one run of Table 1 (advect) or Table 2 (burgers); b = None is
    the Problem's default threshold.  Cached: several pins share runs."""
    flux, t_end, u0 = ("advect", 1.0, I.u0_cos) if test == "advect" else ("burgers", 0.1, I.u0_sin)
    P = O.Problem(dim=1, nx=E, p=p, flux=flux, stab=stab, a=(1.0, 0.0), lambda_nu=lambda_nu, b=b)
    X, _ = I.sample_points(1, E, 1, P.box, 8)
    U = O.project(P, u0(X))
    n, dt, last = I.nsteps_to(t_end, I.cfl_dt(cfl if p < 3 else 0.02, [1.0], [1.0 / E]))
    U = O.rk(P, U, dt, n, p + 1 if p >= 1 else 3)      # SSP-RK of order p + 1, as in Sec. 5
    if last > 0:
        U = O.rk(P, U, last, 1, p + 1 if p >= 1 else 3)
    ex = u0(X - t_end) if test == "advect" else exact_burgers(X, t_end)
    return O.l1_error(P, U, ex)


@pytest.mark.parametrize("test", ["advect", "burgers"])
@pytest.mark.parametrize("p", [1, 2, 3])
def test_paper_tables_dg_lo(oracle_mod, test, p):
    """Tables 1-2 (Sec. 5.1-5.2), E = 16, 32, 64.

    Both sides integrate with SSP-RK of order p + 1.  LO is dominated by the O(h)
    viscosity and matches to 3 %.  For Burgers the paper's LO numbers come out with
    lambda_e = 1 (the global bound of |F'(u)| = |u| for sin(2 pi x)); the element-wise
    maximum is 15-25 % less dissipative.  DG matches to 25 %: the time scheme moves these
    errors by under 0.5 % (order 3 against p + 1), so the difference is spatial, the
    paper's Lagrange nodes (nodal initial data) against the L2 projection here."""
    O = oracle_mod
    rows = [r for r in _load_tables() if r[0] == test and r[1] == p and r[2] <= 64]
    for _, _, E, dg, lo, _ in rows:
        e_lo = run_1d(O, test, p, E, "lo", lambda_nu=1.0 if test == "burgers" else 0.0)
        assert abs(e_lo / lo - 1) < 0.03, (E, e_lo, lo)
        e_dg = run_1d(O, test, p, E, "dg")
        assert abs(e_dg / dg - 1) < 0.25, (E, e_dg, dg)


@pytest.mark.parametrize("test", ["advect", "burgers"])
@pytest.mark.parametrize("p", [1, 2, 3])
def test_paper_tables_weno_column(oracle_mod, test, p):
    """The WENO columns of Tables 1-2 with the threshold b = 0.1 of Eq. (gensensor)
    (reading R5, the tolerance of the remark in Sec. 4).  The paper prints WENO = DG to
    its three digits for p = 2, 3 on every mesh, and for p = 1 from 256 cells on, with
    WENO above DG on the coarser p = 1 meshes (Table 1: 10x DG at 16 cells, 1.8x at 128;
    Table 2: 1.8x at 16 cells).  The oracle: WENO within 2 % of DG at p = 2, 3 (16-64
    cells; p = 3 Table 1 to 32), WENO over 1.2x DG at p = 1 on 16-64 cells and within 2 %
    of DG at 256 cells; and the WENO values within the DG column's 25 % of the paper's
    WENO column where the paper prints WENO = DG.  The unthresholded sensor (b = 0) fails
    this: its WENO error is 1.7-50x DG at p = 2, 3 (checked at 16 cells)."""
    O = oracle_mod
    rows = {r[2]: r for r in _load_tables() if r[0] == test and r[1] == p}
    Es = [16, 32] if (p == 3 and test == "advect") else [16, 32, 64]
    for E in Es:
        dg, weno = run_1d(O, test, p, E, "dg"), run_1d(O, test, p, E, "weno")
        if p == 1:
            assert weno > 1.2 * dg, (E, weno, dg)
        else:
            assert abs(weno / dg - 1) < 0.02, (E, weno, dg)
            assert abs(weno / rows[E][5] - 1) < 0.25, (E, weno, rows[E][5])
    if p == 1:
        dg, weno = run_1d(O, test, 1, 256, "dg"), run_1d(O, test, 1, 256, "weno")
        assert abs(weno / dg - 1) < 0.02, (weno, dg)
        assert abs(weno / rows[256][5] - 1) < 0.25, (weno, rows[256][5])
    else:
        dg, w0 = run_1d(O, test, p, 16, "dg"), run_1d(O, test, p, 16, "weno", b=0.0)
        assert w0 > 1.5 * dg, (w0, dg)


@pytest.mark.parametrize("test", ["advect", "burgers"])
def test_sensor_ratio_below_threshold_on_smooth_data(oracle_mod, test):
    """Why the WENO column equals DG (Tables 1-2): on the L2 projection of the exact
    solution at t_end (cos for Table 1, the Burgers solution at t = 0.1 for Table 2) the
    sensor ratio ||U - U*||_e / ||U||_e stays below b = 0.1 in every cell for p = 2 on
    16-2048 cells and p = 3 on 16-512 (the paper's meshes), and for p = 1 from 256 cells
    on; on 16-64 cells at p = 1 it exceeds b somewhere (the p = 1 WENO errors there are
    above DG's, as in the paper).  So gamma^b = 0 and the stabilized residual is the
    plain DG residual on these states."""
    O = oracle_mod
    t_end, f = (1.0, lambda x: I.u0_cos(x - 1.0)) if test == "advect" else \
        (0.1, lambda x: exact_burgers(x, 0.1))
    flux = "advect" if test == "advect" else "burgers"
    for p, Es in ((1, (16, 32, 64, 256, 512, 1024, 2048)), (2, (16, 32, 64, 128, 256, 512, 1024, 2048)),
                  (3, (16, 32, 64, 128, 256, 512))):
        for E in Es:
            P = O.Problem(dim=1, nx=E, p=p, flux=flux, a=(1.0, 0.0))
            assert P.b == 0.1
            X, _ = I.sample_points(1, E, 1, P.box, 8)
            g, r, _ = O.sensor(P, O.project(P, f(X)))
            if p == 1 and E <= 64:
                assert np.max(r) > P.b, (p, E)
            else:
                assert np.max(r) < P.b and np.all(g == 0.0), (p, E, np.max(r))


@pytest.mark.parametrize("p", [1, 2, 3])
def test_eoc_smooth_advection(oracle_mod, p):
    """Optimal EOC ~ p + 1 (Table 1) for DG and for WENO (rate at least p + 0.8) on the
    finest meshes these pins run: 128 -> 256 cells at p = 1 (where the paper's WENO
    column reaches DG), 32 -> 64 -> 128 at p = 2, 16 -> 32 at p = 3."""
    O = oracle_mod
    Es = {1: [128, 256], 2: [32, 64, 128], 3: [16, 32]}[p]
    for stab in ("dg", "weno"):
        e = [run_1d(O, "advect", p, E, stab) for E in Es]
        for e1, e2 in zip(e, e[1:]):
            eoc = math.log(e1 / e2) / math.log(2)
            assert eoc > p + 0.8, (stab, e, eoc)


# ---------------------------------------------------------------------------------------
# SSP Runge-Kutta of order p + 1 (Sec. 5 convergence studies; reading R14)
# ---------------------------------------------------------------------------------------

def _operator_matrix(O, P):
    """Matrix of a linear residual (DG advection) by its action on unit vectors."""
    n = P.K * P.E
    A = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        A[:, j] = O.residual(P, e.reshape(P.K, P.E)).reshape(-1)
    return A


@pytest.mark.parametrize("order", [2, 3, 4])
def test_ssp_rk_one_step_error_on_linear_operator(oracle_mod, order):
    """One step of each scheme on the linear DG advection operator against the exact
    propagator exp(dt A) (SciPy): the error falls like dt^(order + 1) when dt halves."""
    expm = pytest.importorskip("scipy.linalg").expm
    O = oracle_mod
    P = O.Problem(dim=1, nx=6, p=2, flux="advect", a=(1.0, 0.0), stab="dg")
    A = _operator_matrix(O, P)
    U = I.random_state(1, 2, P.E, seed=41, smooth=True)
    errs = []
    for dt in (4e-3, 2e-3):
        exact = expm(dt * A) @ U.reshape(-1)
        errs.append(np.linalg.norm(O.rk(P, U, dt, 1, order).reshape(-1) - exact))
    rate = np.log2(errs[0] / errs[1])
    assert abs(rate - (order + 1)) < 0.25, (order, errs, rate)


@pytest.mark.parametrize("order", [2, 3, 4])
def test_ssp_rk_global_order_on_burgers(oracle_mod, order):
    """Global time error of the nonlinear DG Burgers system (smooth data, no
    stabilization) against a 32x finer step of the same scheme: it falls like dt^order,
    which checks the nonlinear order conditions as well."""
    O = oracle_mod
    P = O.Problem(dim=1, nx=8, p=2, flux="burgers", stab="dg")
    X, _ = I.sample_points(1, 8, 1, P.box, 8)
    U0 = O.project(P, 0.5 + 0.3 * np.sin(2 * np.pi * X))
    T = 0.1
    ref = O.rk(P, U0, T / 512, 512, order)
    errs = [np.linalg.norm(O.rk(P, U0, T / n, n, order) - ref) for n in (16, 32)]
    rate = np.log2(errs[0] / errs[1])
    assert abs(rate - order) < 0.3, (order, errs, rate)


def test_rk_order_three_is_eq_ssp(oracle_mod):
    O = oracle_mod
    P = O.Problem(dim=2, nx=5, ny=5, p=2, flux="burgers", a=(1.0, 1.0))
    U = I.random_state(2, 2, P.E, seed=43, smooth=True)
    assert np.array_equal(O.rk(P, U, 1e-3, 3, 3), O.rk3(P, U, 1e-3, 3))

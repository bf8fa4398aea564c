"""Python access to the plain FP64 CPU oracle (``dgw_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()`` and by
the CPU-baseline leg of ``bench.py``.  The CUDA library never imports, links or calls it,
and this module imports nothing from the library.

The oracle follows the paper section by section (Sec. 2 DG residual with the local
Lax-Friedrichs flux, Sec. 3 dissipative stabilization, Sec. 4 WENO sensor, Eq. (ssp)
SSP-RK3); the readings taken where the paper is silent are listed at the top of
``dgw_oracle.c``.

State arrays are NumPy float64 of shape ``(K, E)`` (mode-major, element e = iy*nx + ix,
mode k = i + (p+1)*j).
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dgw_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

BC = {"periodic": 0, "inflow_zero": 1, "outflow": 2, "reflect": 3, "state": 4}

# Threshold b of Eq. (gensensor) when none is given (reading R5): the remark of Sec. 4
# switches the sensor off below a prescribed tolerance, and b = 0.1 (the smaller of the
# two values Sec. 5.6 names) reproduces the WENO columns of Tables 1-2 (WENO = DG for
# p = 2, 3; for p = 1 from 256 cells).  The Euler runs of Sec. 5.6 use the unmodified
# sensor gamma_e (b = 0) and treat b > 0 as the variant to compare.
B_SCALAR = 0.1
B_EULER = 0.0
FLUX = {"advect": 0, "rotation": 1, "burgers": 2, "kpp": 3, "euler": 4}
STAB = {"dg": 0, "lo": 1, "weno": 2, "zhao": 3}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP if available).  Returns the library path."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-D_DEFAULT_SOURCE"]
    tmp = _LIB + f".{os.getpid()}.tmp"
    try:
        subprocess.run(base + ["-fopenmp", _SRC, "-o", tmp, "-lm"], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + [_SRC, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Problem(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("p", ctypes.c_int),
        ("x0", ctypes.c_double), ("x1", ctypes.c_double),
        ("y0", ctypes.c_double), ("y1", ctypes.c_double),
        ("bc", ctypes.c_int * 4),
        ("flux", ctypes.c_int),
        ("a", ctypes.c_double * 2), ("center", ctypes.c_double * 2),
        ("omega", ctypes.c_double), ("lambda_nu", ctypes.c_double),
        ("stab", ctypes.c_int),
        ("q", ctypes.c_double), ("b", ctypes.c_double), ("w_nbr", ctypes.c_double),
        ("eps_w", ctypes.c_double), ("eps_s", ctypes.c_double),
        ("theta", ctypes.c_double), ("gas_gamma", ctypes.c_double),
        ("t", ctypes.c_double), ("bstate", (ctypes.c_double * 4) * 2),
        ("bsplit", ctypes.c_double * 4), ("bspeed", ctypes.c_double * 4),
        ("bbelow", ctypes.c_int * 4), ("babove", ctypes.c_int * 4),
    ]


@dataclasses.dataclass
class Problem:
    """Mesh, degree, flux and stabilization of one scalar conservation law."""
    dim: int
    nx: int
    p: int
    ny: int = 1
    box: tuple = (0.0, 1.0, 0.0, 1.0)
    bc: tuple = ("periodic",) * 4
    flux: str = "advect"
    a: tuple = (1.0, 0.0)
    center: tuple = (0.5, 0.5)
    omega: float = 1.0
    lambda_nu: float = 0.0
    stab: str = "weno"
    q: float = 1.0
    b: float = None          # None: B_SCALAR for the scalar laws, B_EULER for the Euler system
    w_nbr: float = 1e-2
    eps_w: float = 1e-6
    eps_s: float = 1e-12
    theta: float = 1.0
    gas_gamma: float = 1.4
    # prescribed boundary states (Euler, bc "state", reading R19): the time of the
    # evaluation, two conservative states, and per side the split position along the side
    # at t = 0, its speed, and the ghost below / from it (0, 1: bstate[0], [1]; 2: wall)
    t: float = 0.0
    bstate: tuple = ((0.0, 0.0, 0.0, 0.0), (0.0, 0.0, 0.0, 0.0))
    bsplit: tuple = (0.0, 0.0, 0.0, 0.0)
    bspeed: tuple = (0.0, 0.0, 0.0, 0.0)
    bbelow: tuple = (0, 0, 0, 0)
    babove: tuple = (0, 0, 0, 0)

    def __post_init__(self):
        if self.b is None:
            self.b = B_EULER if self.flux == "euler" else B_SCALAR

    @property
    def E(self) -> int:
        return self.nx * (self.ny if self.dim == 2 else 1)

    @property
    def K(self) -> int:
        """Rows of the state: modes per element, times dim + 2 components for the Euler system."""
        return (self.p + 1) ** self.dim * self.ncomp

    @property
    def ncomp(self) -> int:
        return self.dim + 2 if self.flux == "euler" else 1

    @property
    def h(self) -> float:
        return (self.box[1] - self.box[0]) / self.nx

    def _c(self) -> _Problem:
        s = _Problem()
        s.dim, s.nx, s.ny, s.p = self.dim, self.nx, self.ny if self.dim == 2 else 1, self.p
        s.x0, s.x1, s.y0, s.y1 = [float(v) for v in self.box]
        for i, b in enumerate(self.bc):
            s.bc[i] = BC[b]
        s.flux = FLUX[self.flux]
        s.a[0], s.a[1] = self.a
        s.center[0], s.center[1] = self.center
        s.omega, s.lambda_nu = self.omega, self.lambda_nu
        s.stab = STAB[self.stab]
        s.q, s.b, s.w_nbr, s.eps_w, s.eps_s = self.q, self.b, self.w_nbr, self.eps_w, self.eps_s
        s.theta = self.theta
        s.gas_gamma = self.gas_gamma
        s.t = self.t
        for i in range(2):
            for c in range(4):
                s.bstate[i][c] = self.bstate[i][c]
        for f in range(4):
            s.bsplit[f], s.bspeed[f] = self.bsplit[f], self.bspeed[f]
            s.bbelow[f], s.babove[f] = self.bbelow[f], self.babove[f]
        return s


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            pp = ctypes.POINTER(_Problem)
            L.orc_check.argtypes = [pp]
            L.orc_residual.argtypes = [pp, dp, dp]
            L.orc_sensor.argtypes = [pp, dp, dp, dp, dp]
            L.orc_lambda.argtypes = [pp, dp, dp]
            L.orc_rk3.argtypes = [pp, dp, ctypes.c_double, ctypes.c_int]
            L.orc_rk2.argtypes = [pp, dp, ctypes.c_double, ctypes.c_int]
            L.orc_rk4.argtypes = [pp, dp, ctypes.c_double, ctypes.c_int]
            L.orc_project.argtypes = [pp, ctypes.c_int, dp, dp]
            L.orc_l1_error.argtypes = [pp, dp, ctypes.c_int, dp]
            L.orc_l1_error.restype = ctypes.c_double
            L.orc_eval.argtypes = [pp, dp, ctypes.c_int, dp]
            L.orc_mass.argtypes = [pp, dp]
            L.orc_mass.restype = ctypes.c_double
            L.orc_seminorm2.argtypes = [pp, dp]
            L.orc_seminorm2.restype = ctypes.c_double
            L.orc_candidate.argtypes = [pp, dp, ctypes.c_long, ctypes.c_int, dp]
            L.orc_llf.argtypes = [pp] + [ctypes.c_double] * 6
            L.orc_llf.restype = ctypes.c_double
            L.orc_euler_llf.argtypes = [pp, dp, dp, ctypes.c_double, dp]
            L.orc_euler_llf2.argtypes = [pp, dp, dp, ctypes.c_double, ctypes.c_double, dp]
            L.orc_wave_speed.argtypes = [pp] + [ctypes.c_double] * 6
            L.orc_wave_speed.restype = ctypes.c_double
            L.orc_legendre.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double]
            L.orc_legendre.restype = ctypes.c_double
            L.orc_gauss_legendre.argtypes = [ctypes.c_int, dp, dp]
            lp = ctypes.POINTER(ctypes.c_long)
            L.orc_residual_at.argtypes = [pp, dp, lp, ctypes.c_long, dp]
            L.orc_sensor_at.argtypes = [pp, dp, lp, ctypes.c_long, dp]
            L.orc_set_threads.argtypes = [ctypes.c_int]
            L.orc_get_threads.restype = ctypes.c_int
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _state(P: Problem, U) -> np.ndarray:
    U = np.ascontiguousarray(np.asarray(U, dtype=np.float64))
    if U.shape != (P.K, P.E):
        raise ValueError(f"state shape {U.shape} != {(P.K, P.E)}")
    return U


def _checked(P: Problem) -> _Problem:
    c = P._c()
    if lib().orc_check(ctypes.byref(c)) != 0:
        raise ValueError(f"oracle rejects problem {P}")
    return c


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return lib().orc_get_threads()


def residual(P: Problem, U) -> np.ndarray:
    """L = M^{-1} R_stab(U) (Eq. weak2 plus the stabilization of Sec. 3)."""
    c, U = _checked(P), _state(P, U)
    L = np.zeros_like(U)
    lib().orc_residual(ctypes.byref(c), _ptr(U), _ptr(L))
    return L


def residual_at(P: Problem, U, idx) -> np.ndarray:
    """Residual of the elements listed in idx only: shape (K, len(idx))."""
    c, U = _checked(P), _state(P, U)
    idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int64))
    out = np.zeros((P.K, idx.size))
    lib().orc_residual_at(ctypes.byref(c), _ptr(U), idx.ctypes.data_as(ctypes.POINTER(ctypes.c_long)),
                          idx.size, _ptr(out))
    return out


def sensor_at(P: Problem, U, idx) -> np.ndarray:
    c, U = _checked(P), _state(P, U)
    idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int64))
    out = np.zeros(idx.size)
    lib().orc_sensor_at(ctypes.byref(c), _ptr(U), idx.ctypes.data_as(ctypes.POINTER(ctypes.c_long)),
                        idx.size, _ptr(out))
    return out


def sensor(P: Problem, U):
    """Returns (gamma, ratio, weights[E,5]) of the WENO sensor (Sec. 4)."""
    c, U = _checked(P), _state(P, U)
    g = np.zeros(P.E)
    r = np.zeros(P.E)
    w = np.zeros((P.E, 5))
    lib().orc_sensor(ctypes.byref(c), _ptr(U), _ptr(g), _ptr(r), _ptr(w))
    return g, r, w


def lam(P: Problem, U) -> np.ndarray:
    c, U = _checked(P), _state(P, U)
    out = np.zeros(P.E)
    lib().orc_lambda(ctypes.byref(c), _ptr(U), _ptr(out))
    return out


def rk3(P: Problem, U, dt: float, nsteps: int) -> np.ndarray:
    """nsteps steps of the optimal SSP-RK3 scheme (Eq. ssp); returns the new state."""
    c, U = _checked(P), _state(P, U).copy()
    lib().orc_rk3(ctypes.byref(c), _ptr(U), float(dt), int(nsteps))
    return U


def rk(P: Problem, U, dt: float, nsteps: int, order: int = 3) -> np.ndarray:
    """nsteps steps of the SSP Runge-Kutta scheme of the given order: 2 (Heun), 3
    (Eq. ssp) or 4 (Ketcheson's ten-stage method); returns the new state."""
    c, U = _checked(P), _state(P, U).copy()
    fn = {2: lib().orc_rk2, 3: lib().orc_rk3, 4: lib().orc_rk4}[order]
    fn(ctypes.byref(c), _ptr(U), float(dt), int(nsteps))
    return U


def gauss_legendre(n: int):
    x = np.zeros(n)
    w = np.zeros(n)
    lib().orc_gauss_legendre(int(n), _ptr(x), _ptr(w))
    return x, w


def project(P: Problem, samples, nq: int = 8) -> np.ndarray:
    """L2 projection of samples given at the nq-point Gauss points of every element
    (Euler system: samples of the dim + 2 conserved variables, shape (dim + 2, E nq^dim),
    one component after the other)."""
    if P.flux == "euler":
        f = np.asarray(samples, dtype=np.float64).reshape(P.ncomp, -1)
        Ps = dataclasses.replace(P, flux="advect", bc=tuple("outflow" if b in ("reflect", "state") else b for b in P.bc))
        return np.concatenate([project(Ps, f[c], nq) for c in range(P.ncomp)], axis=0)
    c = _checked(P)
    f = np.ascontiguousarray(np.asarray(samples, dtype=np.float64)).reshape(-1)
    if f.size != P.E * nq ** P.dim:
        raise ValueError("sample count")
    U = np.zeros((P.K, P.E))
    lib().orc_project(ctypes.byref(c), int(nq), _ptr(f), _ptr(U))
    return U


def l1_error(P: Problem, U, samples, nq: int = 8) -> float:
    c, U = _checked(P), _state(P, U)
    f = np.ascontiguousarray(np.asarray(samples, dtype=np.float64)).reshape(-1)
    return lib().orc_l1_error(ctypes.byref(c), _ptr(U), int(nq), _ptr(f))


def evaluate(P: Problem, U, nq: int) -> np.ndarray:
    c, U = _checked(P), _state(P, U)
    out = np.zeros(P.E * nq ** P.dim)
    lib().orc_eval(ctypes.byref(c), _ptr(U), int(nq), _ptr(out))
    return out


def mass(P: Problem, U) -> float:
    c, U = _checked(P), _state(P, U)
    return lib().orc_mass(ctypes.byref(c), _ptr(U))


def seminorm2(P: Problem, coeffs) -> float:
    c = _checked(P)
    v = np.ascontiguousarray(np.asarray(coeffs, dtype=np.float64))
    return lib().orc_seminorm2(ctypes.byref(c), _ptr(v))


def candidate(P: Problem, U, e: int, face: int):
    c, U = _checked(P), _state(P, U)
    out = np.zeros(P.K)
    rc = lib().orc_candidate(ctypes.byref(c), _ptr(U), int(e), int(face), _ptr(out))
    return None if rc != 0 else out


def llf(P: Problem, um, up, x, y, nx, ny) -> float:
    c = _checked(P)
    return lib().orc_llf(ctypes.byref(c), um, up, x, y, nx, ny)


def euler_llf(P: Problem, um, up, n) -> np.ndarray:
    """LLF flux of the Euler system between conservative states um (own) and up across a
    face of outward unit normal n: +-1 in 1D (reading R15), (nx, ny) in 2D (R17)."""
    c = _checked(P)
    a = np.ascontiguousarray(np.asarray(um, dtype=np.float64))
    b = np.ascontiguousarray(np.asarray(up, dtype=np.float64))
    H = np.zeros(P.ncomp)
    if P.dim == 1:
        lib().orc_euler_llf(ctypes.byref(c), _ptr(a), _ptr(b), float(n), _ptr(H))
    else:
        lib().orc_euler_llf2(ctypes.byref(c), _ptr(a), _ptr(b), float(n[0]), float(n[1]), _ptr(H))
    return H


def wave_speed(P: Problem, um, up, x, y, nx, ny) -> float:
    c = _checked(P)
    return lib().orc_wave_speed(ctypes.byref(c), um, up, x, y, nx, ny)


def legendre(n: int, a: int, x: float) -> float:
    return lib().orc_legendre(int(n), int(a), float(x))

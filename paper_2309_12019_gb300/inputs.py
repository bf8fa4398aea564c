"""Seeded synthetic inputs for the scalar conservation laws and the Euler problems of the
paper's Sec. 5.

This module holds no arithmetic of the method itself: it only places sample points,
evaluates initial data (closed-form functions of x), draws seeded random states and
states the time-step recipe.  Both the CUDA path and the CPU oracle consume what it
produces, and it imports neither of them.

Sample layout (shared by the projection entry points of both sides): for element
``e = iy*nx + ix`` and the ``nq``-point Gauss-Legendre rule ``g`` on [-1, 1], sample
``t = a + nq*b`` sits at ``x = xc + hx/2*g[a]``, ``y = yc + hy/2*g[b]``.
"""
from __future__ import annotations

import math

import numpy as np

SEED = 2309012019


def gauss_nodes(nq: int) -> np.ndarray:
    """Gauss-Legendre nodes on [-1, 1] (NumPy's rule)."""
    return np.polynomial.legendre.leggauss(nq)[0]


def sample_points(dim: int, nx: int, ny: int, box, nq: int = 8):
    """Physical coordinates of the projection samples, shape (E, nq**dim) each."""
    g = gauss_nodes(nq)
    x0, x1, y0, y1 = box
    hx = (x1 - x0) / nx
    xc = x0 + (np.arange(nx) + 0.5) * hx
    if dim == 1:
        X = xc[:, None] + 0.5 * hx * g[None, :]
        return X, np.zeros_like(X)
    hy = (y1 - y0) / ny
    yc = y0 + (np.arange(ny) + 0.5) * hy
    # element e = iy*nx + ix; sample t = a + nq*b
    Xe = np.broadcast_to(xc[None, :], (ny, nx)).reshape(-1)
    Ye = np.broadcast_to(yc[:, None], (ny, nx)).reshape(-1)
    ga = np.tile(g, nq)          # a fastest
    gb = np.repeat(g, nq)
    X = Xe[:, None] + 0.5 * hx * ga[None, :]
    Y = Ye[:, None] + 0.5 * hy * gb[None, :]
    return X, Y


# --------------------------------------------------------------------------------------
# Initial data of the workloads
# --------------------------------------------------------------------------------------

def u0_cos(x, y=None):
    """Sec. 5.1 smooth advection datum cos(2 pi (x - 0.5))."""
    return np.cos(2.0 * np.pi * (x - 0.5))


def u0_sin(x, y=None):
    """Sec. 5.2 Burgers datum sin(2 pi x)."""
    return np.sin(2.0 * np.pi * x)


def u0_mixed_1d(x, y=None):
    """1D advection profile: square wave on [0.2,0.4], plus a Gaussian exp(-300(x-0.6)^2)
    everywhere, plus 0.5 sin(2 pi x) on [0.7,0.9]."""
    u = np.where((x >= 0.2) & (x <= 0.4), 1.0, 0.0)
    u = u + np.exp(-300.0 * (x - 0.6) ** 2)
    u = u + np.where((x >= 0.7) & (x <= 0.9), 0.5 * np.sin(2.0 * np.pi * x), 0.0)
    return u


def u0_rotation(x, y):
    """Solid-body rotation datum (Sec. 5.3): slotted cylinder, cone and hump of radius 0.15."""
    r_cyl = np.hypot(x - 0.5, y - 0.75)
    r_cone = np.hypot(x - 0.5, y - 0.25)
    r_hump = np.hypot(x - 0.25, y - 0.5)
    u = np.zeros_like(x)
    cyl = (r_cyl <= 0.15) & ((np.abs(x - 0.5) >= 0.025) | (y >= 0.85))
    u = np.where(cyl, 1.0, u)
    u = np.where(r_cone <= 0.15, 1.0 - r_cone / 0.15, u)
    u = np.where(r_hump <= 0.15, 0.25 + 0.25 * np.cos(np.pi * r_hump / 0.15), u)
    return u


def u0_kpp(x, y):
    """KPP datum (Sec. 5.5): 7 pi / 2 inside the unit disc, pi / 4 outside."""
    return np.where(np.hypot(x, y) <= 1.0, 3.5 * np.pi, 0.25 * np.pi)


def fourier_steps_params(dim: int, rng: np.random.Generator, nmodes: int = 8, max_steps: int = 3,
                         min_steps: int = 0):
    """Random smooth-plus-steps datum: nmodes Fourier modes with amplitude ~U(0,1) plus
    min_steps..max_steps unit steps (indicators of random periodic intervals / rectangles)."""
    amp = rng.uniform(0.0, 1.0, nmodes)
    phase = rng.uniform(0.0, 2.0 * np.pi, nmodes)
    if dim == 1:
        k = rng.integers(1, 9, size=(nmodes, 1))
    else:
        k = rng.integers(-4, 5, size=(nmodes, 2))
        zero = np.all(k == 0, axis=1)
        k[zero, 0] = 1
    nsteps = int(rng.integers(min_steps, max_steps + 1))
    lo = rng.uniform(0.0, 1.0, size=(nsteps, dim))
    width = rng.uniform(0.05, 0.4, size=(nsteps, dim))
    return dict(amp=amp, phase=phase, k=k, lo=lo, width=width)


def u0_fourier_steps(params, x, y=None, xp=np):
    """sum_j a_j sin(2 pi k_j.x + phi_j) plus unit steps on periodic intervals/rectangles.
    x, y: NumPy arrays (xp=np) or torch tensors (xp=torch)."""
    k = params["k"]
    u = xp.zeros_like(x)
    for j in range(len(params["amp"])):
        arg = float(k[j, 0]) * x if k.shape[1] == 1 else float(k[j, 0]) * x + float(k[j, 1]) * y
        u = u + float(params["amp"][j]) * xp.sin(2.0 * math.pi * arg + float(params["phase"][j]))
    for s in range(len(params["lo"])):
        coords = [x] if k.shape[1] == 1 else [x, y]
        inside = None
        for c, lo, w in zip(coords, params["lo"][s], params["width"][s]):
            t = xp.remainder(c - float(lo), 1.0) < float(w)
            inside = t if inside is None else (inside & t)
        u = u + xp.where(inside, 1.0, 0.0)
    return u


def ensemble_instances(n: int = 512, seed: int = SEED):
    """The batched-ensemble workload: n independent periodic instances on the unit
    interval / square, each 1D Burgers or 2D linear advection with v = (cos t, sin t)
    (coin flip), cells log-uniform in [64, 4096] (1D) or side log-uniform in [32, 512]
    (2D), degree uniform in {1, 2, 3}, initial data u0_fourier_steps, and the time step
    dt = CFL_p / sum_i(max|f_i'| / h) with max|f'| bounded by the sum of amplitudes plus
    steps (Burgers) or |cos t|, |sin t| (advection).  CFL_p = 0.1, 0.05, 0.025 for
    p = 1, 2, 3: the stabilization term gamma nu grad^2 has spectral radius 6, 15, 28.3
    gamma lambda / h per direction for p = 1, 2, 3 (largest eigenvalue of the scaled
    element stiffness), and SSP-RK3 is stable on the negative axis up to 2.51, so at
    gamma = 1 in 2D lambda dt / h must stay below 0.21, 0.084, 0.044.  Instance i uses
    the generator seeded with seed + i."""
    out = []
    for i in range(n):
        rng = np.random.default_rng(seed + i)
        dim = 1 if rng.uniform() < 0.5 else 2
        if dim == 1:
            cells = int(round(math.exp(rng.uniform(math.log(64), math.log(4096)))))
        else:
            cells = int(round(math.exp(rng.uniform(math.log(32), math.log(512)))))
        p = int(rng.integers(1, 4))
        theta = float(rng.uniform(0.0, 2.0 * math.pi))
        params = fourier_steps_params(dim, rng)
        h = 1.0 / cells
        cfl = {1: 0.1, 2: 0.05, 3: 0.025}[p]
        if dim == 1:
            bound = float(np.sum(params["amp"])) + len(params["lo"])
            dt = cfl_dt(cfl, [bound], [h])
            a = (1.0, 0.0)
            flux = "burgers"
        else:
            a = (math.cos(theta), math.sin(theta))
            dt = cfl_dt(cfl, [abs(a[0]), abs(a[1])], [h, h])
            flux = "advect"
        out.append(dict(dim=dim, nx=cells, ny=cells if dim == 2 else 1, p=p, flux=flux, a=a, dt=dt,
                        init=params))
    return out


def adjoint_field(seed: int):
    """Datum of the adjoint workload: 4 Fourier modes plus exactly one unit step on the
    periodic unit square (control: seed, target: another seed)."""
    return fourier_steps_params(2, np.random.default_rng(seed), nmodes=4, max_steps=1, min_steps=1)


def sample_points_xp(dim: int, nx: int, ny: int, box, nq: int, xp, **kw):
    """sample_points for an array namespace xp (np or torch; kw go to xp.tensor/asarray)."""
    g = gauss_nodes(nq)
    x0, x1, y0, y1 = box
    hx = (x1 - x0) / nx
    if xp is np:
        X, Y = sample_points(dim, nx, ny, box, nq)
        return X, Y
    gt = xp.tensor(g, **kw)
    xc = x0 + (xp.arange(nx, **kw) + 0.5) * hx
    if dim == 1:
        X = xc[:, None] + 0.5 * hx * gt[None, :]
        return X, xp.zeros_like(X)
    hy = (y1 - y0) / ny
    yc = y0 + (xp.arange(ny, **kw) + 0.5) * hy
    Xe = xc[None, :].expand(ny, nx).reshape(-1)
    Ye = yc[:, None].expand(ny, nx).reshape(-1)
    ga = gt.repeat(nq)                 # a fastest
    gb = gt.repeat_interleave(nq)
    X = Xe[:, None] + 0.5 * hx * ga[None, :]
    Y = Ye[:, None] + 0.5 * hy * gb[None, :]
    return X, Y


# --------------------------------------------------------------------------------------
# Random modal states for parity tests
# --------------------------------------------------------------------------------------

def random_state(dim: int, p: int, E: int, seed: int, smooth: bool = False,
                 scale: float = 1.0, offset: float = 0.0) -> np.ndarray:
    """Seeded random modal coefficients, shape ((p+1)**dim, E).

    ``smooth=True`` lets the coefficient of total degree s decay like 4**-s, which keeps
    neighbouring elements unrelated (so sensors fire) but the per-element polynomials tame.
    """
    rng = np.random.default_rng(seed)
    K = (p + 1) ** dim
    U = rng.standard_normal((K, E)) * scale
    if smooth:
        for k in range(K):
            i, j = k % (p + 1), k // (p + 1)
            U[k] *= 0.25 ** (i + (j if dim == 2 else 0))
    U[0] += offset
    return U


def cfl_dt(cfl: float, speeds, h) -> float:
    """Time step of the workloads: dt = CFL / sum_i (max|f_i'| / dx_i)."""
    return cfl / sum(s / hh for s, hh in zip(speeds, h))


def nsteps_to(t_end: float, dt: float):
    """Whole steps of size dt to t_end, the last one shortened to land on t_end."""
    n = int(math.floor(t_end / dt + 1e-9))
    last = t_end - n * dt
    if last < 1e-12 * dt:
        return n, dt, 0.0
    return n, dt, last


# --------------------------------------------------------------------------------------
# Shock tubes of the Euler system (Sec. 5.6), primitive states (rho, v, p), gamma = 1.4
# --------------------------------------------------------------------------------------
# Shock tubes of Sec. 5.6.  Where the paper gives no diaphragm position it is read as
# the usual one of each problem (Sod, Lax: the centre; modified Sod: x = 0.3;
# Shu-Osher: x = -4).  An inlet is read as a zero-gradient side: the state there stays at
# its initial value up to t_end (supersonic inflow for Shu-Osher; for the modified Sod
# problem the rarefaction's head reaches x = 0 only at t = 0.7).  "lam" bounds |v| + c
# over the solution and sets the time step.
SHOCK_TUBES = {
    "sod": dict(box=(0.0, 1.0), jumps=(0.5,), states=((1.0, 0.0, 1.0), (0.125, 0.0, 0.1)),
                bc=("reflect", "reflect"), t_end=0.231, nx=128, p=2, lam=2.5),
    "sod_modified": dict(box=(0.0, 1.0), jumps=(0.3,), states=((1.0, 0.75, 1.0), (0.125, 0.0, 0.1)),
                         bc=("outflow", "reflect"), t_end=0.2, nx=128, p=2, lam=2.8),
    "lax": dict(box=(0.0, 2.0), jumps=(1.0,), states=((0.445, 0.698, 3.528), (0.5, 0.0, 0.571)),
                bc=("outflow", "outflow"), t_end=0.14, nx=512, p=2, lam=5.0),
    "shu_osher": dict(box=(-5.0, 5.0), jumps=(-4.0,), states=((3.857143, 2.629369, 10.3333), "sine"),
                      bc=("outflow", "reflect"), t_end=1.8, nx=512, p=2, lam=5.0),
    # Woodward-Colella blast wave: the paper's three states (its middle pressure is 0.1)
    # between reflecting walls, the jumps read as the cited problem's x = 0.1 and 0.9 (the
    # paper gives none); |v| + c stays below 60 (c = 37.4 in the left state)
    "blast": dict(box=(0.0, 1.0), jumps=(0.1, 0.9), states=((1.0, 0.0, 1000.0), (1.0, 0.0, 0.1), (1.0, 0.0, 100.0)),
                  bc=("reflect", "reflect"), t_end=0.038, nx=512, p=2, lam=60.0),
}

GAS_GAMMA = 1.4


def shock_tube_primitive(name: str, x):
    """(rho, v, p) of the initial data at the points x (any shape)."""
    d = SHOCK_TUBES[name]
    x = np.asarray(x, dtype=np.float64)
    region = np.zeros(x.shape, dtype=np.int64)
    for j in d["jumps"]:
        region += (x >= j).astype(np.int64)
    out = np.zeros((3,) + x.shape)
    for r, st in enumerate(d["states"]):
        sel = region == r
        if isinstance(st, str):        # Shu-Osher: a density wave ahead of the shock
            out[0][sel] = 1.0 + 0.2 * np.sin(5.0 * x[sel])
            out[1][sel] = 0.0
            out[2][sel] = 1.0
        else:
            for c in range(3):
                out[c][sel] = st[c]
    return out


def shock_tube_samples(name: str, nx: int, nq: int = 8, gamma: float = GAS_GAMMA):
    """Conservative samples (rho, rho v, rho E) at the projection points of a 1D mesh of
    nx elements, shape (3, nx * nq).  In a cell that a diaphragm cuts, every sample is
    the cell's Gauss mean of the data, so that the projection there is the cell mean (the
    L2 projection of a jump inside a cell overshoots, here into negative pressure)."""
    d = SHOCK_TUBES[name]
    X, _ = sample_points(1, nx, 1, (d["box"][0], d["box"][1], 0.0, 1.0), nq)
    rho, v, p = shock_tube_primitive(name, X)
    q = np.stack([rho, rho * v, p / (gamma - 1.0) + 0.5 * rho * v * v])    # (3, nx, nq)
    w = np.polynomial.legendre.leggauss(nq)[1] / 2.0
    h = (d["box"][1] - d["box"][0]) / nx
    left = d["box"][0] + np.arange(nx) * h
    cut = np.zeros(nx, dtype=bool)
    for j in d["jumps"]:
        cut |= (left < j) & (j < left + h)
    q = np.where(cut[None, :, None], (q * w).sum(axis=2, keepdims=True), q)
    return q.reshape(3, -1)


def euler_cfl(p: int, dim: int = 1) -> float:
    """Courant number of the Euler workloads, dt = cfl h / lam: inside the SSP-RK3
    stability interval of the stabilization term for gamma = 1 (radius 6, 15, 28.3 times
    lam dt / h per direction for p = 1, 2, 3; the directions add in 2D)."""
    return {1: 0.1, 2: 0.1, 3: 0.05}[p] / dim


def random_euler_state(p: int, E: int, seed: int, amp: float = 0.05, gamma: float = GAS_GAMMA,
                       dim: int = 1) -> np.ndarray:
    """Seeded random modal state of the Euler system, shape ((dim + 2) K, E) with
    K = (p+1)^dim, rows comp K + k: cell means from random primitive states (rho in
    [1, 1.4], each velocity component normal with deviation 0.5, p in [1, 1.5]) and small
    random higher modes (amp (1 + comp)), so that density and pressure stay positive."""
    rng = np.random.default_rng(seed)
    K = (p + 1) ** dim
    U = np.zeros(((dim + 2) * K, E))
    rho = 1.0 + 0.4 * rng.random(E)
    v = 0.5 * rng.standard_normal((dim, E))
    pr = 1.0 + 0.5 * rng.random(E)
    U[0] = rho
    for a in range(dim):
        U[(1 + a) * K] = rho * v[a]
    U[(dim + 1) * K] = pr / (gamma - 1.0) + 0.5 * rho * (v * v).sum(axis=0)
    for c in range(dim + 2):
        U[c * K + 1:(c + 1) * K] = amp * (1 + c) * rng.standard_normal((K - 1, E))
    return U


# 2D problems of Sec. 5.6 whose data jump along cell faces at the paper's mesh sizes.
# Outflow boundaries for the rarefaction problems, as the paper states.
# Kelvin-Helmholtz: the denser, left-moving state fills the strip |y - 0.5| < 0.25 and
# the boundaries are periodic (the paper gives neither; this is the usual set-up of the
# cited problem).  Triple point: three states in the subdomains the paper names, walls
# all round.
EULER_2D = {
    "kelvin_helmholtz": dict(box=(0.0, 1.0, 0.0, 1.0), bc=("periodic",) * 4, t_end=1.0, nx=512, ny=512, p=2,
                             lam=3.0),
    "triple_point": dict(box=(0.0, 7.0, 0.0, 3.0), bc=("reflect",) * 4, t_end=4.0, nx=896, ny=384, p=2, lam=3.0),
    # the two four-quadrant rarefaction problems, the paper's first and second initial
    # conditions; quadrants numbered counterclockwise from x > 1/2, y > 1/2
    "rarefaction_1": dict(box=(0.0, 1.0, 0.0, 1.0), bc=("outflow",) * 4, t_end=0.2, nx=256, ny=256, p=2, lam=3.0,
                          states=((1.0, 0.6233, 0.6233, 1.5), (0.389, -0.6233, 0.6233, 0.4),
                                  (1.0, -0.6233, -0.6233, 1.5), (0.389, 0.6233, -0.6233, 0.4))),
    "rarefaction_2": dict(box=(0.0, 1.0, 0.0, 1.0), bc=("outflow",) * 4, t_end=0.25, nx=256, ny=256, p=2, lam=3.0,
                          states=((1.0, 0.0312, 0.0312, 0.5), (0.927, -0.0312, 0.0312, 0.45),
                                  (1.0, -0.0312, -0.0312, 0.5), (0.927, 0.0312, -0.0312, 0.45))),
    # double Mach reflection: the Mach 10 shock at 60 degrees to the wall y = 0; post-shock
    # (L) left of x = 1/6 + y / sqrt 3, pre-shock (R) right of it; sides prescribed (reading
    # R19): x = 0 post-shock; x = 4 outflow (supersonic); y = 0 post-shock for x < 1/6, wall
    # beyond; y = 1 post-shock for x < 1/6 + (1 + 20 t) / sqrt 3, pre-shock beyond.  The
    # paper's finest mesh of its figure, 384 x 96, p = 2, t = 0.2; |v| + c stays below 20.
    "double_mach": dict(box=(0.0, 4.0, 0.0, 1.0), bc=("state", "outflow", "state", "state"), t_end=0.2,
                        nx=384, ny=96, p=2, lam=20.0,
                        states=((8.0, 8.25 * math.cos(math.pi / 6), -8.25 * math.sin(math.pi / 6), 116.5),
                                (1.4, 0.0, 0.0, 1.0))),
}


def double_mach_boundary(gamma: float = 1.4):
    """dgw / oracle Problem fields of the double Mach reflection's prescribed sides:
    bstate (post-shock, pre-shock; conservative), and per side (-x, +x, -y, +y) the split
    along the side at t = 0, its speed and the ghost below / from it (0 post-shock,
    1 pre-shock, 2 wall)."""
    st = []
    for rho, vx, vy, pr in EULER_2D["double_mach"]["states"]:
        st.append((rho, rho * vx, rho * vy, pr / (gamma - 1.0) + 0.5 * rho * (vx * vx + vy * vy)))
    r3 = math.sqrt(3.0)
    return dict(bstate=tuple(st), bsplit=(10.0, 0.0, 1.0 / 6.0, 1.0 / 6.0 + 1.0 / r3),
                bspeed=(0.0, 0.0, 0.0, 20.0 / r3), bbelow=(0, 0, 0, 0), babove=(1, 0, 2, 1))


def euler2d_primitive(name: str, x, y):
    """(rho, vx, vy, p) of the initial data and the region label at the points (x, y)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    if name == "kelvin_helmholtz":
        inner = np.abs(y - 0.5) < 0.25
        rho = np.where(inner, 2.0, 1.0)
        vx = np.where(inner, -0.5, 0.5)
        vy = 0.01 * np.sin(2.0 * np.pi * (x - 0.5))
        pr = np.full(x.shape, 2.5)
        return np.stack([rho, vx, vy, pr]), inner.astype(np.int64)
    if name.startswith("rarefaction_"):
        region = np.where(x > 0.5, np.where(y > 0.5, 0, 3), np.where(y > 0.5, 1, 2))
        st = np.asarray(EULER_2D[name]["states"])[region]
        return np.moveaxis(st, -1, 0), region
    if name == "double_mach":
        region = np.where(x < 1.0 / 6.0 + y / math.sqrt(3.0), 0, 1)
        st = np.asarray(EULER_2D[name]["states"])[region]
        return np.moveaxis(st, -1, 0), region
    if name == "triple_point":
        region = np.where(x <= 1.0, 0, np.where(y <= 1.5, 1, 2))
        rho = np.array([1.0, 0.125, 1.0])[region]
        pr = np.array([1.0, 0.1, 0.1])[region]
        return np.stack([rho, 0.0 * rho, 0.0 * rho, pr]), region
    raise ValueError(name)


def euler2d_samples(name: str, nx: int, ny: int, nq: int = 8, gamma: float = GAS_GAMMA):
    """Conservative samples (rho, rho vx, rho vy, rho E) at the projection points of an
    nx x ny mesh, shape (4, E nq^2); a cell whose samples straddle two regions gets its
    Gauss mean in every sample (as for the shock tubes)."""
    d = EULER_2D[name]
    X, Y = sample_points(2, nx, ny, d["box"], nq)
    (rho, vx, vy, pr), region = euler2d_primitive(name, X, Y)
    q = np.stack([rho, rho * vx, rho * vy, pr / (gamma - 1.0) + 0.5 * rho * (vx * vx + vy * vy)])
    g, w = np.polynomial.legendre.leggauss(nq)
    w2 = (np.tile(w, nq) * np.repeat(w, nq)) / 4.0           # sample t = a + nq b
    cut = region.min(axis=1) != region.max(axis=1)
    q = np.where(cut[None, :, None], (q * w2).sum(axis=2, keepdims=True), q)
    return q.reshape(4, -1)


def sod_train_samples(nx: int, period: int = 64, nq: int = 8, gamma: float = GAS_GAMMA):
    """A periodic train of Sod shock tubes on [0, 1): cells alternate between Sod's left
    and right states in runs of period / 2 cells, so that every period cells carry a
    shock, a contact and a rarefaction once the diaphragms are removed (a large-mesh
    workload with the structure of Sec. 5.6's Sod problem).  Conservative samples at
    the projection points, shape (3, nx * nq); nx a multiple of period."""
    if nx % period or period % 2:
        raise ValueError("nx must be a multiple of an even period")
    cell = np.arange(nx)
    left = (cell % period) < period // 2
    rho = np.where(left, 1.0, 0.125)
    pr = np.where(left, 1.0, 0.1)
    rho = np.repeat(rho, nq)
    pr = np.repeat(pr, nq)
    return np.stack([rho, np.zeros_like(rho), pr / (gamma - 1.0)])

"""Thin Python binding of libdgw (include/dgw.h): argument marshalling only.

Every computation runs in the library's CUDA kernels; this module converts torch tensors
to device pointers and the current torch stream to a ``cudaStream_t``, and raises
``DGWError`` on any non-zero status.  There is no CPU fallback: if the library cannot be
loaded, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

BC = {"periodic": 0, "inflow_zero": 1, "outflow": 2, "reflect": 3, "state": 4}
FLUX = {"advect": 0, "rotation": 1, "burgers": 2, "kpp": 3, "euler": 4}
STAB = {"dg": 0, "lo": 1, "weno": 2, "zhao": 3}
PREC = {"fp64": 0, "fp32": 1}

# Threshold b of Eq. (gensensor) when a Problem gives none: 0.1 for the scalar laws (the
# tolerance of the remark in Sec. 4, as dgw_defaults sets it), 0 for the Euler system
# (Sec. 5.6 runs the unmodified sensor and compares b > 0 as a variant).
B_SCALAR = 0.1
B_EULER = 0.0

STATUS = {0: "DGW_OK", -1: "DGW_EINVAL", -2: "DGW_ENOMEM", -3: "DGW_ECUDA", -4: "DGW_EUNSUPPORTED",
          -5: "DGW_ETIMEOUT", -6: "DGW_ENONFINITE"}


class DGWError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Mesh(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("x0", ctypes.c_double), ("x1", ctypes.c_double),
                ("y0", ctypes.c_double), ("y1", ctypes.c_double),
                ("bc", ctypes.c_int * 4)]


class Flux(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("a", ctypes.c_double * 2), ("center", ctypes.c_double * 2),
                ("omega", ctypes.c_double), ("lambda_nu", ctypes.c_double), ("gas_gamma", ctypes.c_double),
                ("bstate", (ctypes.c_double * 4) * 2), ("bsplit", ctypes.c_double * 4),
                ("bspeed", ctypes.c_double * 4), ("bbelow", ctypes.c_int * 4), ("babove", ctypes.c_int * 4)]


class Params(ctypes.Structure):
    _fields_ = [("stab", ctypes.c_int), ("q", ctypes.c_double), ("b", ctypes.c_double),
                ("w_nbr", ctypes.c_double), ("eps_w", ctypes.c_double), ("eps_s", ctypes.c_double),
                ("prec", ctypes.c_int), ("theta", ctypes.c_double), ("rk_order", ctypes.c_int)]


# every symbol declared in include/dgw.h
EXPORTS = ("dgw_defaults", "dgw_create", "dgw_destroy", "dgw_sizes", "dgw_set_params", "dgw_project",
           "dgw_residual", "dgw_sensor", "dgw_rk_step", "dgw_rk_step_host", "dgw_mass",
           "dgw_sync_status", "dgw_debug", "dgw_set_stage_kernel", "dgw_set_time", "dgw_get_time", "dgw_residual_vjp", "dgw_adjoint_step", "dgw_rk_step_stages", "dgw_adjoint_step_stages", "dgw_misfit", "dgw_batch_create", "dgw_batch_destroy", "dgw_batch_sizes",
           "dgw_batch_set_dt", "dgw_batch_project", "dgw_batch_rk_step", "dgw_batch_autotune",
           "dgw_batch_schedule", "dgw_batch_set_schedule", "dgw_batch_sync_status", "dgw_batch_debug", "dgw_rk_step_noalloc", "dgw_selftest_sincos", "dgw_selftest_tc_volume",
           "dgw_last_error", "dgw_version")


def load(build: bool = True):
    """Loads (building first if needed) the in-tree libdgw.so."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build() if build else _build.LIB
        L = ctypes.CDLL(path)
        vp, i64p, ip, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int), \
            ctypes.POINTER(ctypes.c_double)
        L.dgw_defaults.argtypes = [ctypes.POINTER(Mesh), ctypes.POINTER(Flux), ctypes.POINTER(Params)]
        L.dgw_defaults.restype = None
        L.dgw_create.argtypes = [ctypes.POINTER(Mesh), ctypes.c_int, ctypes.POINTER(Flux),
                                 ctypes.POINTER(Params), ctypes.POINTER(vp)]
        L.dgw_destroy.argtypes = [vp]
        L.dgw_sizes.argtypes = [vp, i64p, ip, ip]
        L.dgw_set_params.argtypes = [vp, ctypes.POINTER(Params)]
        L.dgw_project.argtypes = [vp, ctypes.c_int, vp, vp, vp]
        L.dgw_residual.argtypes = [vp, vp, vp, vp]
        L.dgw_sensor.argtypes = [vp, vp, vp, vp]
        L.dgw_rk_step.argtypes = [vp, vp, ctypes.c_double, ctypes.c_int, vp]
        L.dgw_rk_step_host.argtypes = [vp, vp, vp, ctypes.c_double, ctypes.c_int, vp]
        L.dgw_mass.argtypes = [vp, vp, dp, vp]
        L.dgw_sync_status.argtypes = [vp, vp]
        L.dgw_debug.argtypes = [vp, ctypes.c_int]
        L.dgw_set_stage_kernel.argtypes = [vp, ctypes.c_int]
        L.dgw_set_time.argtypes = [vp, ctypes.c_double, vp]
        L.dgw_get_time.argtypes = [vp, dp, vp]
        L.dgw_residual_vjp.argtypes = [vp, vp, vp, vp, vp]
        L.dgw_adjoint_step.argtypes = [vp, vp, vp, vp, ctypes.c_double, vp]
        L.dgw_misfit.argtypes = [vp, vp, vp, dp, vp, vp]
        L.dgw_rk_step_stages.argtypes = [vp, vp, ctypes.c_double, vp, vp, vp, vp]
        L.dgw_adjoint_step_stages.argtypes = [vp, vp, vp, vp, vp, vp, ctypes.c_double, vp]
        L.dgw_batch_create.argtypes = [ctypes.c_int, ctypes.POINTER(Mesh), ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(Flux), ctypes.POINTER(Params), ctypes.POINTER(vp)]
        L.dgw_batch_destroy.argtypes = [vp]
        L.dgw_batch_sizes.argtypes = [vp, i64p, i64p]
        L.dgw_batch_set_dt.argtypes = [vp, dp]
        L.dgw_batch_project.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp, vp]
        L.dgw_batch_rk_step.argtypes = [vp, vp, ctypes.c_int, vp]
        L.dgw_batch_autotune.argtypes = [vp, vp, ctypes.c_int, ip, vp]
        L.dgw_batch_schedule.argtypes = [vp, ctypes.c_int, ctypes.c_int, ip, ip]
        L.dgw_batch_set_schedule.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.dgw_batch_sync_status.argtypes = [vp, vp]
        L.dgw_batch_debug.argtypes = [vp, ctypes.c_longlong, ctypes.c_int]
        L.dgw_rk_step_noalloc.argtypes = [ctypes.POINTER(Mesh), ctypes.c_int, ctypes.POINTER(Flux),
                                          ctypes.POINTER(Params), vp, ctypes.c_double, ctypes.c_int, vp]
        L.dgw_selftest_sincos.argtypes = [vp, vp, vp, ctypes.c_int64, vp]
        L.dgw_selftest_tc_volume.argtypes = [vp, vp, ctypes.c_int64, ctypes.c_int, ctypes.POINTER(ctypes.c_float), vp]
        L.dgw_last_error.restype = ctypes.c_char_p
        L.dgw_version.restype = ctypes.c_char_p
        for name in EXPORTS:
            getattr(L, name)
        _lib = L
        return L


def _check(status: int):
    if status != 0:
        raise DGWError(status, load().dgw_last_error().decode())


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


@dataclasses.dataclass
class Problem:
    """Mesh, degree, flux and stabilization of one scalar conservation law, or of the
    Euler system in 1D or 2D (flux "euler"), host side."""
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
    prec: str = "fp64"
    theta: float = 1.0
    rk_order: int = 3
    gas_gamma: float = 1.4
    # bc "state" sides (2D Euler): see dgw_flux in include/dgw.h; t is the start time
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
    def ncomp(self) -> int:
        return self.dim + 2 if self.flux == "euler" else 1

    @property
    def K(self) -> int:
        """Rows of the state: modes per element (times 3 components for the Euler system)."""
        return (self.p + 1) ** self.dim * self.ncomp

    def c_structs(self):
        m = Mesh()
        m.dim, m.nx, m.ny = self.dim, self.nx, self.ny if self.dim == 2 else 1
        m.x0, m.x1, m.y0, m.y1 = [float(v) for v in self.box]
        for i, b in enumerate(self.bc):
            m.bc[i] = BC[b]
        f = Flux()
        f.kind = FLUX[self.flux]
        f.a[0], f.a[1] = self.a
        f.center[0], f.center[1] = self.center
        f.omega, f.lambda_nu = self.omega, self.lambda_nu
        f.gas_gamma = self.gas_gamma
        for i in range(2):
            for c in range(4):
                f.bstate[i][c] = self.bstate[i][c]
        for k in range(4):
            f.bsplit[k], f.bspeed[k] = self.bsplit[k], self.bspeed[k]
            f.bbelow[k], f.babove[k] = self.bbelow[k], self.babove[k]
        s = Params()
        s.stab, s.q, s.b, s.w_nbr = STAB[self.stab], self.q, self.b, self.w_nbr
        s.eps_w, s.eps_s, s.prec, s.theta = self.eps_w, self.eps_s, PREC[self.prec], self.theta
        s.rk_order = self.rk_order
        return m, f, s


class Context:
    """Owns one dgw_ctx.  Methods mirror the C entry points of include/dgw.h."""

    def __init__(self, problem: Problem):
        L = load()
        self.problem = problem
        m, f, s = problem.c_structs()
        h = ctypes.c_void_p()
        _check(L.dgw_create(ctypes.byref(m), problem.p, ctypes.byref(f), ctypes.byref(s), ctypes.byref(h)))
        self._h = h
        E, K, eb = ctypes.c_int64(), ctypes.c_int(), ctypes.c_int()
        _check(L.dgw_sizes(h, ctypes.byref(E), ctypes.byref(K), ctypes.byref(eb)))
        self.E, self.K, self.elem_bytes = E.value, K.value, eb.value
        if problem.t != 0.0:
            self.set_time(problem.t, stream=0)

    @property
    def dtype(self):
        import torch
        return torch.float64 if self.elem_bytes == 8 else torch.float32

    def close(self):
        if getattr(self, "_h", None):
            load().dgw_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _state(self, U):
        if not U.is_cuda or U.dtype != self.dtype or not U.is_contiguous() or U.numel() != self.K * self.E:
            raise ValueError(f"state must be a contiguous CUDA {self.dtype} tensor of {self.K}x{self.E}")
        return _ptr(U)

    def set_params(self, **kw):
        self.problem = dataclasses.replace(self.problem, **kw)
        _, _, s = self.problem.c_structs()
        _check(load().dgw_set_params(self._h, ctypes.byref(s)))

    def project(self, samples, U, nq: int = 8, stream=None):
        import torch
        if samples.dtype != torch.float64 or not samples.is_cuda or not samples.is_contiguous():
            raise ValueError("samples must be a contiguous CUDA float64 tensor")
        P = self.problem
        if samples.numel() != P.ncomp * self.E * nq ** P.dim:
            raise ValueError(f"expected {P.ncomp} x {self.E} x {nq ** P.dim} samples")
        _check(load().dgw_project(self._h, nq, _ptr(samples), self._state(U), _stream(stream)))

    def residual(self, U, L, stream=None):
        _check(load().dgw_residual(self._h, self._state(U), self._state(L), _stream(stream)))

    def sensor(self, U, gamma, stream=None):
        import torch
        if gamma.dtype != torch.float64 or not gamma.is_cuda or gamma.numel() != self.E:
            raise ValueError("gamma must be a CUDA float64 tensor of E entries")
        _check(load().dgw_sensor(self._h, self._state(U), _ptr(gamma), _stream(stream)))

    def rk_step(self, U, dt: float, nsteps: int = 1, stream=None):
        _check(load().dgw_rk_step(self._h, self._state(U), float(dt), int(nsteps), _stream(stream)))

    def rk_step_host(self, U_in, U_out, dt: float, nsteps: int = 1, stream=None):
        for t in (U_in, U_out):
            if t.is_cuda or t.dtype != self.dtype or not t.is_contiguous() or t.numel() != self.K * self.E:
                raise ValueError("host state must be a contiguous CPU tensor of the context dtype")
        _check(load().dgw_rk_step_host(self._h, _ptr(U_in), _ptr(U_out), float(dt), int(nsteps),
                                       _stream(stream)))

    def mass(self, U, stream=None) -> float:
        out = ctypes.c_double()
        _check(load().dgw_mass(self._h, self._state(U), ctypes.byref(out), _stream(stream)))
        return out.value

    def sync_status(self, stream=None):
        _check(load().dgw_sync_status(self._h, _stream(stream)))

    def set_time(self, t: float, stream=None):
        """The context's time, read by "state" sides (dgw_set_time)."""
        _check(load().dgw_set_time(self._h, float(t), _stream(stream)))

    def get_time(self, stream=None) -> float:
        t = ctypes.c_double()
        _check(load().dgw_get_time(self._h, ctypes.byref(t), _stream(stream)))
        return t.value

    def debug(self, wait_limit: int):
        """Poll limit of the stage kernels' bounded TMA waits (dgw_debug)."""
        _check(load().dgw_debug(self._h, int(wait_limit)))

    def set_stage_kernel(self, choice: int):
        """0 automatic, 1 the tile kernel, 2 the persistent kernel (dgw_set_stage_kernel)."""
        _check(load().dgw_set_stage_kernel(self._h, int(choice)))

    def residual_vjp(self, U, lam, out, stream=None):
        """out = J_L(U)^T lam (dgw_residual_vjp)."""
        _check(load().dgw_residual_vjp(self._h, self._state(U), self._state(lam), self._state(out), _stream(stream)))

    def adjoint_step(self, U_n, lam_np1, lam_n, dt: float, stream=None):
        """lam_n = (dU^{n+1}/dU^n)^T lam_np1 for one SSP-RK3 step from U_n (dgw_adjoint_step)."""
        _check(load().dgw_adjoint_step(self._h, self._state(U_n), self._state(lam_np1), self._state(lam_n),
                                       float(dt), _stream(stream)))

    def rk_step_stages(self, U, dt: float, U1, U2, U_next=None, stream=None):
        """One SSP-RK3 step from U keeping its stage states U1, U2; U^{n+1} to U_next if
        given (dgw_rk_step_stages)."""
        _check(load().dgw_rk_step_stages(self._h, self._state(U), float(dt), self._state(U1), self._state(U2),
                                         None if U_next is None else self._state(U_next), _stream(stream)))

    def adjoint_step_stages(self, U_n, U1, U2, lam_np1, lam_n, dt: float, stream=None):
        """dgw_adjoint_step with the step's stage states given (dgw_adjoint_step_stages)."""
        _check(load().dgw_adjoint_step_stages(self._h, self._state(U_n), self._state(U1), self._state(U2),
                                              self._state(lam_np1), self._state(lam_n), float(dt),
                                              _stream(stream)))

    def misfit(self, U, U_target, grad=None, stream=None) -> float:
        """J = 1/2 int (U_h - U_target)^2, and grad = dJ/dU if given (dgw_misfit)."""
        J = ctypes.c_double()
        g = self._state(grad) if grad is not None else None
        _check(load().dgw_misfit(self._h, self._state(U), self._state(U_target), ctypes.byref(J), g,
                                 _stream(stream)))
        return J.value


class Batch:
    """Owns one dgw_batch: many independent problems advanced by one persistent kernel per
    dimension.  Methods mirror the dgw_batch_* entry points of include/dgw.h."""

    def __init__(self, problems, prec: str = "fp32"):
        L = load()
        n = len(problems)
        meshes, fluxes, params = (Mesh * n)(), (Flux * n)(), None
        ps = (ctypes.c_int * n)()
        for i, pr in enumerate(problems):
            pr = dataclasses.replace(pr, prec=prec)
            m, f, s = pr.c_structs()
            meshes[i], fluxes[i], ps[i] = m, f, pr.p
            params = params or s
        h = ctypes.c_void_p()
        _check(L.dgw_batch_create(n, meshes, ps, fluxes, ctypes.byref(params), ctypes.byref(h)))
        self._h = h
        self.problems = list(problems)
        self.prec = prec
        total = ctypes.c_int64()
        offs = (ctypes.c_int64 * n)()
        _check(L.dgw_batch_sizes(h, ctypes.byref(total), offs))
        self.total = total.value
        self.offsets = list(offs)

    @property
    def dtype(self):
        import torch
        return torch.float64 if self.prec == "fp64" else torch.float32

    def close(self):
        if getattr(self, "_h", None):
            load().dgw_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _state(self, U):
        if not U.is_cuda or U.dtype != self.dtype or not U.is_contiguous() or U.numel() < self.total:
            raise ValueError(f"packed state must be a contiguous CUDA {self.dtype} tensor of {self.total}")
        return _ptr(U)

    def view(self, U, i):
        """Instance i of the packed state as a (K, E) tensor view."""
        pr = self.problems[i]
        return U[self.offsets[i]:self.offsets[i] + pr.K * pr.E].view(pr.K, pr.E)

    def set_dt(self, dts):
        arr = (ctypes.c_double * len(dts))(*[float(d) for d in dts])
        _check(load().dgw_batch_set_dt(self._h, arr))

    def project(self, samples, U, first: int = 0, count=None, nq: int = 8, stream=None):
        """Projects instances first .. first+count-1 from their concatenated samples."""
        import torch
        if samples.dtype != torch.float64 or not samples.is_cuda or not samples.is_contiguous():
            raise ValueError("samples must be a contiguous CUDA float64 tensor")
        count = len(self.problems) - first if count is None else count
        _check(load().dgw_batch_project(self._h, int(nq), int(first), int(count), _ptr(samples),
                                        self._state(U), _stream(stream)))

    def rk_step(self, U, nsteps: int = 1, stream=None):
        _check(load().dgw_batch_rk_step(self._h, self._state(U), int(nsteps), _stream(stream)))

    def autotune(self, U, steps: int = 2, stream=None) -> int:
        c = ctypes.c_int()
        _check(load().dgw_batch_autotune(self._h, self._state(U), int(steps), ctypes.byref(c), _stream(stream)))
        return c.value

    def sync_status(self, stream=None):
        _check(load().dgw_batch_sync_status(self._h, _stream(stream)))

    def schedule(self, dim: int, p: int):
        """(tile rows, tiles per work item) of the group (dim, p) (dgw_batch_schedule)."""
        rows, chunk = ctypes.c_int(), ctypes.c_int()
        _check(load().dgw_batch_schedule(self._h, int(dim), int(p), ctypes.byref(rows), ctypes.byref(chunk)))
        return rows.value, chunk.value

    def set_schedule(self, dim: int, p: int, rows: int, chunk: int):
        _check(load().dgw_batch_set_schedule(self._h, int(dim), int(p), int(rows), int(chunk)))

    def debug(self, wait_limit: int, unreachable: bool):
        _check(load().dgw_batch_debug(self._h, int(wait_limit), 1 if unreachable else 0))


def rk_step_noalloc(problem: Problem, U, dt: float, nsteps: int = 1, stream=None):
    """dgw_rk_step_noalloc: SSP-RK3 steps with the stage states in the library's fixed
    device array (no allocation; see include/dgw.h for the size limit and the rules)."""
    import torch
    want = torch.float64 if problem.prec == "fp64" else torch.float32
    if not U.is_cuda or U.dtype != want or not U.is_contiguous() or U.numel() != problem.K * problem.E:
        raise ValueError(f"state must be a contiguous CUDA {want} tensor of {problem.K}x{problem.E}")
    m, f, s = problem.c_structs()
    _check(load().dgw_rk_step_noalloc(ctypes.byref(m), problem.p, ctypes.byref(f), ctypes.byref(s), _ptr(U),
                                      float(dt), int(nsteps), _stream(stream)))


def selftest_sincos(x, stream=None):
    """sin and cos of a CUDA float32 tensor by the kernels' reduced-argument path."""
    import torch
    if x.dtype != torch.float32 or not x.is_cuda or not x.is_contiguous():
        raise ValueError("x must be a contiguous CUDA float32 tensor")
    s, c = torch.empty_like(x), torch.empty_like(x)
    _check(load().dgw_selftest_sincos(_ptr(x), _ptr(s), _ptr(c), x.numel(), _stream(stream)))
    return s, c


def version() -> str:
    return load().dgw_version().decode()


def selftest_tc_volume(U, out, variant: int, stream=None) -> float:
    """The Q3 KPP volume term of U (float [16][ntiles * 128]) into out, on the CUDA cores
    (variant 0) or the tensor cores (variant 1); returns the kernel's time in ms
    (dgw_selftest_tc_volume)."""
    if U.numel() % (16 * 128) or out.numel() != U.numel():
        raise ValueError("U and out: float [16][ntiles * 128]")
    ms = ctypes.c_float()
    _check(load().dgw_selftest_tc_volume(_ptr(U), _ptr(out), U.numel() // (16 * 128), int(variant),
                                          ctypes.byref(ms), _stream(stream)))
    return ms.value

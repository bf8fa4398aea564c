"""dgw_rk_step_noalloc: SSP-RK3 steps for callers that cannot allocate device memory
(applications whose device memory belongs to another allocator, real-time code that may
not allocate after start-up).  It must give the same states as dgw_create + dgw_rk_step,
call after call, with its stage states in the library's fixed device array.  This file is
collected last on purpose."""
import ctypes

import numpy as np
import pytest

import helpers as H
from paper_2309_12019_gb300 import dgw


def _call(problem, U, dt, nsteps, stream):
    L = dgw.load()
    m, f, s = problem.c_structs()
    return L.dgw_rk_step_noalloc(ctypes.byref(m), problem.p, ctypes.byref(f), ctypes.byref(s),
                                 ctypes.c_void_p(U.data_ptr()), float(dt), int(nsteps), ctypes.c_void_p(stream))


def test_noalloc_rejects_oversized_state():
    """Checked before any device work, so it runs without a GPU too."""
    L = dgw.load()
    P = dgw.Problem(**H.spec(2, 3, 1024, flux="kpp", bc="outflow"), prec="fp32")   # 67 MB state
    m, f, s = P.c_structs()
    rc = L.dgw_rk_step_noalloc(ctypes.byref(m), P.p, ctypes.byref(f), ctypes.byref(s),
                               ctypes.c_void_p(16), 1e-4, 1, None)
    assert rc == -1
    assert "exceeds the fixed stage capacity" in L.dgw_last_error().decode()


@pytest.mark.gpu
@pytest.mark.parametrize("dim,p,flux,bc,prec,n", [
    (2, 2, "rotation", "inflow_zero", "fp64", 40),
    (2, 3, "kpp", "outflow", "fp32", 48),
    (1, 2, "burgers", "periodic", "fp64", 200),
])
def test_noalloc_matches_context_path(dim, p, flux, bc, prec, n):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    s = H.spec(dim, p, n, flux=flux, bc=bc)
    P = dgw.Problem(**s, prec=prec)
    U0 = H.state_for(s, seed=77)
    dtype = torch.float64 if prec == "fp64" else torch.float32
    dt = 0.02 / n
    stream = torch.cuda.Stream()
    ctx = dgw.Context(P)
    Uref = torch.tensor(U0, dtype=dtype, device="cuda")
    Unew = Uref.clone()
    tol = 1e-12 if prec == "fp64" else 2e-5
    for call in range(2):   # two calls in a row, each continuing from the last state
        with torch.cuda.stream(stream):
            ctx.rk_step(Uref, dt, 3)
            rc = _call(P, Unew, dt, 3, stream.cuda_stream)
            assert rc == 0, dgw.load().dgw_last_error().decode()
        stream.synchronize()
        assert H.rel_l2(Unew.double().cpu().numpy(), Uref.double().cpu().numpy()) <= tol, call
        # the same stage kernels with the same tables and launch shapes (the context path
        # replays them from a graph, which changes no bit), so the states agree exactly
        assert torch.equal(Unew, Uref), call
    ctx.close()

"""The C ABI without a GPU: the library loads, exports every entry point that
include/dgw.h declares, and rejects bad arguments synchronously (before touching the
device)."""
import ctypes
import os
import re

import pytest

from paper_2309_12019_gb300 import dgw

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "dgw.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dgw_[a-z_0-9]+)\s*\(", src)))


def test_header_and_binding_agree():
    assert declared_functions() == sorted(dgw.EXPORTS)


def test_library_exports_every_declared_symbol():
    L = dgw.load()
    for name in declared_functions():
        assert hasattr(L, name), name
    assert dgw.version().startswith("dgw")


def _create(**kw):
    L = dgw.load()
    P = dgw.Problem(**{**dict(dim=2, nx=8, ny=8, p=2), **kw})
    m, f, s = P.c_structs()
    h = ctypes.c_void_p()
    rc = L.dgw_create(ctypes.byref(m), P.p, ctypes.byref(f), ctypes.byref(s), ctypes.byref(h))
    if rc == 0:
        L.dgw_destroy(h)
    return rc, L.dgw_last_error().decode()


@pytest.mark.parametrize("kw,status", [
    (dict(dim=3), -1), (dict(nx=0), -1), (dict(p=0), -4), (dict(p=4), -4),
    (dict(box=(0.0, 1.0, 0.0, 2.0)), -4),              # non-square cells
    (dict(bc=("periodic", "outflow", "periodic", "periodic")), -1),
    (dict(b=1.5), -1), (dict(q=0.0), -1), (dict(w_nbr=0.3), -1), (dict(eps_w=0.0), -1),
    (dict(lambda_nu=-1.0), -1),
    # the Euler system: reflecting walls only with it, inflow_zero only without it
    (dict(flux="euler", bc=("periodic", "periodic", "inflow_zero", "outflow")), -1),
    (dict(dim=1, bc=("reflect", "reflect", "periodic", "periodic")), -1),
    (dict(dim=1, flux="euler", bc=("inflow_zero", "outflow", "periodic", "periodic")), -1),
    (dict(dim=1, flux="euler", gas_gamma=1.0), -1),
    (dict(dim=1, flux="euler", gas_gamma=float("nan")), -1),
])
def test_bad_arguments_rejected(kw, status):
    rc, msg = _create(**kw)
    assert rc == status and msg


def test_null_arguments():
    L = dgw.load()
    assert L.dgw_create(None, 2, None, None, None) == -1
    assert L.dgw_residual(None, None, None, None) == -1
    assert L.dgw_destroy(None) == 0


def test_defaults():
    L = dgw.load()
    m, f, s = dgw.Mesh(), dgw.Flux(), dgw.Params()
    L.dgw_defaults(ctypes.byref(m), ctypes.byref(f), ctypes.byref(s))
    assert (m.dim, s.stab, s.q, s.b, s.w_nbr, s.eps_w) == (1, 2, 1.0, 0.1, 1e-2, 1e-6)
    assert f.gas_gamma == 1.4

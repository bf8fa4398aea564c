"""Batched ensemble (dgw_batch_*): independent instances of uneven size, degree and
dimension advanced by the persistent kernels, against the oracle instance by instance
and against the single-mesh context path."""
import ctypes

import numpy as np
import pytest

import helpers as H
from paper_2309_12019_gb300 import dgw

torch = pytest.importorskip("torch")

MIX = [  # dim, p, n (cells per side), flux
    (1, 1, 100, "burgers"), (1, 2, 129, "burgers"), (1, 3, 300, "burgers"), (1, 2, 7, "burgers"),
    (2, 1, 17, "advect"), (2, 2, 33, "advect"), (2, 3, 40, "advect"), (2, 2, 5, "advect"),
    (2, 3, 12, "advect"), (1, 1, 1, "burgers"),
]


def _specs(seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for dim, p, n, fl in MIX:
        s = H.spec(dim, p, n, flux=fl)
        if fl == "advect":
            th = rng.uniform(0, 2 * np.pi)
            s["a"] = (float(np.cos(th)), float(np.sin(th)))
        out.append(s)
    return out


def _batch(specs, prec):
    return dgw.Batch([dgw.Problem(**s) for s in specs], prec=prec)


def _pack(b, states, dtype):
    U = torch.zeros(b.total, dtype=dtype, device="cuda")
    for i, Ui in enumerate(states):
        b.view(U, i).copy_(torch.tensor(Ui, dtype=dtype))
    return U


pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_batch_fp64_matches_oracle(oracle_mod):
    specs = _specs()
    b = _batch(specs, "fp64")
    states = [H.state_for(s, seed=900 + i) for i, s in enumerate(specs)]
    dts = [0.005 / s["nx"] for s in specs]   # CFL ~0.015 on these random states
    b.set_dt(dts)
    U = _pack(b, states, torch.float64)
    b.rk_step(U, 6)
    b.sync_status()
    for i, s in enumerate(specs):
        ref = oracle_mod.rk3(oracle_mod.Problem(**s), states[i], dts[i], 6)
        got = b.view(U, i).cpu().numpy()
        assert H.rel_l2(got, ref) <= 1e-12, (i, s)


def test_batch_fp32_matches_context_path():
    """Same arithmetic as dgw_rk_step instance by instance (the batch stages tiles with
    plain L2 loads, the context path with TMA): agreement to float rounding."""
    specs = _specs(1)
    b = _batch(specs, "fp32")
    states = [H.state_for(s, seed=950 + i) for i, s in enumerate(specs)]
    dts = [0.005 / s["nx"] for s in specs]   # CFL ~0.015 on these random states
    b.set_dt(dts)
    U = _pack(b, states, torch.float32)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        b.rk_step(U, 10)
    st.synchronize()
    for i, s in enumerate(specs):
        ctx = dgw.Context(dgw.Problem(**s, prec="fp32"))
        Ui = torch.tensor(states[i], dtype=torch.float32, device="cuda")
        ctx.rk_step(Ui, dts[i], 10)
        torch.cuda.synchronize()
        assert H.rel_l2(b.view(U, i).double().cpu().numpy(), Ui.double().cpu().numpy()) <= 1e-6, i
        ctx.close()


def test_batch_autotune_and_repeatability():
    specs = _specs(2)
    b = _batch(specs, "fp32")
    states = [H.state_for(s, seed=990 + i) for i, s in enumerate(specs)]
    b.set_dt([0.005 / s["nx"] for s in specs])
    U0 = _pack(b, states, torch.float32)
    U1 = U0.clone()
    b.rk_step(U1, 5)
    chunk = b.autotune(U0, steps=2)
    assert chunk in (1, 2, 4, 8, 16)
    for dim, p in ((1, 1), (1, 2), (1, 3), (2, 1), (2, 2), (2, 3)):
        rows, c = b.schedule(dim, p)
        assert rows in ((1,) if dim == 1 else (2, 4, 8)) and c in (1, 2, 4, 8, 16)
    U2 = U0.clone()        # autotuning worked on a copy: U0 is untouched
    b.rk_step(U2, 5)
    torch.cuda.synchronize()
    b.sync_status()
    assert torch.equal(U1, U2)     # the schedule changes, not the arithmetic


@pytest.mark.parametrize("rows,chunk", [(2, 1), (8, 16), (4, 3)])
def test_batch_tile_heights_bitwise(rows, chunk):
    """Every tile height of the 2D float batch kernels (and odd work-item sizes) gives the
    same bits as the default schedule; heights that are not built are refused."""
    specs = _specs(5)
    b = _batch(specs, "fp32")
    states = [H.state_for(s, seed=970 + i) for i, s in enumerate(specs)]
    b.set_dt([0.005 / s["nx"] for s in specs])
    U0 = _pack(b, states, torch.float32)
    U1 = U0.clone()
    b.rk_step(U1, 4)
    for p in (1, 2, 3):
        b.set_schedule(2, p, rows, chunk)
        b.set_schedule(1, p, 1, chunk)
    U2 = U0.clone()
    b.rk_step(U2, 4)
    torch.cuda.synchronize()
    b.sync_status()
    assert torch.equal(U1, U2)
    with pytest.raises(dgw.DGWError):
        b.set_schedule(2, 2, 3, 4)
    with pytest.raises(dgw.DGWError):
        b.set_schedule(1, 2, 4, 4)


def test_ensemble_fp32_members_match_oracle(oracle_mod):
    """FP32 members of the 512-instance ensemble workload (the smooth ones, without unit
    steps: the 6 smallest 1D and 3 smallest 2D) against the FP64 oracle after 10 steps:
    relative L2 <= 2e-5 and every cell within 4e-4 of the RMS cell norm."""
    from paper_2309_12019_gb300 import inputs as I
    insts = I.ensemble_instances(512)
    size = lambda i: insts[i]["nx"] * insts[i]["ny"]
    smooth = [i for i in range(512) if len(insts[i]["init"]["lo"]) == 0]
    pick = (sorted([i for i in smooth if insts[i]["dim"] == 1], key=size)[:6] +
            sorted([i for i in smooth if insts[i]["dim"] == 2], key=size)[:3])
    specs, refs, samples = [], [], []
    for i in pick:
        d = insts[i]
        s = dict(dim=d["dim"], nx=d["nx"], ny=d["ny"], p=d["p"], box=(0.0, 1.0, 0.0, 1.0),
                 bc=("periodic",) * 4, flux=d["flux"], a=d["a"], stab="weno")
        X, Y = I.sample_points(d["dim"], d["nx"], d["ny"], s["box"], 8)
        f = I.u0_fourier_steps(d["init"], X, Y)
        samples.append(f.reshape(-1))
        refs.append(oracle_mod.project(oracle_mod.Problem(**s), f))
        specs.append(s)
    b = _batch(specs, "fp32")
    dts = [insts[i]["dt"] for i in pick]
    b.set_dt(dts)
    U = torch.zeros(b.total, dtype=torch.float32, device="cuda")
    b.project(torch.tensor(np.concatenate(samples), device="cuda"), U, nq=8)
    b.rk_step(U, 10)
    b.sync_status()
    for j, s in enumerate(specs):
        ref = oracle_mod.rk3(oracle_mod.Problem(**s), refs[j], dts[j], 10)
        got = b.view(U, j).double().cpu().numpy()
        assert H.rel_l2(got, ref) <= 2e-5, (j, s["dim"], s["p"], s["nx"])
        assert H.cell_err(got, ref) <= 4e-4, (j, s["dim"], s["p"], s["nx"])


def test_batch_bounded_wait_gives_up():
    """A wait that can never be satisfied (each item asks for one tile more than its
    instance has) gives up after its spin limit: the launch ends, the status is
    DGW_ETIMEOUT, and the batch is usable afterwards."""
    specs = _specs(3)
    b = _batch(specs, "fp32")
    states = [H.state_for(s, seed=7 + i) for i, s in enumerate(specs)]
    b.set_dt([0.005 / s["nx"] for s in specs])
    U = _pack(b, states, torch.float32)
    b.debug(wait_limit=2000, unreachable=True)
    b.rk_step(U, 3)
    with pytest.raises(dgw.DGWError) as ei:
        b.sync_status()
    assert ei.value.status == -5
    b.debug(wait_limit=1 << 24, unreachable=False)
    U = _pack(b, states, torch.float32)
    b.rk_step(U, 3)
    b.sync_status()
    assert torch.isfinite(U).all()


def test_batch_rejects_unsupported_flux():
    L = dgw.load()
    P = dgw.Problem(**H.spec(2, 2, 8, flux="kpp"))
    m, f, s = P.c_structs()
    ps = (ctypes.c_int * 1)(2)
    h = ctypes.c_void_p()
    assert L.dgw_batch_create(1, ctypes.byref(m), ps, ctypes.byref(f), ctypes.byref(s), ctypes.byref(h)) == -4


def test_ensemble_workload_instances_match_oracle(oracle_mod):
    """Instances of the 512-member ensemble workload itself (their own sizes, degrees,
    fluxes, initial data and time steps; the 8 smallest 1D and 4 smallest 2D ones, to
    keep the oracle quick): both sides project the same samples, then the FP64 batch is
    compared with the oracle after 4 steps."""
    from paper_2309_12019_gb300 import inputs as I
    insts = I.ensemble_instances(512)
    size = lambda i: insts[i]["nx"] * insts[i]["ny"]
    pick = (sorted([i for i in range(512) if insts[i]["dim"] == 1], key=size)[:8] +
            sorted([i for i in range(512) if insts[i]["dim"] == 2], key=size)[:4])
    specs, refs, samples = [], [], []
    for i in pick:
        d = insts[i]
        s = dict(dim=d["dim"], nx=d["nx"], ny=d["ny"], p=d["p"], box=(0.0, 1.0, 0.0, 1.0),
                 bc=("periodic",) * 4, flux=d["flux"], a=d["a"], stab="weno")
        X, Y = I.sample_points(d["dim"], d["nx"], d["ny"], s["box"], 8)
        f = I.u0_fourier_steps(d["init"], X, Y)
        samples.append(f.reshape(-1))
        refs.append(oracle_mod.project(oracle_mod.Problem(**s), f))
        specs.append(s)
    b = _batch(specs, "fp64")
    dts = [insts[i]["dt"] for i in pick]
    b.set_dt(dts)
    U = torch.zeros(b.total, dtype=torch.float64, device="cuda")
    b.project(torch.tensor(np.concatenate(samples), device="cuda"), U, nq=8)
    b.rk_step(U, 4)
    b.sync_status()
    for j, s in enumerate(specs):
        ref = oracle_mod.rk3(oracle_mod.Problem(**s), refs[j], dts[j], 4)
        assert H.rel_l2(b.view(U, j).cpu().numpy(), ref) <= 1e-12, (j, s["dim"], s["p"], s["nx"])


def test_batch_zhao_fp64_matches_oracle(oracle_mod):
    """The batch kernels with the Zhao et al. sensor (stab = zhao), against the oracle."""
    specs = [dict(s, stab="zhao") for s in _specs(4)]
    b = _batch(specs, "fp64")
    states = [H.state_for(s, seed=930 + i) for i, s in enumerate(specs)]
    dts = [0.005 / s["nx"] for s in specs]
    b.set_dt(dts)
    U = _pack(b, states, torch.float64)
    b.rk_step(U, 4)
    b.sync_status()
    for i, s in enumerate(specs):
        ref = oracle_mod.rk3(oracle_mod.Problem(**s), states[i], dts[i], 4)
        assert H.rel_l2(b.view(U, i).cpu().numpy(), ref) <= 1e-12, (i, s)

"""Parity of the 1D Euler kernel (Sec. 5.6) with the FP64 oracle, through the C ABI.

Bars (written in each test): FP64 residuals, sensors and short RK3 runs to 1e-12
relative L2 (|d gamma| <= 1e-12); the full Sod run (about 2200 stages) to 1e-9, the
rounding differences of that many nonlinear stages; FP32 residuals on float-rounded
input to 1e-5 relative L2 per component, FP32 RK3 runs to 2e-5.  Meshes of 300 cells
span three 128-cell tiles and a ragged tail.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import helpers as H
from paper_2309_12019_gb300 import dgw
from paper_2309_12019_gb300 import inputs as I

pytestmark = pytest.mark.gpu

BCS = {"periodic": ("periodic", "periodic"), "reflect": ("reflect", "reflect"),
       "wall_out": ("reflect", "outflow"), "outflow": ("outflow", "outflow")}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dgw.load()


def spec(p, nx=300, stab="weno", bc="wall_out", box=None, **kw):
    box = box or (0.0, 1.0)
    return dict(dim=1, nx=nx, p=p, box=(box[0], box[1], 0.0, 1.0), bc=BCS[bc] + ("periodic", "periodic"),
                flux="euler", stab=stab, **kw)


def ctx_for(s, prec="fp64"):
    return dgw.Context(dgw.Problem(**s, prec=prec))


def dev(U, prec):
    return torch.tensor(U, dtype=torch.float64 if prec == "fp64" else torch.float32, device="cuda").contiguous()


def residual(ctx, U):
    Ud = dev(U, ctx.problem.prec)
    L = torch.empty_like(Ud)
    ctx.residual(Ud, L)
    torch.cuda.synchronize()
    return L.double().cpu().numpy()


def per_comp_rel(got, ref, p):
    n1 = p + 1
    return max(H.rel_l2(got[c * n1:(c + 1) * n1], ref[c * n1:(c + 1) * n1]) for c in range(3))


def per_comp_cell(got, ref, p, dim=1):
    """Largest per-cell error of any component (helpers.cell_err)."""
    K = (p + 1) ** dim
    return max(H.cell_err(got[c * K:(c + 1) * K], ref[c * K:(c + 1) * K]) for c in range(dim + 2))


# per-cell FP32 bars: one residual on a float-rounded state, and 20 steps of a shock tube
# (where the float and double runs differ most next to the shocks)
FP32_CELL_TOL = 1e-4
FP32_CELL_TOL_STEPS = 1e-3


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("stab", ["dg", "lo", "weno", "zhao"])
@pytest.mark.parametrize("bc", sorted(BCS))
def test_residual_fp64(oracle_mod, p, stab, bc):
    s = spec(p, stab=stab, bc=bc)
    U = I.random_euler_state(p, s["nx"], seed=10 * p + len(stab) + len(bc), amp=0.1)
    ref = oracle_mod.residual(oracle_mod.Problem(**s), U)
    assert per_comp_rel(residual(ctx_for(s), U), ref, p) <= 1e-12


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("stab", ["weno", "zhao"])
def test_sensor_fp64(oracle_mod, p, stab):
    s = spec(p, stab=stab, bc="reflect")
    U = I.random_euler_state(p, s["nx"], seed=40 + p, amp=0.1)
    ref = oracle_mod.sensor(oracle_mod.Problem(**s), U)[0]
    ctx = ctx_for(s)
    g = torch.empty(ctx.E, dtype=torch.float64, device="cuda")
    ctx.sensor(dev(U, "fp64"), g)
    torch.cuda.synchronize()
    assert np.max(np.abs(g.cpu().numpy() - ref)) <= 1e-12
    assert np.mean(ref > 1e-3) > 0.05


def test_fixed_lambda_fp64(oracle_mod):
    s = spec(2, stab="lo", bc="periodic", lambda_nu=3.0)
    U = I.random_euler_state(2, s["nx"], seed=3, amp=0.1)
    ref = oracle_mod.residual(oracle_mod.Problem(**s), U)
    assert per_comp_rel(residual(ctx_for(s), U), ref, 2) <= 1e-12


@pytest.mark.parametrize("p,bc,rk", [(1, "reflect", 3), (2, "wall_out", 3), (3, "periodic", 3),
                                      (2, "reflect", 2), (2, "outflow", 4)])
def test_rk_fp64_random(oracle_mod, p, bc, rk):
    s = spec(p, stab="weno", bc=bc)
    U = I.random_euler_state(p, s["nx"], seed=60 + p, amp=0.05)
    dt = I.euler_cfl(p) / s["nx"] / 3.0
    ref = oracle_mod.rk(oracle_mod.Problem(**s), U, dt, 6, rk)
    ctx = dgw.Context(dgw.Problem(**s, prec="fp64", rk_order=rk))
    Ud = dev(U, "fp64")
    ctx.rk_step(Ud, dt, 6)
    torch.cuda.synchronize()
    ctx.sync_status()
    assert per_comp_rel(Ud.cpu().numpy(), ref, p) <= 1e-12


def _shock_tube(name, nx, p):
    d = I.SHOCK_TUBES[name]
    s = spec(p, nx=nx, stab="weno", bc="reflect", box=d["box"])
    s["bc"] = tuple(d["bc"]) + ("periodic", "periodic")
    n, dt, last = I.nsteps_to(d["t_end"], I.euler_cfl(p) * (d["box"][1] - d["box"][0]) / nx / d["lam"])
    return s, n, dt, last


@pytest.mark.parametrize("name,nx,p,nmax", [("sod", 128, 2, None), ("sod_modified", 128, 2, None),
                                            ("shu_osher", 512, 2, 400), ("shu_osher", 512, 3, 50),
                                            ("lax", 512, 2, 300)])
def test_shock_tube_fp64_runs(oracle_mod, name, nx, p, nmax):
    """Shock tubes at the paper's sizes: device projection, then every step to t_end (Sod,
    modified Sod) or the first nmax steps, against the oracle.  The sensor ratio is
    scale-free: in a cell whose slopes are at rounding level it takes O(1) values set by
    the rounding, so the two sides' different summation orders seed differences that a
    strong shock amplifies.  Shu-Osher at p = 3 agrees to 2e-12 after 50 steps and
    drifts apart beyond (2e-7 after 100 steps on GB300), hence its shorter horizon."""
    s, n, dt, last = _shock_tube(name, nx, p)
    if nmax is not None:
        n, last = min(n, nmax), 0.0
    f = I.shock_tube_samples(name, nx, 8)
    P = oracle_mod.Problem(**s)
    U0 = oracle_mod.project(P, f, 8)
    ctx = ctx_for(s)
    Ud = torch.empty((ctx.K, ctx.E), dtype=torch.float64, device="cuda")
    ctx.project(torch.tensor(f, device="cuda").contiguous(), Ud, 8)
    torch.cuda.synchronize()
    assert H.rel_l2(Ud.cpu().numpy(), U0) <= 1e-14
    ref = oracle_mod.rk3(P, U0, dt, n)
    ctx.rk_step(Ud, dt, n)
    if last > 0:
        ref = oracle_mod.rk3(P, ref, last, 1)
        ctx.rk_step(Ud, last, 1)
    torch.cuda.synchronize()
    ctx.sync_status()
    assert per_comp_rel(Ud.cpu().numpy(), ref, p) <= 1e-9
    if name == "sod":      # between reflecting walls the mass is conserved
        assert abs(ctx.mass(Ud) - oracle_mod.mass(P, U0)) <= 1e-13


@pytest.mark.parametrize("p,stab", [(1, "weno"), (2, "zhao"), (3, "weno"), (2, "lo")])
def test_residual_fp32(oracle_mod, p, stab):
    s = spec(p, stab=stab, bc="wall_out")
    U = I.random_euler_state(p, s["nx"], seed=80 + p, amp=0.1).astype(np.float32).astype(np.float64)
    ref = oracle_mod.residual(oracle_mod.Problem(**s), U)
    got = residual(ctx_for(s, "fp32"), U)
    assert per_comp_rel(got, ref, p) <= 1e-5
    assert per_comp_cell(got, ref, p) <= FP32_CELL_TOL


@pytest.mark.parametrize("name,p", [("sod", 1), ("sod", 3), ("lax", 2), ("sod_modified", 2), ("shu_osher", 3)])
def test_shock_tube_fp32_steps(oracle_mod, name, p):
    """Twenty FP32 steps of a shock tube from its projected initial data, at the paper's
    cell counts (there the modified Sod and Shu-Osher diaphragms cut a cell)."""
    d = I.SHOCK_TUBES[name]
    s, _, dt, _ = _shock_tube(name, d["nx"], p)
    f = I.shock_tube_samples(name, d["nx"], 8)
    P = oracle_mod.Problem(**s)
    U0 = oracle_mod.project(P, f, 8).astype(np.float32).astype(np.float64)
    ref = oracle_mod.rk3(P, U0, dt, 20)
    ctx = ctx_for(s, "fp32")
    Ud = dev(U0, "fp32")
    ctx.rk_step(Ud, dt, 20)
    torch.cuda.synchronize()
    ctx.sync_status()
    got = Ud.double().cpu().numpy()
    assert per_comp_rel(got, ref, p) <= 2e-5
    assert per_comp_cell(got, ref, p) <= FP32_CELL_TOL_STEPS
    assert d["t_end"] > 20 * dt


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_host_entry_matches_device_entry(prec):
    s = spec(2, nx=1000, bc="reflect")
    U = I.random_euler_state(2, s["nx"], seed=5).astype(np.float64 if prec == "fp64" else np.float32)
    ctx = ctx_for(s, prec)
    dt = 0.02 / s["nx"]
    Ud = dev(U, prec)
    ctx.rk_step(Ud, dt, 4)
    Uh = torch.tensor(U).pin_memory()
    out = torch.empty_like(Uh).pin_memory()
    ctx.rk_step_host(Uh, out, dt, 4)
    torch.cuda.synchronize()
    assert np.array_equal(out.numpy(), Ud.cpu().numpy())


def test_negative_pressure_is_reported():
    """No positivity safeguard: a state with negative pressure gives non-finite results,
    which the stage kernel flags (a NaN from a square root, no fault)."""
    s = spec(1, nx=200, stab="dg", bc="periodic")
    U = I.random_euler_state(1, s["nx"], seed=9)
    U[4, 17] = -5.0                     # rho E < rho v^2 / 2 in cell 17
    ctx = ctx_for(s)
    Ud = dev(U, "fp64")
    ctx.rk_step(Ud, 1e-4, 1)
    with pytest.raises(dgw.DGWError) as e:
        ctx.sync_status()
    assert e.value.status == -6
    ctx.sync_status()                   # the flag was cleared


def test_other_paths_refuse_the_euler_system():
    s = spec(2, nx=64, bc="periodic")
    ctx = ctx_for(s)
    U = dev(I.random_euler_state(2, 64, seed=1), "fp64")
    with pytest.raises(dgw.DGWError) as e:
        ctx.residual_vjp(U, U.clone(), torch.empty_like(U))
    assert e.value.status == -4
    with pytest.raises(dgw.DGWError) as e:
        dgw.Batch([dgw.Problem(**s)])
    assert e.value.status == -4
    with pytest.raises(dgw.DGWError) as e:
        dgw.rk_step_noalloc(dgw.Problem(**s, prec="fp64"), U, 1e-3, 1)
    assert e.value.status == -4


@pytest.mark.parametrize("prec,p,stab", [("fp64", 2, "weno"), ("fp32", 2, "zhao"), ("fp32", 3, "weno")])
def test_sod_train_steps(oracle_mod, prec, p, stab):
    """Fifty steps of the Sod-train workload (a shock tube every 64 cells, periodic) on
    4160 cells: 32 full 128-cell tiles and a ragged one of 64."""
    nx = 4160
    s = spec(p, nx=nx, stab=stab, bc="periodic")
    P = oracle_mod.Problem(**s)
    U0 = oracle_mod.project(P, I.sod_train_samples(nx), 8)
    if prec == "fp32":
        U0 = U0.astype(np.float32).astype(np.float64)
    dt = I.euler_cfl(p) / nx / 2.5
    ref = oracle_mod.rk3(P, U0, dt, 50)
    ctx = ctx_for(s, prec)
    Ud = dev(U0, prec)
    ctx.rk_step(Ud, dt, 50)
    torch.cuda.synchronize()
    ctx.sync_status()
    assert per_comp_rel(Ud.double().cpu().numpy(), ref, p) <= (1e-12 if prec == "fp64" else 2e-5)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("state", ["projected", "random"])
def test_sod_train_full_size_sampled(oracle_mod, prec, state):
    """The large-mesh workload in the bench's launch configuration (2^22 cells, p = 2):
    the residual at sampled cells (both ends, tile borders and a seeded random sample)
    against the oracle evaluated cell by cell, on the oracle's projection of the Sod
    train (the GPU projection is compared with it everywhere) and on a seeded random
    state, both rounded to the kernel precision and fed to both sides."""
    import bench
    w = bench.WORKLOADS["sod_train_4194304_q2"]
    s = bench.spec_of(w)
    P = oracle_mod.Problem(**s)
    ctx = ctx_for(s, prec)
    if state == "projected":
        f = bench.initial_samples(w)
        U0 = oracle_mod.project(P, f, 8)
        Ug = torch.empty((ctx.K, ctx.E), dtype=ctx.dtype, device="cuda")
        ctx.project(torch.tensor(f, device="cuda").contiguous(), Ug)
        torch.cuda.synchronize()
        assert H.rel_l2(Ug.double().cpu().numpy(), U0) <= (1e-14 if prec == "fp64" else 1e-7)
        del Ug
    else:
        U0 = I.random_euler_state(2, ctx.E, seed=91, amp=0.05)
    if prec == "fp32":
        U0 = U0.astype(np.float32).astype(np.float64)
    U = dev(U0, prec)
    L = torch.empty_like(U)
    ctx.residual(U, L)
    torch.cuda.synchronize()
    ctx.sync_status()
    E = ctx.E
    rng = np.random.default_rng(77)
    idx = np.unique(np.concatenate([[0, 1, 127, 128, E // 2 - 1, E // 2, E - 129, E - 128, E - 2, E - 1],
                                    np.arange(0, E, 64)[:3000] + 31, rng.integers(0, E, 3000)]))
    ref = oracle_mod.residual_at(P, U0, idx)
    got = L.double().cpu().numpy()[:, idx]
    assert per_comp_rel(got, ref, 2) <= (1e-12 if prec == "fp64" else 1e-5)


# ---------------------------------------------------------------------------------
# 2D Euler system (reading R17): meshes of 37 x 11 cells span two 32-wide tiles (one
# ragged) and three 4-row tiles (one ragged)
# ---------------------------------------------------------------------------------
BCS2 = {"periodic": ("periodic",) * 4, "walls": ("reflect",) * 4,
        "mixed": ("reflect", "outflow", "periodic", "periodic"), "mixed2": ("periodic", "periodic", "outflow", "reflect")}


def spec2(p, nx=37, ny=11, stab="weno", bc="walls", box=None, **kw):
    box = box or (0.0, nx / 16.0, 0.0, ny / 16.0)
    return dict(dim=2, nx=nx, ny=ny, p=p, box=box, bc=BCS2[bc] if isinstance(bc, str) else tuple(bc),
                flux="euler", stab=stab, **kw)


def per_comp_rel2(got, ref, p):
    K = (p + 1) ** 2
    return max(H.rel_l2(got[c * K:(c + 1) * K], ref[c * K:(c + 1) * K]) for c in range(4))


def state2(p, E, seed, amp=0.02):
    return I.random_euler_state(p, E, seed, amp=amp, dim=2)


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("stab", ["dg", "lo", "weno", "zhao"])
@pytest.mark.parametrize("bc", sorted(BCS2))
def test_2d_residual_fp64(oracle_mod, p, stab, bc):
    s = spec2(p, stab=stab, bc=bc)
    U = state2(p, 37 * 11, seed=100 * p + len(stab) + len(bc))
    ref = oracle_mod.residual(oracle_mod.Problem(**s), U)
    assert np.isfinite(ref).all()
    assert per_comp_rel2(residual(ctx_for(s), U), ref, p) <= 1e-12


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("stab", ["weno", "zhao"])
def test_2d_sensor_fp64(oracle_mod, p, stab):
    s = spec2(p, stab=stab, bc="mixed")
    U = state2(p, 37 * 11, seed=7 + p, amp=0.05)
    ref = oracle_mod.sensor(oracle_mod.Problem(**s), U)[0]
    ctx = ctx_for(s)
    g = torch.empty(ctx.E, dtype=torch.float64, device="cuda")
    ctx.sensor(dev(U, "fp64"), g)
    torch.cuda.synchronize()
    assert np.max(np.abs(g.cpu().numpy() - ref)) <= 1e-12
    assert np.mean(ref > 1e-3) > 0.05


@pytest.mark.parametrize("p,bc", [(1, "walls"), (2, "periodic"), (3, "mixed2")])
def test_2d_rk3_fp64(oracle_mod, p, bc):
    s = spec2(p, bc=bc)
    U = state2(p, 37 * 11, seed=300 + p)
    dt = I.euler_cfl(p, 2) / 16.0 / 3.0
    ref = oracle_mod.rk3(oracle_mod.Problem(**s), U, dt, 6)
    ctx = ctx_for(s)
    Ud = dev(U, "fp64")
    ctx.rk_step(Ud, dt, 6)
    torch.cuda.synchronize()
    ctx.sync_status()
    assert per_comp_rel2(Ud.cpu().numpy(), ref, p) <= 1e-12


@pytest.mark.parametrize("p,stab", [(1, "weno"), (2, "zhao"), (3, "lo")])
def test_2d_residual_fp32(oracle_mod, p, stab):
    s = spec2(p, stab=stab, bc="mixed")
    U = state2(p, 37 * 11, seed=400 + p).astype(np.float32).astype(np.float64)
    ref = oracle_mod.residual(oracle_mod.Problem(**s), U)
    got = residual(ctx_for(s, "fp32"), U)
    assert per_comp_rel2(got, ref, p) <= 1e-5
    assert per_comp_cell(got, ref, p, dim=2) <= FP32_CELL_TOL


def _problem2d(name, nx, ny, p):
    d = I.EULER_2D[name]
    s = dict(dim=2, nx=nx, ny=ny, p=p, box=d["box"], bc=d["bc"], flux="euler", stab="weno")
    if name == "double_mach":
        s.update(I.double_mach_boundary())
    dt = I.euler_cfl(p, 2) * (d["box"][1] - d["box"][0]) / nx / d["lam"]
    return s, dt, I.euler2d_samples(name, nx, ny, 8)


def rel_to_state(got, ref, p):
    """Largest component error over the largest component norm: the momenta of these
    problems start at or near zero, so their own norms are no scale for rounding."""
    K = (p + 1) ** 2
    scale = max(np.linalg.norm(ref[c * K:(c + 1) * K]) for c in range(4))
    return max(np.linalg.norm(got[c * K:(c + 1) * K] - ref[c * K:(c + 1) * K]) for c in range(4)) / scale


@pytest.mark.parametrize("name,nx,ny", [("kelvin_helmholtz", 32, 32), ("triple_point", 56, 24),
                                        ("rarefaction_1", 32, 32), ("rarefaction_2", 32, 32)])
@pytest.mark.parametrize("prec,stab,bar", [("fp64", "lo", 1e-12), ("fp64", "weno", 1e-9), ("fp32", "weno", 2e-5)])
def test_2d_problems_steps(oracle_mod, name, nx, ny, prec, stab, bar):
    """The paper's 2D problems on reduced meshes: device projection, then 20 steps.  With
    the WENO sensor the FP64 bar is looser: the sensor, computed from the density, is
    scale-free and ill-conditioned where the density is flat to rounding (the
    Kelvin-Helmholtz layers away from the shear), and the two sides' rounding there
    moves gamma, which also scales the stabilization of the momenta."""
    s, dt, f = _problem2d(name, nx, ny, 2)
    s["stab"] = stab
    P = oracle_mod.Problem(**s)
    U0 = oracle_mod.project(P, f, 8)
    ctx = ctx_for(s, prec)
    Ud = torch.empty((ctx.K, ctx.E), dtype=ctx.dtype, device="cuda")
    ctx.project(torch.tensor(f, device="cuda").contiguous(), Ud, 8)
    torch.cuda.synchronize()
    assert H.rel_l2(Ud.double().cpu().numpy(), U0) <= (1e-14 if prec == "fp64" else 1e-7)
    if prec == "fp32":
        U0 = U0.astype(np.float32).astype(np.float64)
    Ud = dev(U0, prec)                  # both sides step from the oracle's projection
    ref = oracle_mod.rk3(P, U0, dt, 20)
    ctx.rk_step(Ud, dt, 20)
    torch.cuda.synchronize()
    ctx.sync_status()
    assert rel_to_state(Ud.double().cpu().numpy(), ref, 2) <= bar


@pytest.mark.parametrize("prec,stab,bar", [("fp64", "weno", 1e-12), ("fp32", "lo", 1e-5), ("fp32", "weno", 1e-5)])
def test_2d_full_size_sampled(oracle_mod, prec, stab, bar):
    """The paper's Kelvin-Helmholtz mesh (512^2 cells, p = 2, periodic) in the bench's
    launch configuration: the residual of a seeded random state (rounded to the kernel
    precision, fed to both sides) at ~2000 sampled cells (corners, tile borders, random)
    against the oracle cell by cell; the GPU projection of the Kelvin-Helmholtz data is
    compared with the oracle's everywhere."""
    s, dt, f = _problem2d("kelvin_helmholtz", 512, 512, 2)
    s["stab"] = stab
    P = oracle_mod.Problem(**s)
    ctx = ctx_for(s, prec)
    Ug = torch.empty((ctx.K, ctx.E), dtype=ctx.dtype, device="cuda")
    ctx.project(torch.tensor(f, device="cuda").contiguous(), Ug, 8)
    torch.cuda.synchronize()
    assert H.rel_l2(Ug.double().cpu().numpy(), oracle_mod.project(P, f, 8)) <= (1e-14 if prec == "fp64" else 1e-7)
    del Ug
    U0 = state2(2, 512 * 512, seed=93)
    if prec == "fp32":
        U0 = U0.astype(np.float32).astype(np.float64)
    U = dev(U0, prec)
    L = torch.empty_like(U)
    ctx.residual(U, L)
    torch.cuda.synchronize()
    ctx.sync_status()
    rng = np.random.default_rng(5)
    rows = [0, 3, 4, 127, 128, 255, 256, 383, 384, 511]
    idx = np.unique(np.concatenate([[r * 512 + c for r in rows for c in (0, 31, 32, 255, 511)],
                                    rng.integers(0, 512 * 512, 1500)]))
    ref = oracle_mod.residual_at(P, U0, idx)
    got = L.double().cpu().numpy()[:, idx]
    assert per_comp_rel2(got, ref, 2) <= bar


def test_2d_host_entry_and_negative_pressure():
    s = spec2(2, bc="walls")
    U = state2(2, 37 * 11, seed=11)
    ctx = ctx_for(s)
    Ud = dev(U, "fp64")
    ctx.rk_step(Ud, 1e-3, 3)
    Uh = torch.tensor(U).pin_memory()
    out = torch.empty_like(Uh).pin_memory()
    ctx.rk_step_host(Uh, out, 1e-3, 3)
    torch.cuda.synchronize()
    assert np.array_equal(out.numpy(), Ud.cpu().numpy())
    U[3 * 9, 50] = -5.0                 # rho E < rho |v|^2 / 2 in cell 50
    Ud = dev(U, "fp64")
    ctx.rk_step(Ud, 1e-4, 1)
    with pytest.raises(dgw.DGWError) as e:
        ctx.sync_status()
    assert e.value.status == -6


def _golden_ranges():
    import os
    rows = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "euler2d_density_ranges.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            name, stab, lo, hi = line.split()
            rows[(name, stab)] = (float(lo), float(hi))
    return rows


@pytest.mark.parametrize("name", ["rarefaction_1", "rarefaction_2"])
@pytest.mark.parametrize("stab", ["lo", "weno"])
def test_2d_rarefaction_density_ranges_match_the_paper(name, stab):
    """The rarefaction interactions at the paper's 256^2 cells, p = 2, FP64, run to the
    paper's final times on the GPU: the range of the density cell means matches the range
    the paper prints for its LO and WENO solutions to 0.003 (its values are taken on its
    own nodes; the unstabilized DG extremes depend on them and are not compared)."""
    lo, hi = _golden_ranges()[(name, stab)]
    d = I.EULER_2D[name]
    s = dict(dim=2, nx=256, ny=256, p=2, box=d["box"], bc=d["bc"], flux="euler", stab=stab)
    ctx = ctx_for(s)
    U = torch.empty((ctx.K, ctx.E), dtype=torch.float64, device="cuda")
    ctx.project(torch.tensor(I.euler2d_samples(name, 256, 256, 8), device="cuda").contiguous(), U, 8)
    n, dt, last = I.nsteps_to(d["t_end"], I.euler_cfl(2, 2) / 256 / d["lam"])
    ctx.rk_step(U, dt, n)
    if last > 0:
        ctx.rk_step(U, last, 1)
    torch.cuda.synchronize()
    ctx.sync_status()
    rho = U[0].cpu().numpy()
    assert abs(rho.min() - lo) <= 3e-3 and abs(rho.max() - hi) <= 3e-3, (rho.min(), rho.max(), lo, hi)


def test_2d_kelvin_helmholtz_lo_range_matches_the_paper():
    """Kelvin-Helmholtz at the paper's 512^2 cells, p = 2, to t = 1 (30,720 steps), FP32,
    LO: the density cell means span the paper's printed LO range to 0.003.  (The WENO
    solution's vortices are sensitive to every rounding; its range is reported, not
    held.)"""
    name = "kelvin_helmholtz"
    lo, hi = _golden_ranges()[(name, "lo")]
    d = I.EULER_2D[name]
    s = dict(dim=2, nx=512, ny=512, p=2, box=d["box"], bc=d["bc"], flux="euler", stab="lo")
    ctx = ctx_for(s, "fp32")
    U = torch.empty((ctx.K, ctx.E), dtype=torch.float32, device="cuda")
    ctx.project(torch.tensor(I.euler2d_samples(name, 512, 512, 8), device="cuda").contiguous(), U, 8)
    n, dt, last = I.nsteps_to(d["t_end"], I.euler_cfl(2, 2) / 512 / d["lam"])
    ctx.rk_step(U, dt, n)
    if last > 0:
        ctx.rk_step(U, last, 1)
    torch.cuda.synchronize()
    ctx.sync_status()
    rho = U[0].double().cpu().numpy()
    assert abs(rho.min() - lo) <= 3e-3 and abs(rho.max() - hi) <= 3e-3, (rho.min(), rho.max(), lo, hi)


@pytest.mark.parametrize("rk", [2, 4])
def test_2d_rk_orders_fp64(oracle_mod, rk):
    """The SSP Runge-Kutta schemes of order 2 and 4 on the 2D Euler system against the
    oracle's (six steps, walls, p = 2)."""
    s = spec2(2, bc="walls")
    U = state2(2, 37 * 11, seed=500 + rk)
    dt = I.euler_cfl(2, 2) / 16.0 / 3.0
    ref = oracle_mod.rk(oracle_mod.Problem(**s), U, dt, 6, rk)
    ctx = dgw.Context(dgw.Problem(**s, prec="fp64", rk_order=rk))
    Ud = dev(U, "fp64")
    ctx.rk_step(Ud, dt, 6)
    torch.cuda.synchronize()
    ctx.sync_status()
    assert per_comp_rel2(Ud.cpu().numpy(), ref, 2) <= 1e-12


# ---------------------------------------------------------------------------------
# prescribed boundary states (reading R19; the double Mach reflection of Sec. 5.6)
# ---------------------------------------------------------------------------------
def _cons(rho, vx, vy, pr):
    return (rho, rho * vx, rho * vy, pr / 0.4 + 0.5 * rho * (vx * vx + vy * vy))


def smooth_state2(p, nx, ny, seed, amp=0.02):
    """A random modal state (state2) whose cell means follow smooth fields of the cell
    centre (rho, velocity and pressure within 10 % of (1.2, 0.2, -0.1, 1)): neighbouring
    cells differ by small jumps only, so that several steps keep density and pressure
    positive (state2's independent cell means collide into near-vacuum within a few
    steps)."""
    U = state2(p, nx * ny, seed, amp)
    K = (p + 1) ** 2
    j, i = np.divmod(np.arange(nx * ny), nx)
    x, y = 2 * np.pi * (i + 0.5) / nx, 2 * np.pi * (j + 0.5) / ny
    rho = 1.2 + 0.1 * np.sin(x) * np.cos(y)
    vx, vy = 0.2 + 0.1 * np.cos(x + y), -0.1 + 0.1 * np.sin(x - y)
    pr = 1.0 + 0.1 * np.cos(x) * np.sin(y)
    for c, m in enumerate(_cons(rho, vx, vy, pr)):
        U[c * K] = m
    return U


STATE_SIDES = dict(bstate=(_cons(1.1, 0.3, -0.2, 0.9), _cons(1.3, -0.1, 0.25, 1.1)),
                   bsplit=(0.171, 0.233, 0.313, 0.051), bspeed=(0.0, 0.7, -0.4, 1.3),
                   bbelow=(0, 2, 1, 0), babove=(1, 0, 2, 1))


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("stab", ["dg", "lo", "weno"])
def test_2d_prescribed_states_residual_fp64(oracle_mod, p, stab):
    """Every side prescribed (two states and walls, switching along the sides at moving
    splits), at a time set on the context: the residual against the oracle at 1e-12."""
    s = spec2(p, stab=stab, bc=("state",) * 4, **STATE_SIDES)
    U = state2(p, 37 * 11, seed=700 + p)
    ref = oracle_mod.residual(oracle_mod.Problem(**s, t=0.05), U)
    ctx = ctx_for(s)
    ctx.set_time(0.05)
    assert per_comp_rel2(residual(ctx, U), ref, p) <= 1e-12


@pytest.mark.parametrize("prec,bar,order", [("fp64", 1e-12, 3), ("fp32", 1e-5, 3), ("fp64", 1e-12, 2)])
def test_2d_prescribed_states_steps(oracle_mod, prec, bar, order):
    """Six SSP-RK3 (or SSP-RK2) steps with moving splits from t = 0.02: each stage reads
    its stage time (t, t + dt, t + dt / 2; RK2: t, t + dt) on the device; the context's
    time advances by dt per step, and the cached graph replays stay right as it moves."""
    s = spec2(2, bc=("state",) * 4, rk_order=order, **STATE_SIDES)
    U = smooth_state2(2, 37, 11, seed=733)
    if prec == "fp32":
        U = U.astype(np.float32).astype(np.float64)
    dt, n = 2e-3, 6
    so = {k: v for k, v in s.items() if k != "rk_order"}
    ref = oracle_mod.rk(oracle_mod.Problem(**so, t=0.02), U, dt, n, order=order)
    ctx = ctx_for(s, prec)
    ctx.set_time(0.02)
    Ud = dev(U, prec)
    torch.cuda.synchronize()
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        ctx.rk_step(Ud, dt, n)
    st.synchronize()
    ctx.sync_status()
    assert np.isfinite(ref).all()
    assert per_comp_rel2(Ud.double().cpu().numpy(), ref, 2) <= bar
    assert abs(ctx.get_time() - (0.02 + n * dt)) < 1e-15


def test_2d_prescribed_states_refusals():
    """Prescribed states are built for the 2D Euler system with SSP-RK of order 2 or 3."""
    for s, kw in ((dict(dim=1, nx=8, p=2, box=(0.0, 1.0, 0.0, 1.0), bc=("state", "outflow", "periodic", "periodic"),
                        flux="euler", stab="weno"), {}),
                  (H.spec(2, 2, 8, bc="outflow"), {}),
                  (spec2(2, bc=("state",) * 4, **STATE_SIDES), {"rk_order": 4})):
        if s.get("flux") != "euler":
            s = dict(s, bc=("state", "outflow", "outflow", "outflow"))
        with pytest.raises(dgw.DGWError) as ei:
            dgw.Context(dgw.Problem(**s, **kw))
        assert ei.value.status == -4


@pytest.mark.parametrize("prec,bar", [("fp64", 1e-12), ("fp32", 1e-5)])
@pytest.mark.parametrize("stab", ["lo", "weno"])
def test_2d_double_mach_residual(oracle_mod, prec, stab, bar):
    """The double Mach reflection's data and sides on a reduced mesh (48 x 12 cells,
    p = 2): the residual at t = 0 and at t = 0.05, when the split on the top side has
    moved by 0.58 (seven cells), against the oracle."""
    s, _, f = _problem2d("double_mach", 48, 12, 2)
    s["stab"] = stab
    U0 = oracle_mod.project(oracle_mod.Problem(**s), f, 8)
    if prec == "fp32":
        U0 = U0.astype(np.float32).astype(np.float64)
    ctx = ctx_for(s, prec)
    for t in (0.0, 0.05):
        ref = oracle_mod.residual(oracle_mod.Problem(**s, t=t), U0)
        ctx.set_time(t)
        assert rel_to_state(residual(ctx, U0), ref, 2) <= bar, t


@pytest.mark.parametrize("stab", ["lo", "weno"])
def test_2d_double_mach_first_step_loses_positivity(oracle_mod, stab):
    """The scheme as read loses positivity on the double Mach reflection in its first
    step: the first stage is plain DG at the shock (the sensor and the dissipation both
    vanish on the constant cells on either side) and drives the pressure at the far side
    of the pre-shock cells below zero; the second stage's wave speeds are then NaN.  The
    oracle shows it, and the GPU path reports it as DGW_ENONFINITE."""
    s, dt, f = _problem2d("double_mach", 48, 12, 2)
    s["stab"] = stab
    P = oracle_mod.Problem(**s)
    U0 = oracle_mod.project(P, f, 8)
    assert not np.isfinite(oracle_mod.rk3(P, U0, dt, 1)).all()
    ctx = ctx_for(s, "fp64")
    Ud = dev(U0, "fp64")
    ctx.rk_step(Ud, dt, 1)
    torch.cuda.synchronize()
    with pytest.raises(dgw.DGWError) as ei:
        ctx.sync_status()
    assert ei.value.status == -6

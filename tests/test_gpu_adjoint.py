"""Discrete adjoint (dgw_residual_vjp, dgw_adjoint_step, checkpointed rollout): against
central differences of the FP64 oracle (dot-product tests and full gradients), and on
the 512^2 Q2 Burgers workload against central differences of the FP64 GPU forward map
along 16 random directions (<= 1e-4 relative)."""
import numpy as np
import pytest

import helpers as H
from paper_2309_12019_gb300 import dgw
from paper_2309_12019_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _fd(fun, eps=1e-7):
    """Central difference.  The sensor ratio ||d||/||c|| makes the residual nonlinear on
    the scale r ||c||, down to ~1e-5 on these random states, so the step must be small;
    at 1e-7 the round-off of the FP64 oracle is still ~1e-9 relative."""
    return (fun(eps) - fun(-eps)) / (2 * eps)


def _mass_diag(s):
    """M_kk = (h/2)^d prod 2/(2i+1): the closed-form Legendre mass matrix."""
    p, d, h = s["p"], s["dim"], 1.0 / s["nx"]
    k = np.arange((p + 1) ** d)
    i, j = k % (p + 1), k // (p + 1)
    m = 0.5 * h * 2.0 / (2 * i + 1)
    if d == 2:
        m = m * 0.5 * h * 2.0 / (2 * j + 1)
    return m


VJP_CASES = [(1, 1, "burgers", "weno"), (1, 2, "burgers", "lo"), (1, 3, "advect", "weno"),
             (1, 3, "burgers", "weno"), (2, 1, "advect", "dg"), (2, 2, "burgers", "weno"),
             (2, 3, "burgers", "weno"), (2, 2, "advect", "lo"), (2, 1, "burgers", "weno")]


@pytest.mark.parametrize("dim,p,flux,stab", VJP_CASES)
def test_vjp_dot_product(oracle_mod, dim, p, flux, stab):
    """<J_L(U)^T lam, delta> = <lam, J_L(U) delta>, the right side by central differences of
    the oracle residual (FP64)."""
    s = H.spec(dim, p, 40 if dim == 1 else 9, flux=flux, stab=stab)
    P = oracle_mod.Problem(**s)
    U = H.state_for(s, seed=31)
    rng = np.random.default_rng(32)
    lam = rng.standard_normal(U.shape)
    delta = rng.standard_normal(U.shape)
    ctx = dgw.Context(dgw.Problem(**s, prec="fp64"))
    out = torch.empty(U.shape, dtype=torch.float64, device="cuda")
    ctx.residual_vjp(torch.tensor(U, device="cuda"), torch.tensor(lam, device="cuda"), out)
    torch.cuda.synchronize()
    lhs = float(np.sum(out.cpu().numpy() * delta))
    rhs = _fd(lambda t: float(np.sum(lam * oracle_mod.residual(P, U + t * delta))))
    assert abs(lhs - rhs) <= 1e-6 * max(abs(lhs), abs(rhs), 1.0), (lhs, rhs)


@pytest.mark.parametrize("dim,p,flux", [(1, 2, "burgers"), (2, 2, "burgers"), (2, 3, "advect")])
def test_adjoint_step_dot_product(oracle_mod, dim, p, flux):
    s = H.spec(dim, p, 32 if dim == 1 else 8, flux=flux, stab="weno")
    P = oracle_mod.Problem(**s)
    U = H.state_for(s, seed=41)
    rng = np.random.default_rng(42)
    lam = rng.standard_normal(U.shape)
    delta = rng.standard_normal(U.shape)
    dt = 0.01 / s["nx"]
    ctx = dgw.Context(dgw.Problem(**s, prec="fp64"))
    out = torch.empty(U.shape, dtype=torch.float64, device="cuda")
    ctx.adjoint_step(torch.tensor(U, device="cuda"), torch.tensor(lam, device="cuda"), out, dt)
    torch.cuda.synchronize()
    lhs = float(np.sum(out.cpu().numpy() * delta))
    rhs = _fd(lambda t: float(np.sum(lam * oracle_mod.rk3(P, U + t * delta, dt, 1))))
    assert abs(lhs - rhs) <= 1e-6 * max(abs(lhs), abs(rhs), 1.0), (lhs, rhs)


def test_rollout_gradient_matches_oracle_fd(oracle_mod):
    """Checkpointed rollout (25 steps, checkpoints every 6: a ragged last segment) of 2D
    Burgers Q2, FP64: gradient of the misfit against central differences of the oracle."""
    from paper_2309_12019_gb300 import adjoint
    s = H.spec(2, 2, 10, flux="burgers", stab="weno")
    P = oracle_mod.Problem(**s)
    U0 = H.state_for(s, seed=51)
    Ut = H.state_for(s, seed=52)
    dt, n = 0.0005, 25      # lambda dt / h ~ 0.02: inside the SSP-RK3 region with the stabilization
    M = _mass_diag(s)[:, None]
    ctx = dgw.Context(dgw.Problem(**s, prec="fp64"))
    U0t = torch.tensor(U0, device="cuda", requires_grad=True)
    J = adjoint.misfit(ctx, adjoint.rollout(ctx, U0t, dt, n, every=6), torch.tensor(Ut, device="cuda"))
    J.backward()
    g = U0t.grad.cpu().numpy()

    def J_orc(V):
        UT = oracle_mod.rk3(P, V, dt, n)
        return 0.5 * float(np.sum(M * (UT - Ut) ** 2))

    assert abs(float(J) - J_orc(U0)) <= 1e-12 * abs(J_orc(U0))
    rng = np.random.default_rng(53)
    for _ in range(4):
        v = rng.standard_normal(U0.shape)
        fd = _fd(lambda t: J_orc(U0 + t * v))
        assert abs(float(np.sum(g * v)) - fd) <= 1e-6 * abs(fd), (float(np.sum(g * v)), fd)


def test_fp32_vjp_and_gradient_match_fp64():
    """The FP32 adjoint against the FP64 adjoint of the same problem: one VJP on smooth
    projected data, and a 60-step checkpointed gradient on the adjoint workload's datum."""
    from paper_2309_12019_gb300 import adjoint
    n = 64
    s = dict(dim=2, nx=n, ny=n, p=2, box=(0.0, 1.0, 0.0, 1.0), bc=("periodic",) * 4, flux="burgers",
             a=(1.0, 1.0), stab="weno", b=0.0)
    c32 = dgw.Context(dgw.Problem(**s, prec="fp32"))
    c64 = dgw.Context(dgw.Problem(**s, prec="fp64"))
    f0 = torch.tensor(_field(s, I.adjoint_field(I.SEED + 7001)).reshape(-1), device="cuda")
    ft = torch.tensor(_field(s, I.adjoint_field(I.SEED + 7002)).reshape(-1), device="cuda")
    U32, Ut32 = (torch.empty((9, n * n), dtype=torch.float32, device="cuda") for _ in range(2))
    U64, Ut64 = (torch.empty((9, n * n), dtype=torch.float64, device="cuda") for _ in range(2))
    c32.project(f0, U32); c32.project(ft, Ut32); c64.project(f0, U64); c64.project(ft, Ut64)
    lam = torch.randn(9, n * n, dtype=torch.float64, device="cuda")
    o32, o64 = torch.empty_like(U32), torch.empty_like(U64)
    c32.residual_vjp(U32, lam.float(), o32)
    c64.residual_vjp(U64, lam, o64)
    torch.cuda.synchronize()
    assert H.rel_l2(o32.double().cpu().numpy(), o64.cpu().numpy()) <= 1e-4
    dt = I.cfl_dt(0.1, [5.0, 5.0], [1.0 / n, 1.0 / n])
    grads = []
    for c, U, Ut in ((c32, U32, Ut32), (c64, U64, Ut64)):
        Ug = U.clone().requires_grad_(True)
        adjoint.misfit(c, adjoint.rollout(c, Ug, dt, 60, every=20), Ut).backward()
        grads.append(Ug.grad.double().cpu().numpy())
    assert H.rel_l2(grads[0], grads[1]) <= 1e-4


def _field(s, params):
    X, Y = I.sample_points(2, s["nx"], s["ny"], s["box"], 8)
    return I.u0_fourier_steps(params, X, Y)


def test_burgers_512_q2_fp32_gradient_vs_fd16():
    """The adjoint workload: 2D Burgers (u^2/2, u^2/2) on the periodic unit square, 512^2
    Q2, FP32 forward and adjoint, 200 SSP-RK3 steps, checkpoints every 20, misfit against
    a target grown from another seeded field.  The FP32 gradient agrees with central
    differences of the FP64 forward map along 16 random directions to 1e-4.  The
    directions are random smooth fields (8 seeded Fourier modes, projected, unit L2 norm
    of the function): a cell-wise random vector has a projection ~1/sqrt(N) on the
    gradient and drives the sensor ratio of smooth cells across its kink at d = 0.
    The workload runs the unthresholded sensor (b = 0): with b > 0 the scheme jumps where
    a ratio crosses b, and the FP32 and FP64 trajectories, or the two sides of a central
    difference, can then take different sides in a few cells."""
    from paper_2309_12019_gb300 import adjoint
    n, steps = 512, 200
    s = dict(dim=2, nx=n, ny=n, p=2, box=(0.0, 1.0, 0.0, 1.0), bc=("periodic",) * 4, flux="burgers",
             a=(1.0, 1.0), stab="weno", b=0.0)
    pc, pt = I.adjoint_field(I.SEED + 5001), I.adjoint_field(I.SEED + 5002)
    bound = float(np.sum(pc["amp"])) + 1.0
    dt = I.cfl_dt(0.1, [bound, bound], [1.0 / n, 1.0 / n])
    c32 = dgw.Context(dgw.Problem(**s, prec="fp32"))
    c64 = dgw.Context(dgw.Problem(**s, prec="fp64"))
    U0 = torch.empty((9, n * n), dtype=torch.float32, device="cuda")
    c32.project(torch.tensor(_field(s, pc).reshape(-1), device="cuda"), U0)
    Ut = torch.empty_like(U0)
    c32.project(torch.tensor(_field(s, pt).reshape(-1), device="cuda"), Ut)
    c32.rk_step(Ut, dt, steps)
    U0g = U0.clone().requires_grad_(True)
    J = adjoint.misfit(c32, adjoint.rollout(c32, U0g, dt, steps, every=20), Ut)
    J.backward()
    g = U0g.grad.double()
    c32.sync_status()
    U0d, Utd = U0.double(), Ut.double()

    def J64(V):
        W = V.clone()
        c64.rk_step(W, dt, steps)
        return c64.misfit(W, Utd)

    rng = np.random.default_rng(54)
    M = torch.tensor(_mass_diag(s)[:, None], device="cuda")
    worst = 0.0
    for _ in range(16):
        pv = I.fourier_steps_params(2, rng, nmodes=8, max_steps=0)
        v = torch.empty_like(U0d)
        c64.project(torch.tensor(_field(s, pv).reshape(-1), device="cuda"), v)
        v /= torch.sqrt((M * v * v).sum())
        eps = 1e-4
        fd = (J64(U0d + eps * v) - J64(U0d - eps * v)) / (2 * eps)
        ad = float((g * v).sum())
        worst = max(worst, abs(ad - fd) / abs(fd))
    assert worst <= 1e-4, worst


def test_adjoint_refuses_zhao_sensor():
    """The discrete adjoint differentiates the DG, LO and WENO stabilizations; a context
    with the Zhao et al. comparison sensor gets DGW_EUNSUPPORTED, not a wrong gradient."""
    s = H.spec(2, 2, 8, flux="burgers", stab="zhao")
    ctx = dgw.Context(dgw.Problem(**s, prec="fp64"))
    U = torch.zeros((ctx.K, ctx.E), dtype=torch.float64, device="cuda")
    with pytest.raises(dgw.DGWError) as ei:
        ctx.residual_vjp(U, U.clone(), torch.empty_like(U))
    assert ei.value.status == -4
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_stored_stages_match_recomputed_adjoint_step(prec):
    """dgw_rk_step_stages writes the stage states that dgw_rk_step computes (its U^{n+1}
    equals dgw_rk_step's bit for bit), and dgw_adjoint_step_stages on them equals
    dgw_adjoint_step, which recomputes them, bit for bit."""
    s = H.spec(2, 2, 24, flux="burgers", stab="weno")
    c = dgw.Context(dgw.Problem(**s, prec=prec))
    dtype = torch.float64 if prec == "fp64" else torch.float32
    U = torch.tensor(H.state_for(s, seed=77), dtype=dtype, device="cuda")
    lam = torch.tensor(H.state_for(s, seed=78), dtype=dtype, device="cuda")
    dt = 2e-3
    ref = U.clone()
    c.rk_step(ref, dt, 1, stream=0)
    U1, U2, nxt = torch.empty_like(U), torch.empty_like(U), torch.empty_like(U)
    c.rk_step_stages(U, dt, U1, U2, nxt)
    a, b = torch.empty_like(U), torch.empty_like(U)
    c.adjoint_step(U, lam, a, dt)
    c.adjoint_step_stages(U, U1, U2, lam, b, dt)
    torch.cuda.synchronize()
    assert torch.equal(nxt, ref)
    assert torch.equal(a, b)

"""Throughput of the WENO-stabilized RKDG SSP-RK3 step on one GB300.

Workload (default): the 2D KPP problem u_t + div(sin u, cos u) = 0 on
[-2,2]x[-2.5,1.5], 1024x1024 square cells, Q3 (16 modes per cell, 16,777,216 DOFs),
FP32 state and arithmetic, outflow boundaries, lambda_e = 2, WENO sensor with q = 1,
SSP-RK3 at CFL 0.02 (dt = 3.90625e-5; the stabilization term gamma nu K limits the step:
lambda dt / h must stay below 0.044 at p = 3 in 2D).  Initial data 7 pi/2 inside the unit disc,
pi/4 outside, L2-projected by the library from 8x8 Gauss samples per cell.

A "step" is one full SSP-RK3 step (three fused stage kernels).  The metric is
DOF-updates per second per stage: 3 * N_dof * steps / time.  The three state arrays
(67 MB each) together exceed the 129 MB L2, so no explicit L2 flush is needed.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
For N > 1 (torchrun) every rank advances its own replica of the workload ("replicas
only": the single-mesh path is not sharded) and value is the sum over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2309_12019_gb300 import inputs as I  # noqa: E402

WORKLOADS = {
    "kpp_1024x1024_q3": dict(dim=2, nx=1024, ny=1024, p=3, box=(-2.0, 2.0, -2.5, 1.5),
                             bc=("outflow",) * 4, flux="kpp", lambda_nu=2.0, stab="weno",
                             cfl=0.02, speeds=(1.0, 1.0), u0="kpp"),
    "rotation_256x256_q2": dict(dim=2, nx=256, ny=256, p=2, box=(0.0, 1.0, 0.0, 1.0),
                                bc=("inflow_zero",) * 4, flux="rotation", center=(0.5, 0.5), omega=1.0,
                                stab="weno", cfl=0.05, speeds=(0.5, 0.5), u0="rotation"),
    "advect1d_128_p2": dict(dim=1, nx=128, ny=1, p=2, box=(0.0, 1.0, 0.0, 1.0), bc=("periodic",) * 4,
                            flux="advect", a=(1.0, 0.0), stab="weno", cfl=0.1, speeds=(1.0,), u0="mixed1d"),
}
# the KPP workload with the comparison sensor of Zhao et al. (Sec. 5.6) in place of Eq. (sensor),
# and with the ten-stage SSP Runge-Kutta of order 4 (order p + 1, as in Sec. 5's studies)
WORKLOADS["kpp_1024x1024_q3_zhao"] = dict(WORKLOADS["kpp_1024x1024_q3"], stab="zhao")
WORKLOADS["kpp_1024x1024_q3_rk4"] = dict(WORKLOADS["kpp_1024x1024_q3"], rk_order=4)
# the 1D Euler system (Sec. 5.6): Sod's shock tube at the paper's size (128 cells, p = 2,
# reflecting walls, to t = 0.231), and a periodic train of Sod tubes (one every 64 cells)
# on 2^22 cells as the large-mesh workload; |v| + c <= 2.5 sets the step
for _name, _nx, _p in (("sod", 128, 2), ("shu_osher", 512, 3)):
    _d = I.SHOCK_TUBES[_name]
    WORKLOADS[f"{_name}_{_nx}_q{_p}"] = dict(dim=1, nx=_nx, ny=1, p=_p, box=(_d["box"][0], _d["box"][1], 0.0, 1.0),
                                             bc=tuple(_d["bc"]) + ("periodic", "periodic"), flux="euler",
                                             stab="weno", cfl=I.euler_cfl(_p), speeds=(_d["lam"],),
                                             u0="tube:" + _name, t_end=_d["t_end"])
# the 2D Euler problems of Sec. 5.6: Kelvin-Helmholtz at the paper's 512^2 cells (p = 2, to
# t = 1.0), on 1024^2 cells (state arrays of 151 MB, above L2: the profiling case) and on
# 2048^2 cells, the triple point at 896 x 384
for _name, _nx, _ny in (("kelvin_helmholtz", 512, 512), ("kelvin_helmholtz", 1024, 1024),
                        ("kelvin_helmholtz", 2048, 2048), ("triple_point", 896, 384)):
    _d = I.EULER_2D[_name]
    WORKLOADS[f"{_name}_{_nx}x{_ny}_q2"] = dict(dim=2, nx=_nx, ny=_ny, p=2, box=_d["box"], bc=_d["bc"], flux="euler",
                                                stab="weno", cfl=I.euler_cfl(2, 2), speeds=(_d["lam"], _d["lam"]),
                                                u0="euler2d:" + _name, t_end=_d["t_end"])
WORKLOADS["sod_train_4194304_q2"] = dict(dim=1, nx=1 << 22, ny=1, p=2, box=(0.0, 1.0, 0.0, 1.0),
                                         bc=("periodic",) * 4, flux="euler", stab="weno",
                                         cfl=I.euler_cfl(2), speeds=(2.5,), u0="sod_train")
STAGES_PER_STEP = {2: 2, 3: 3, 4: 10}

SPEC_KEYS = ("dim", "nx", "ny", "p", "box", "bc", "flux", "lambda_nu", "stab", "center", "omega", "a", "rk_order")


def spec_of(w):
    return {k: w[k] for k in SPEC_KEYS if k in w}


def initial_samples(w):
    X, Y = I.sample_points(w["dim"], w["nx"], w["ny"], w["box"], 8)
    if w["u0"] == "kpp":
        f = I.u0_kpp(X, Y)
    elif w["u0"] == "rotation":
        f = I.u0_rotation(X, Y)
    elif w["u0"].startswith("euler2d:"):
        f = I.euler2d_samples(w["u0"][8:], w["nx"], w["ny"], 8)
    elif w["u0"].startswith("tube:"):
        f = I.shock_tube_samples(w["u0"][5:], w["nx"], 8)
    elif w["u0"] == "sod_train":
        f = I.sod_train_samples(w["nx"], nq=8)
    else:
        f = I.u0_mixed_1d(X)
    return np.ascontiguousarray(f.reshape(-1))


def dofs_of(w):
    """State rows times cells: (p+1)^dim modes, dim + 2 components for the Euler system."""
    return w["nx"] * w["ny"] * (w["p"] + 1) ** w["dim"] * (w["dim"] + 2 if w["flux"] == "euler" else 1)


def dt_of(w):
    h = (w["box"][1] - w["box"][0]) / w["nx"]
    if w["flux"] == "euler":        # dt = CFL h / lam, the CFL already halved in 2D
        return w["cfl"] * h / w["speeds"][0]
    return I.cfl_dt(w["cfl"], w["speeds"], [h] * w["dim"])


# DRAM bytes (read + write) per stage launch of the stage kernel at the 1024^2 Q3 KPP
# workload, averaged over the three stages of one step, as one ncu capture of the
# kernel in its current form measured them (dram__bytes_read.sum + dram__bytes_write.sum).
# None until the current kernel has been captured: the figure of an earlier kernel is
# not reported.
STAGE_TRAFFIC_BYTES = 132.2e6

# FP32 peak of one GB300 from its unit counts and maximum clock: 152 SMs x 128 FP32
# lanes x 2 flops per FMA x 2.07 GHz.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def qform_flops(p, dim):
    """Flops of one seminorm quadratic form v^T G v over the parity-class blocks of G."""
    n1 = p + 1
    k = n1 ** dim
    pairs = sum(1 for a in range(1, k) for b in range(a, k)
                if (a % n1 + b % n1) % 2 == 0 and (a // n1 + b // n1) % 2 == 0)
    return 2 * pairs + 2 * (k - 1) + 3


def _interp_sym_flops(n1, nq):
    """Flops of the values of sum_i r_i P_i at nq symmetric Gauss nodes from the even and
    odd parts (P_0 = 1 and the vanishing odd terms at the centre left out)."""
    f = (nq // 2) * (2 * (n1 - 1) + 2 - 1 + 2)     # per pair: e, o chains (first o a product), +-
    if nq % 2:
        f += 2 * len(range(2, n1, 2))
    return f


def _project_sym_flops(n1, nq, deriv):
    """Flops of sum_q W_q P_i(g_q) f_q (or P_i') for all i on symmetric nodes: sums and
    differences of the pairs, then one product per pair (and the centre where its row
    does not vanish by parity); P_0' = 0 skipped."""
    npair = nq // 2
    f = 2 * npair
    for i in range(1 if deriv else 0, n1):
        even_fn = (i % 2 == 1) if deriv else (i % 2 == 0)
        terms = npair + (1 if (nq % 2 and even_fn) else 0)
        f += 2 * terms - 1
    return f


def stage_flops_per_cell(dim, p, flux, stab):
    """FP32 flops of one stage per cell as the stage kernel evaluates it (an FMA counts 2,
    any other arithmetic operation 1): symmetric-node interpolations and projections,
    structural zeros and unit factors left out, the parity-sparse quadratic forms of the
    sensor; and the number of sin/cos pairs (KPP flux).  Faces: dim owned faces per cell."""
    n1, nq = p + 1, p + 2
    k = n1 ** dim
    kpp = flux == "kpp"
    red = 5                                        # packed 2 pi reduction of one sin/cos argument
    f = 0
    if stab in ("weno", "zhao"):                   # Hermite candidates, indicators, blend
        qf = qform_flops(p, dim)
        for axis in range(dim):
            shift = sum(2 * (n1 - 1 - ((c % n1) if axis == 0 else (c // n1))) for c in range(1, k))
            f += 2 * (shift + qf + 4 + 3 * (k - 1))
        f += 2 * qf + 2 + 3 + 1 + (k - 1) + 3
    if dim == 2:                                   # volume, one Gauss row at a time
        per_row = (2 * n1 * (n1 - 1)               # the polynomial reduced to the row
                   + _interp_sym_flops(n1, nq)     # values at the row's points
                   + _project_sym_flops(n1, nq, True) + _project_sym_flops(n1, nq, False)
                   + 2 * sum((i > 0) + (j > 0) for i in range(n1) for j in range(n1)))
        f += nq * per_row
        npts = nq * nq
    else:
        npts = nq
        f += _interp_sym_flops(n1, nq) + _project_sym_flops(n1, nq, True)
    f += npts * (red if kpp else 2)
    nfq = nq if dim == 2 else 1                    # faces: traces at the points, LLF, lift
    llf = 2 * red + 12 if kpp else 6
    if dim == 2:
        f += dim * (2 * _interp_sym_flops(n1, nq) + nfq * llf + _project_sym_flops(n1, nq, False))
    else:
        f += dim * (nfq * llf + 1)
    f += 2 * dim * k                               # face traces
    f += 4 * n1 + 2 * k if dim == 2 else 2 + 2 * n1   # face contributions
    if stab != "dg":                               # gamma nu K c
        for c in range(k):
            i, j = c % n1, c // n1
            s1 = sum(1 for m in range(1, n1) if (i + m) % 2 == 0 and i > 0)
            s2 = sum(1 for m in range(1, n1) if (j + m) % 2 == 0 and j > 0) if dim == 2 else 0
            f += 2 * (s1 + s2) + 5
    f += 6 * k                                     # M^-1 and the RK combination
    sincos = (npts + dim * nfq * 2) if kpp else 0
    return f, sincos


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        for line in (self.out or "").strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as td
        torch.cuda.set_device(local)
        td.init_process_group("nccl", device_id=torch.device("cuda", local))
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as td
        td.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as td
    dev = "cuda" if td.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    td.all_reduce(t, op=td.ReduceOp.MAX)
    return float(t.item())


def run_gpu(w, prec, steps, warmup, world, local, measure_e2e):
    import torch

    from paper_2309_12019_gb300 import dgw
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    ctx = dgw.Context(dgw.Problem(**spec_of(w), prec=prec))
    N = ctx.K * ctx.E
    stream = torch.cuda.Stream(device=dev)
    samples = torch.tensor(initial_samples(w), device=dev)
    U = torch.empty((ctx.K, ctx.E), dtype=ctx.dtype, device=dev)
    dt = dt_of(w)
    with torch.cuda.stream(stream):
        ctx.project(samples, U)
        U0 = U.clone()
        ctx.rk_step(U, dt, warmup)
    stream.synchronize()
    del samples
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        with torch.cuda.stream(stream):
            ev0.record(stream)
            ctx.rk_step(U, dt, steps)
            ev1.record(stream)
        ev1.synchronize()
    torch.cuda.synchronize()
    barrier(world)
    t_dev = ev0.elapsed_time(ev1) / 1e3
    ctx.sync_status(stream)
    stages = STAGES_PER_STEP[w.get("rk_order", 3)]
    res = dict(N=N, t=t_dev, clocks=clk.summary(), launches=stages * steps + (steps if stages == 10 else 0),
               stages=stages, mass=ctx.mass(U, stream),
               mean_range=[float(U[0].min()), float(U[0].max())])
    if measure_e2e:
        # end to end through the host-buffer entry point: H2D + step + D2H every step
        Uh = U0.cpu().pin_memory()
        Uo = torch.empty_like(Uh).pin_memory()
        for _ in range(2):
            ctx.rk_step_host(Uh, Uo, dt, 1, stream=stream)
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(steps):
            ctx.rk_step_host(Uh, Uo, dt, 1, stream=stream)
        t_e2e = time.perf_counter() - t0
        res["t_e2e"] = t_e2e
        res["bytes"] = Uh.numel() * Uh.element_size()
    ctx.close()
    return res


def run_ensemble(steps, warmup, local, n=512, autotune=True):
    """The batched ensemble: n independent 1D Burgers / 2D advection instances of uneven
    size and degree (inputs.ensemble_instances), one persistent kernel per dimension."""
    import torch

    from paper_2309_12019_gb300 import dgw
    dev = torch.device("cuda", local)
    insts = I.ensemble_instances(n)
    probs = [dgw.Problem(dim=d["dim"], nx=d["nx"], ny=d["ny"], p=d["p"], flux=d["flux"], a=d["a"],
                         stab="weno", bc=("periodic",) * 4) for d in insts]
    b = dgw.Batch(probs, prec="fp32")
    U = torch.zeros(b.total, dtype=torch.float32, device=dev)
    nq, cap, i = 4, 1 << 25, 0
    while i < n:      # project in chunks of instances (initial data sampled on the GPU)
        parts, tot, j = [], 0, i
        while j < n:
            d = insts[j]
            cnt = d["nx"] * d["ny"] * nq ** d["dim"]
            if parts and tot + cnt > cap:
                break
            X, Y = I.sample_points_xp(d["dim"], d["nx"], d["ny"], (0.0, 1.0, 0.0, 1.0), nq, torch,
                                      dtype=torch.float64, device=dev)
            parts.append(I.u0_fourier_steps(d["init"], X, Y if d["dim"] == 2 else None, xp=torch).reshape(-1))
            tot += cnt
            j += 1
        b.project(torch.cat(parts).contiguous(), U, first=i, count=j - i, nq=nq)
        del parts
        i = j
    b.set_dt([d["dt"] for d in insts])
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        chunk = b.autotune(U, steps=2) if autotune else None
        b.rk_step(U, warmup)
    stream.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        ev0.record(stream)
        b.rk_step(U, steps)
        ev1.record(stream)
    ev1.synchronize()
    b.sync_status(stream)
    t = ev0.elapsed_time(ev1) / 1e3
    N = sum(pr.K * pr.E for pr in probs)
    out = {"workload": f"ensemble_{n}", "value": 3 * N * steps / t, "unit": "DOF-updates/s", "dofs": N,
           "instances": n, "instances_1d": sum(d["dim"] == 1 for d in insts), "steps": steps,
           "ms_per_step": 1e3 * t / steps, "work_item_tiles": chunk, "dtype": "f32",
           "schedule": {f"{d}d_p{p}": b.schedule(d, p) for d in (1, 2) for p in (1, 2, 3)},
           "finite": bool(torch.isfinite(U).all().item())}
    b.close()
    return out


def run_tc_volume(local, ntiles=8192):
    """The Q3 KPP volume term of 1,048,576 cells (the headline workload's count) on the
    CUDA cores as the stage kernel computes it, and on the tensor cores (tcgen05, three
    TF32 passes): the kernels' times from CUDA events, best of 5 after a warm-up."""
    import torch

    from paper_2309_12019_gb300 import dgw
    dev = torch.device("cuda", local)
    U = torch.rand((16, ntiles * 128), dtype=torch.float32, device=dev) * 3.0 + 5.0
    out = torch.empty_like(U)
    t = {}
    for variant in (0, 1):
        dgw.selftest_tc_volume(U, out, variant)
        t[variant] = min(dgw.selftest_tc_volume(U, out, variant) for _ in range(5))
    return {"cells": ntiles * 128, "cuda_cores_us": 1e3 * t[0], "tensor_cores_us": 1e3 * t[1],
            "what": "volume term of the Q3 KPP stage: [cells x 16] x [16 x 25], sin/cos, [cells x 50] x [50 x 16]"}


def run_adjoint(local, n=512, steps=200, every=20):
    """The adjoint workload: 2D Burgers (u^2/2, u^2/2), periodic unit square, n^2 Q2,
    FP32, misfit after `steps` SSP-RK3 steps against a target grown from another seeded
    field; gradient by the checkpointed discrete adjoint (recompute every `every`)."""
    import torch

    from paper_2309_12019_gb300 import adjoint, dgw
    dev = torch.device("cuda", local)
    # the unthresholded sensor (b = 0): the threshold of Eq. (gensensor) makes the scheme
    # jump where a ratio crosses b, and the gradient is that of one smooth piece
    s = dict(dim=2, nx=n, ny=n, p=2, box=(0.0, 1.0, 0.0, 1.0), bc=("periodic",) * 4, flux="burgers",
             a=(1.0, 1.0), stab="weno", b=0.0)
    pc, pt = I.adjoint_field(I.SEED + 5001), I.adjoint_field(I.SEED + 5002)
    dt = I.cfl_dt(0.1, [float(np.sum(pc["amp"])) + 1.0] * 2, [1.0 / n] * 2)
    c = dgw.Context(dgw.Problem(**s, prec="fp32"))
    X, Y = I.sample_points(2, n, n, s["box"], 8)
    U0 = torch.empty((9, n * n), dtype=torch.float32, device=dev)
    Ut = torch.empty_like(U0)
    c.project(torch.tensor(I.u0_fourier_steps(pc, X, Y).reshape(-1), device=dev), U0)
    c.project(torch.tensor(I.u0_fourier_steps(pt, X, Y).reshape(-1), device=dev), Ut)
    c.rk_step(Ut, dt, steps)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    # untimed warm-up: three rollouts of one checkpoint segment with their backward passes
    # on this context (first launches of the adjoint kernels, the context's adjoint
    # buffers, the allocator's room for a segment's recomputed states)
    for _ in range(3):
        Uw = U0.clone().requires_grad_(True)
        adjoint.misfit(c, adjoint.rollout(c, Uw, dt, min(steps, every), every=every), Ut).backward()
    del Uw
    U0g = U0.clone().requires_grad_(True)
    torch.cuda.synchronize()
    ev[0].record()
    J = adjoint.misfit(c, adjoint.rollout(c, U0g, dt, steps, every=every), Ut)
    ev[1].record()
    J.backward()
    ev[2].record()
    ev[2].synchronize()
    c.sync_status()
    fwd, bwd = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
    out = {"workload": f"adjoint_burgers_{n}x{n}_q2", "dtype": "f32", "steps": steps, "checkpoint_every": every,
           "dofs": 9 * n * n, "forward_ms_per_step": fwd / steps, "backward_ms_per_step": bwd / steps,
           "backward_over_forward": bwd / fwd, "misfit": float(J.detach()),
           "grad_finite": bool(torch.isfinite(U0g.grad).all().item())}
    c.close()
    return out


def run_small(name, prec, steps, warmup, local):
    """Throughput of one of the smaller configurations through dgw_rk_step.  Euler
    workloads add the stage kernel's HBM roofline: 8/3 state passes per stage launch
    (read Uk and write Uout in every stage, read Un in two of three)."""
    w = WORKLOADS[name]
    r = run_gpu(w, prec, steps, warmup, 1, local, measure_e2e=False)
    stages = STAGES_PER_STEP[w.get("rk_order", 3)]
    out = {"workload": name, "dtype": "f64" if prec == "fp64" else "f32", "value": stages * r["N"] * steps / r["t"],
           "unit": "DOF-updates/s", "steps": steps, "ms_per_step": 1e3 * r["t"] / steps,
           "cell_mean_range_after": r["mean_range"]}
    if w["flux"] == "euler":
        hbm, src = peaks()
        per_launch = r["t"] / (stages * steps)
        alg = 8.0 / 3.0 * r["N"] * (8 if prec == "fp64" else 4)
        out["roofline"] = {"bound": "hbm", "kernel": "euler_kernel", "achieved": alg / per_launch / 1e9,
                           "peak": hbm, "unit": "GB/s", "frac": alg / per_launch / 1e9 / hbm,
                           "peak_source": src, "bytes_per_launch": alg, "us_per_launch": 1e6 * per_launch}
        out["mass_after"] = r["mass"]
    if "t_end" in w:
        out["time_to_t_end_ms"] = 1e3 * r["t"] / steps * math.ceil(w["t_end"] / dt_of(w) - 1e-9)
    return out


def run_reference(w, steps, warmup, budget_s=12.0, threads=None):
    """The FP64 CPU oracle on this host's cores (or `threads` of them), each step a
    bounded sample: the residual (per-stage work) of a contiguous block of elements."""
    from oracle import oracle as O
    O.build()
    cores = threads or os.cpu_count() or 1
    O.set_threads(os.cpu_count() or 1)        # the projection is set-up, not the sample
    P = O.Problem(**spec_of(w))
    U = O.project(P, initial_samples(w))
    O.set_threads(cores)
    E, K = P.E, P.K
    block = 4096 if cores > 1 else 512
    # calibrate the sample so that all steps fit in the budget
    t0 = time.perf_counter()
    O.residual_at(P, U, np.arange(block))
    per_elem = (time.perf_counter() - t0) / block
    n_el = int(max(block, min(E, budget_s / max(steps + warmup, 1) / per_elem)))
    idx = np.arange(n_el) + (E - n_el) // 2
    for _ in range(warmup):
        O.residual_at(P, U, idx)
    t0 = time.perf_counter()
    for _ in range(steps):
        O.residual_at(P, U, idx)
    t = time.perf_counter() - t0
    value = n_el * K * steps / t
    return value, cores, n_el


def run_reference_configs(budget_s=4.0):
    """The FP64 oracle's per-stage residual throughput on the other configurations, each a
    bounded sample of about budget_s seconds on all host cores: the 1D advection profile
    (128 cells, P2) and the solid-body rotation (256^2, Q2) on their whole meshes, the
    ensemble on its smallest instances (8 of each dimension), and the 512^2 Q2 Burgers
    adjoint workload's forward residual on a contiguous block of cells."""
    from oracle import oracle as O
    O.build()
    cores = os.cpu_count() or 1
    O.set_threads(cores)
    out = {}

    def timed(fn, dofs):
        fn()                                     # warm-up
        n, t0 = 0, time.perf_counter()
        while True:
            fn()
            n += 1
            t = time.perf_counter() - t0
            if t >= budget_s:
                return dofs * n / t, n

    for key, name in (("advect1d_128_p2", "advect1d_128_p2"), ("rotation_256x256_q2", "rotation_256x256_q2")):
        w = WORKLOADS[name]
        P = O.Problem(**spec_of(w))
        U = O.project(P, initial_samples(w))
        v, n = timed(lambda: O.residual(P, U), P.K * P.E)
        out[key] = {"value": v, "unit": "DOF-updates/s", "cores": cores, "kind": "oracle",
                    "sample": f"oracle residual of the whole {w['nx']}x{w['ny']} mesh, {n} repeats"}
    insts = I.ensemble_instances(512)
    size = lambda i: insts[i]["nx"] * insts[i]["ny"]
    pick = (sorted([i for i in range(512) if insts[i]["dim"] == 1], key=size)[:8] +
            sorted([i for i in range(512) if insts[i]["dim"] == 2], key=size)[:8])
    probs, states = [], []
    for i in pick:
        d = insts[i]
        P = O.Problem(dim=d["dim"], nx=d["nx"], ny=d["ny"], p=d["p"], box=(0.0, 1.0, 0.0, 1.0),
                      bc=("periodic",) * 4, flux=d["flux"], a=d["a"], stab="weno")
        X, Y = I.sample_points(d["dim"], d["nx"], d["ny"], P.box, 8)
        probs.append(P)
        states.append(O.project(P, I.u0_fourier_steps(d["init"], X, Y)))
    v, n = timed(lambda: [O.residual(P, U) for P, U in zip(probs, states)], sum(P.K * P.E for P in probs))
    out["ensemble_512"] = {"value": v, "unit": "DOF-updates/s", "cores": cores, "kind": "oracle",
                           "sample": f"oracle residuals of the 8 smallest 1D and 8 smallest 2D instances, {n} repeats"}
    n_ = 512
    P = O.Problem(dim=2, nx=n_, ny=n_, p=2, box=(0.0, 1.0, 0.0, 1.0), bc=("periodic",) * 4, flux="burgers",
                  a=(1.0, 1.0), stab="weno", b=0.0)
    X, Y = I.sample_points(2, n_, n_, P.box, 8)
    U = O.project(P, I.u0_fourier_steps(I.adjoint_field(I.SEED + 5001), X, Y))
    idx = np.arange(16384) + (P.E - 16384) // 2
    v, n = timed(lambda: O.residual_at(P, U, idx), P.K * idx.size)
    out["adjoint_burgers_512x512_q2"] = {"value": v, "unit": "DOF-updates/s", "cores": cores, "kind": "oracle",
                                         "sample": f"oracle forward residual of 16384 contiguous cells, {n} repeats"}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="kpp_1024x1024_q3", choices=sorted(WORKLOADS))
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison run")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end run")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the ensemble and the smaller configurations")
    ap.add_argument("--only", choices=["ensemble", "adjoint"],
                    help="run one secondary leg alone (--steps steps) and print its line")
    ap.add_argument("--no-autotune", action="store_true",
                    help="ensemble: keep the default schedule (for profiling a fixed launch sequence)")
    args = ap.parse_args()
    w = WORKLOADS[args.workload]
    world, rank, local = dist_setup(args)
    if args.warmup < 3:
        args.warmup = 3
    metric = "DOF-updates/sec per SSP-RK3 stage"
    config = {"workload": args.workload, "mesh": f"{w['nx']}x{w['ny']}", "p": w["p"], "flux": w["flux"],
              "stab": w["stab"], "dofs": dofs_of(w),
              "l2": "inputs larger than L2 (three 67 MB FP32 state arrays per stage)",
              "parallelism": f"replicas{world}" if world > 1 else "single"}

    if args.impl == "reference":
        if rank != 0:
            return
        v, cores, n_el = run_reference(w, args.steps, args.warmup)
        sample = f"oracle residual (per-stage work) of {n_el} contiguous cells of the {w['nx']}x{w['ny']} mesh per step"
        line = {"impl": "reference", "metric": metric, "value": v, "unit": "DOF-updates/s", "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config,
                "cpu_baseline": {"value": v, "unit": "DOF-updates/s", "cores": cores, "kind": "oracle",
                                 "sample": sample},
                "e2e": {"value": v, "unit": "DOF-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    if args.only:
        if rank == 0:
            if args.only == "ensemble":
                leg = run_ensemble(args.steps, args.warmup, local, autotune=not args.no_autotune)
            else:
                leg = run_adjoint(local, steps=args.steps, every=min(20, args.steps))
            print(json.dumps(dict(leg, leg=args.only)))
        return

    r32 = run_gpu(w, "fp32", args.steps, args.warmup, world, local, measure_e2e=not args.no_e2e)
    t = max_over_ranks(r32["t"], world)
    t_e2e = max_over_ranks(r32["t_e2e"], world) if "t_e2e" in r32 else float("nan")
    N = r32["N"]
    stages = r32["stages"]
    value = world * stages * N * args.steps / t
    e2e_value = world * stages * N * args.steps / t_e2e
    r64 = None
    if not args.no_fp64:
        st64 = max(3, args.steps // 10)
        r64 = run_gpu(w, "fp64", st64, args.warmup, world, local, measure_e2e=False)
        r64["steps"] = st64
    extras = {}
    if not args.no_extras:
        extras["volume_term_tensor_cores"] = run_tc_volume(local)
        extras["ensemble"] = run_ensemble(100, 3, local)
        extras["adjoint"] = run_adjoint(local)
        extras["others"] = [run_small("kpp_1024x1024_q3_zhao", "fp32", 100, 5, local),
                            run_small("kpp_1024x1024_q3_rk4", "fp32", 40, 3, local),
                            run_small("rotation_256x256_q2", "fp64", 100, 5, local),
                            run_small("rotation_256x256_q2", "fp32", 100, 5, local),
                            run_small("advect1d_128_p2", "fp64", 1280, 10, local),
                            run_small("sod_train_4194304_q2", "fp32", 200, 5, local),
                            run_small("sod_train_4194304_q2", "fp64", 100, 5, local),
                            run_small("sod_128_q2", "fp64", 739, 10, local),
                            run_small("shu_osher_512_q3", "fp64", 9216, 10, local),
                            run_small("kelvin_helmholtz_512x512_q2", "fp32", 200, 5, local),
                            run_small("kelvin_helmholtz_512x512_q2", "fp64", 20, 3, local),
                            run_small("kelvin_helmholtz_2048x2048_q2", "fp32", 50, 3, local),
                            run_small("triple_point_896x384_q2", "fp32", 200, 5, local)]
    if rank != 0:
        return
    hbm, src = peaks()
    per_launch_s = t / (stages * args.steps)   # stage kernels (order 4: plus one light mixing kernel per step)
    alg_bytes = 8.0 / 3.0 * N * 4          # per stage: 8 state-array passes per step / 3 stages
    achieved = alg_bytes / per_launch_s / 1e9
    cells = w["nx"] * w["ny"]
    fpc, sincos = stage_flops_per_cell(w["dim"], w["p"], w["flux"], w["stab"])
    tflops = fpc * cells / per_launch_s / 1e12
    line = {"metric": metric, "value": value, "unit": "DOF-updates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config,
            "roofline": {"bound": "alu", "achieved": tflops, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": tflops / FP32_PEAK_TFLOPS,
                         "traffic": STAGE_TRAFFIC_BYTES if args.workload == "kpp_1024x1024_q3" else None,
                         "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz",
                         "flops_per_cell": fpc, "sincos_per_cell": sincos,
                         "kernel": "stage_kernel_p, persistent (3 launches per step)",
                         "hbm": {"achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                                 "peak_source": src, "bytes_per_launch": alg_bytes}},
            "e2e": {"value": e2e_value, "unit": "DOF-updates/s", "h2d_bytes_per_step": r32.get("bytes"),
                    "d2h_bytes_per_step": r32.get("bytes")} if "t_e2e" in r32 else None,
            "gpu_launches": r32["launches"], "clocks": r32["clocks"], "mass_after": r32["mass"],
            "cell_mean_range_after": r32["mean_range"]}
    if w["flux"] == "euler":      # the Euler kernel is bound by HBM, not by FP32 issue
        line["roofline"] = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                            "frac": achieved / hbm, "traffic": None, "peak_source": src,
                            "bytes_per_launch": alg_bytes, "kernel": "euler_kernel (3 launches per step)"}
        line["config"]["l2"] = f"inputs larger than L2 (three {N * 4 / 1e6:.0f} MB FP32 state arrays per stage)"
    if r64 is not None:
        line["fp64"] = {"value": stages * N * r64["steps"] / r64["t"], "unit": "DOF-updates/s",
                        "ms_per_step": 1e3 * r64["t"] / r64["steps"], "steps": r64["steps"]}
    line.update(extras)
    if not args.no_cpu and world == 1:
        v, cores, n_el = run_reference(w, 3, 1, budget_s=12.0)
        v1, _, n1 = run_reference(w, 2, 1, budget_s=4.0, threads=1)
        line["cpu_baseline"] = {"value": v, "unit": "DOF-updates/s", "cores": cores, "kind": "oracle",
                                "sample": f"oracle residual (per-stage work) of {n_el} contiguous cells, 3 repeats",
                                "value_1_thread": v1,
                                "sample_1_thread": f"{n1} contiguous cells, 2 repeats, one thread"}
        if not args.no_extras:
            line["cpu_baseline"]["other_configs"] = run_reference_configs()
    print(json.dumps(line))


if __name__ == "__main__":
    main()

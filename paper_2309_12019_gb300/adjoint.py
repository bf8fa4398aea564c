"""Gradients of a final-time misfit with respect to the initial DOFs, through the
library's discrete adjoint (dgw_adjoint_step), as torch.autograd.Functions.

rollout(ctx, U0, dt, nsteps, every) advances U0 by nsteps SSP-RK3 steps and keeps a
checkpoint every `every` steps; its backward pass recomputes each segment's states from
its checkpoint (dgw_rk_step) and runs dgw_adjoint_step through the segment in reverse.
misfit(ctx, U, U_target) is J = 1/2 int (U_h - U_target)^2 with dJ/dU from dgw_misfit.
All arithmetic runs in the library's kernels; this module only orders the calls.
"""
from __future__ import annotations

import torch


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx_, U0, dctx, dt, nsteps, every):
        U = U0.detach().clone().contiguous()
        checkpoints = [U.clone()]
        done = 0
        while done < nsteps:
            n = min(every, nsteps - done)
            dctx.rk_step(U, dt, n)
            done += n
            if done < nsteps:
                checkpoints.append(U.clone())
        ctx_.dctx, ctx_.dt, ctx_.nsteps, ctx_.every = dctx, dt, nsteps, every
        ctx_.checkpoints = checkpoints
        return U

    @staticmethod
    def backward(ctx_, gout):
        dctx, dt, nsteps, every = ctx_.dctx, ctx_.dt, ctx_.nsteps, ctx_.every
        lam = gout.detach().clone().contiguous()
        for seg in reversed(range(len(ctx_.checkpoints))):
            start = seg * every
            n = min(every, nsteps - start)
            states = [ctx_.checkpoints[seg].clone()]
            for _ in range(n - 1):
                nxt = states[-1].clone()
                dctx.rk_step(nxt, dt, 1)
                states.append(nxt)
            for Un in reversed(states):
                dctx.adjoint_step(Un, lam, lam, dt)
        ctx_.checkpoints = None
        return lam, None, None, None, None


class _Misfit(torch.autograd.Function):
    @staticmethod
    def forward(ctx_, U, U_target, dctx):
        grad = torch.empty_like(U)
        J = dctx.misfit(U.contiguous(), U_target.contiguous(), grad)
        ctx_.save_for_backward(grad)
        return torch.tensor(J, dtype=torch.float64, device=U.device)

    @staticmethod
    def backward(ctx_, gJ):
        (grad,) = ctx_.saved_tensors
        return grad * gJ.to(grad.dtype), None, None


def rollout(dctx, U0, dt: float, nsteps: int, every: int = 20):
    return _Rollout.apply(U0, dctx, float(dt), int(nsteps), int(every))


def misfit(dctx, U, U_target):
    return _Misfit.apply(U, U_target, dctx)

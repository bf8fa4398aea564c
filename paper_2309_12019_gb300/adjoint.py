"""Gradients of a final-time misfit with respect to the initial DOFs, through the
library's discrete adjoint (dgw_adjoint_step), as torch.autograd.Functions.

rollout(ctx, U0, dt, nsteps, every) advances U0 by nsteps SSP-RK3 steps and keeps a
checkpoint every `every` steps; its backward pass recomputes each segment from its
checkpoint, keeping every step's state and its two stage states (dgw_rk_step_stages),
and runs dgw_adjoint_step_stages through the segment in reverse, so that no stage is
evaluated twice in the backward pass.
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
            states = [ctx_.checkpoints[seg]]
            stages = []
            for i in range(n):
                U1, U2 = torch.empty_like(lam), torch.empty_like(lam)
                nxt = torch.empty_like(lam) if i < n - 1 else None   # the last step needs no U^{n+1}
                dctx.rk_step_stages(states[-1], dt, U1, U2, nxt)
                stages.append((U1, U2))
                if nxt is not None:
                    states.append(nxt)
            for Un, (U1, U2) in zip(reversed(states), reversed(stages)):
                dctx.adjoint_step_stages(Un, U1, U2, lam, lam, dt)
            del states, stages
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

"""Differentiable SSP-RK3 rollouts on top of the library's adjoint (dg_rk_step_vjp).

`rollout(solver, U0, gamma, dt, n_steps, checkpoint_every)` advances U0 by n_steps SSP-RK3
steps and is differentiable with respect to U0 and gamma.  The forward pass keeps only every
`checkpoint_every`-th state; the backward pass recomputes each segment forward from its
checkpoint and then walks it in reverse with the library's step adjoint, which itself
recomputes the stage states.  All arithmetic runs in the CUDA library; this module only
orders the calls and holds the checkpoints.
"""
from __future__ import annotations

import torch


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U0, gamma, solver, dt, n_steps, every):
        if abs(float(gamma) - solver.gamma) > 1e-15 * abs(solver.gamma):
            raise ValueError("gamma must equal the solver's gamma (the context is built for it)")
        checkpoints = []
        solver.set_state(U0.detach().contiguous())
        done = 0
        while done < n_steps:
            checkpoints.append(solver.get_state())  # a fresh tensor
            k = min(every, n_steps - done)
            solver.rk_step(dt, k)
            done += k
        solver.check()
        out = solver.get_state().clone()
        ctx.solver, ctx.dt, ctx.n_steps, ctx.every = solver, dt, n_steps, every
        ctx.checkpoints = checkpoints
        return out

    @staticmethod
    def backward(ctx, gout):
        S, dt, every = ctx.solver, ctx.dt, ctx.every
        lam = gout.detach().contiguous().clone()
        S.adjoint_gammabar()  # start from an empty device accumulator
        n_seg = len(ctx.checkpoints)
        for s in reversed(range(n_seg)):
            k = min(every, ctx.n_steps - s * every)
            S.set_state(ctx.checkpoints[s])
            states = []
            for _ in range(k):  # recompute the segment
                states.append(S.get_state())
                S.rk_step(dt, 1)
            for j in reversed(range(k)):
                S.rk_step_vjp(states[j], dt, lam, defer=True)  # gamma stays on the device
        gbar = S.adjoint_gammabar()
        S.check()
        gg = torch.tensor(gbar, dtype=torch.float64)
        return lam, gg, None, None, None, None


def rollout(solver, U0: torch.Tensor, gamma: torch.Tensor, dt: float, n_steps: int,
            checkpoint_every: int = 20) -> torch.Tensor:
    """n_steps SSP-RK3 steps of U0 (differentiable in U0 and gamma)."""
    return _Rollout.apply(U0, gamma, solver, dt, n_steps, checkpoint_every)

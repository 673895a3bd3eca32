"""Differentiable SSP steps on top of the library's adjoint (dg_rk_step_vjp).

`step(solver, U, gamma, dt)` (the autograd function `DGStep`) is one step of the solver's SSP
scheme, differentiable with respect to U and gamma: the forward pass is dg_rk_step from U,
the backward pass dg_rk_step_vjp, which recomputes the stage states from the saved U.  It
composes into loops the caller writes (every step's input is kept).

`rollout(solver, U0, gamma, dt, n_steps, checkpoint_every)` advances U0 by n_steps steps
with checkpoints: the forward pass keeps only every `checkpoint_every`-th state; the backward
pass recomputes each segment forward from its checkpoint and then walks it in reverse with
the step adjoint.  All arithmetic runs in the CUDA library; this module only orders the
calls and holds the states.
"""
from __future__ import annotations

import torch


def _check_gamma(solver, gamma):
    if abs(float(gamma) - solver.gamma) > 1e-15 * abs(solver.gamma):
        raise ValueError("gamma must equal the solver's gamma (the context is built for it)")


class DGStep(torch.autograd.Function):
    """One SSP step of the solver's scheme: U -> U after dt, differentiable in U and gamma."""

    @staticmethod
    def forward(ctx, U, gamma, solver, dt):
        _check_gamma(solver, gamma)
        U = U.detach().contiguous()
        solver.set_state(U)
        solver.rk_step(dt, 1)
        solver.check()
        out = solver.get_state()  # a fresh tensor
        ctx.save_for_backward(U)
        ctx.solver, ctx.dt = solver, dt
        return out

    @staticmethod
    def backward(ctx, gout):
        (U,) = ctx.saved_tensors
        S = ctx.solver
        lam = gout.detach().contiguous().clone()
        S.adjoint_gammabar()  # start from an empty device accumulator
        g = S.rk_step_vjp(U, ctx.dt, lam)
        S.check()
        return lam, torch.tensor(g, dtype=torch.float64), None, None


def step(solver, U: torch.Tensor, gamma: torch.Tensor, dt: float) -> torch.Tensor:
    """One SSP step of U (differentiable in U and gamma)."""
    return DGStep.apply(U, gamma, solver, dt)


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U0, gamma, solver, dt, n_steps, every):
        _check_gamma(solver, gamma)
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
    """n_steps SSP steps of U0 with checkpoints (differentiable in U0 and gamma)."""
    return _Rollout.apply(U0, gamma, solver, dt, n_steps, checkpoint_every)

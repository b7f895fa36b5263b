"""Differentiable fixed-step SSP-RK3 rollouts of the 1D systems.

`rollout(U0, p, dt, steps)` advances U0 by `steps` RK3 steps of the fixed size dt with the
library's forward kernels and is differentiable with respect to U0: its backward pass runs
the hand-written adjoint kernels (wenozn_rk3_step_vjp) step by step in reverse.  Forward
states are kept every `checkpoint_every` steps; the backward pass recomputes the states of
one segment from its checkpoint (with its stage inputs) and walks it backwards, so memory
holds steps/checkpoint_every + 3 checkpoint_every states; checkpoint_every = 1 keeps every
step's three stage inputs and LF speeds and recomputes nothing.  The time step is an input, not a function of U0 (the adjoint's
convention); choose it from the initial state, e.g. with `cfl_step`.
"""
from __future__ import annotations

import math

import torch

from . import wenozn as W


class WenoZNRollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U0, p, dt, steps, checkpoint_every, ws):
        U = U0.detach().clone().contiguous()
        every = max(1, int(checkpoint_every))
        ctx.p, ctx.dt, ctx.steps, ctx.every, ctx.ws = p, dt, steps, every, ws
        if every == 1:
            # keep every step's stage inputs and LF speeds: the reverse pass recomputes nothing
            ctx.stages = _run_keep_stages(p, ws, U, dt, steps)
        else:
            checkpoints = [U.clone()]
            for k in range(steps):
                W.wenozn_rk3_step(p, U, ws, dt=dt)
                if (k + 1) % every == 0 and k + 1 < steps:
                    checkpoints.append(U.clone())
            ctx.checkpoints = checkpoints
        return U

    @staticmethod
    def backward(ctx, gU):
        lam = gU.detach().clone().contiguous()
        p, dt, ws, every = ctx.p, ctx.dt, ctx.ws, ctx.every
        if every == 1:
            S0, S1, S2, A = ctx.stages
            for k in reversed(range(ctx.steps)):
                W.wenozn_rk3_step_vjp_stages(p, S0[k], S1[k], S2[k], A[k], dt, lam, ws)
            return lam, None, None, None, None, None
        nseg = math.ceil(ctx.steps / every)
        for seg in reversed(range(nseg)):
            k0, k1 = seg * every, min(ctx.steps, (seg + 1) * every)
            U = ctx.checkpoints[seg].clone()
            S0, S1, S2, A = _run_keep_stages(p, ws, U, dt, k1 - k0)
            for k in reversed(range(k1 - k0)):
                W.wenozn_rk3_step_vjp_stages(p, S0[k], S1[k], S2[k], A[k], dt, lam, ws)
        return lam, None, None, None, None, None


def _run_keep_stages(p, ws, U, dt, steps):
    """Advances U in place by `steps` steps, returning every step's stage inputs
    (U^n, U^(1), U^(2)) and LF speeds, written there by the out-of-place step."""
    X = torch.empty((steps + 1,) + tuple(U.shape), dtype=U.dtype, device=U.device)
    S1, S2 = torch.empty_like(X[:steps]), torch.empty_like(X[:steps])
    A = torch.empty((steps, 3), dtype=U.dtype, device=U.device)
    X[0].copy_(U)
    for k in range(steps):
        W.wenozn_rk3_step_keep(p, X[k], X[k + 1], dt, S1[k], S2[k], A[k], ws)
    U.copy_(X[steps])
    return X[:steps], S1, S2, A


def rollout(U0: torch.Tensor, p: W.wenozn_problem, dt: float, steps: int, checkpoint_every: int = 1,
            ws: torch.Tensor | None = None) -> torch.Tensor:
    if ws is None:
        ws = W.vjp_workspace(p, U0.device)
    return WenoZNRollout.apply(U0, p, float(dt), int(steps), int(checkpoint_every), ws)


def cfl_step(p: W.wenozn_problem, U: torch.Tensor) -> float:
    """cfl dx / max(|u| + c) of U (1D), evaluated on the device by the library."""
    a = torch.zeros(2, dtype=torch.float64, device=U.device)
    W.wenozn_max_wavespeed(p, U, a)
    return p.cfl * p.dx / float(a[0].item())

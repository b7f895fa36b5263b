"""Differentiable fixed-step SSP-RK3 rollouts of the 1D systems.

`rollout(U0, p, dt, steps)` advances U0 by `steps` RK3 steps of the fixed size dt with the
library's forward kernels and is differentiable with respect to U0: its backward pass runs
the hand-written adjoint kernels (wenozn_rk3_step_vjp) step by step in reverse.  Forward
states are kept every `checkpoint_every` steps; the backward pass recomputes the states of
one segment from its checkpoint and walks it backwards, so memory holds
steps/checkpoint_every + checkpoint_every states (checkpoint_every = 1 keeps every state and
recomputes nothing).  The time step is an input, not a function of U0 (the adjoint's
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
        checkpoints = [U.clone()]
        for k in range(steps):
            W.wenozn_rk3_step(p, U, ws, dt=dt)
            if (k + 1) % every == 0 and k + 1 < steps:
                checkpoints.append(U.clone())
        ctx.p, ctx.dt, ctx.steps, ctx.every, ctx.ws = p, dt, steps, every, ws
        ctx.checkpoints = checkpoints
        return U

    @staticmethod
    def backward(ctx, gU):
        lam = gU.detach().clone().contiguous()
        p, dt, ws, every = ctx.p, ctx.dt, ctx.ws, ctx.every
        nseg = math.ceil(ctx.steps / every)
        for seg in reversed(range(nseg)):
            k0, k1 = seg * every, min(ctx.steps, (seg + 1) * every)
            states = [ctx.checkpoints[seg]]
            U = ctx.checkpoints[seg].clone()
            for _ in range(k0, k1 - 1):
                W.wenozn_rk3_step(p, U, ws, dt=dt)
                states.append(U.clone())
            for k in reversed(range(k0, k1)):
                W.wenozn_rk3_step_vjp(p, states[k - k0], dt, lam, ws)
        return lam, None, None, None, None, None


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

"""Differentiable fixed-step SSP-RK3 rollouts of the 1D systems.

`rollout(U0, p, dt, steps)` advances U0 by `steps` RK3 steps of the fixed size dt with the
library's forward kernels and is differentiable with respect to U0: its backward pass runs
the hand-written adjoint kernels (wenozn_rk3_vjp_run) over the steps in reverse.  Forward
states are kept every `checkpoint_every` steps; the backward pass recomputes the states of
one segment from its checkpoint (with its stage inputs, one library call) and walks it
backwards (one call), so memory holds steps/checkpoint_every + 3 checkpoint_every states;
checkpoint_every = 1 keeps every step's three stage inputs and LF speeds and recomputes
nothing.  The time step is an input, not a function of U0 (the adjoint's
convention); choose it from the initial state, e.g. with `cfl_step`.
"""
from __future__ import annotations

import torch

from . import wenozn as W


class WenoZNRollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U0, p, dt, steps, checkpoint_every, ws):
        every = max(1, int(checkpoint_every))
        ctx.p, ctx.dt, ctx.steps, ctx.every, ctx.ws = p, dt, steps, every, ws
        if every == 1:
            # keep every step's stage inputs and LF speeds: the reverse pass recomputes nothing
            ctx.keep = _segment_keep(p, ws, U0.detach().contiguous(), dt, steps)
            return ctx.keep[0][steps].clone()
        U = U0.detach().clone().contiguous()
        checkpoints = []
        for k0 in range(0, steps, every):
            checkpoints.append(U.clone())
            W.wenozn_rk3_run(p, U, min(every, steps - k0), ws, dt)
        ctx.checkpoints = checkpoints
        return U

    @staticmethod
    def backward(ctx, gU):
        lam = gU.detach().clone().contiguous()
        p, dt, ws, every, steps = ctx.p, ctx.dt, ctx.ws, ctx.every, ctx.steps
        if every == 1:
            X, S1, S2, A = ctx.keep
            W.wenozn_rk3_vjp_run(p, X, S1, S2, A, steps, dt, lam, ws)
            return lam, None, None, None, None, None
        for seg in reversed(range(len(ctx.checkpoints))):
            m = min(every, steps - seg * every)
            X, S1, S2, A = _segment_keep(p, ws, ctx.checkpoints[seg], dt, m)
            W.wenozn_rk3_vjp_run(p, X, S1, S2, A, m, dt, lam, ws)
        return lam, None, None, None, None, None


def _segment_keep(p, ws, U, dt, steps):
    """`steps` steps from U (unchanged) in one call, keeping every state X[0..steps], the
    stage inputs S1, S2 of every step and the LF speeds of every stage input."""
    X = torch.empty((steps + 1,) + tuple(U.shape), dtype=U.dtype, device=U.device)
    S1 = torch.empty((steps,) + tuple(U.shape), dtype=U.dtype, device=U.device)
    S2 = torch.empty_like(S1)
    A = torch.empty(3 * steps + 1, dtype=U.dtype, device=U.device)
    X[0].copy_(U)
    W.wenozn_rk3_run_keep(p, X, S1, S2, A, steps, dt, ws)
    return X, S1, S2, A


def rollout(U0: torch.Tensor, p: W.wenozn_problem, dt: float, steps: int, checkpoint_every: int = 1,
            ws: torch.Tensor | None = None) -> torch.Tensor:
    if ws is None:
        ws = W.vjp_workspace(p, U0.device)
    return WenoZNRollout.apply(U0, p, float(dt), int(steps), int(checkpoint_every), ws)


def cfl_step(p: W.wenozn_problem, U: torch.Tensor, ws: torch.Tensor | None = None) -> float:
    """The CFL step of U (cfl dx / max(|u| + c) in 1D), computed by the library on the device
    (wenozn_cfl_dt); ws is any workspace of p (a fresh one if None)."""
    return W.wenozn_cfl_dt(p, U, W.workspace(p, U.device) if ws is None else ws)

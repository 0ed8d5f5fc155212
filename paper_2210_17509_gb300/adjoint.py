"""Differentiable evolution: torch.autograd.Function wrappers around the
library's forward step and its hand-written reverse (grmhd_rk_step_adjoint).

``evolve(prim0, gamma, ...)`` maps interior initial primitives (shape
[8, nz, ny, nx]) and the Gamma-law index to the interior primitives after
``nsteps`` steps.  The forward pass keeps a checkpoint (U, P) every
``checkpoint_every`` steps; the backward pass recomputes each segment from its
checkpoint and runs the reverse steps in the library.  With
``keep_last_segment`` (the default) the forward pass records the stages of
the last segment as it runs them, so the backward pass recomputes only the
earlier segments: the memory of one segment's stages (per step U, P and one
primitive array per stage) instead of a recomputation the forward pass has
just done.  ``density_l2`` is the
functional  L = sum rho^2 sqrt(gamma) dV  with its adjoint.  The gradient with
respect to Gamma holds the initial primitives (pressure, not eps) fixed.
Only scheduling and layout (embedding the interior into ghosted arrays)
happen here; all arithmetic runs in the CUDA kernels.
"""
from __future__ import annotations

import dataclasses

import torch

from . import grmhd as G


def _embed(grid: G.Grid, interior: torch.Tensor) -> torch.Tensor:
    full = torch.zeros((8,) + grid.shape, dtype=torch.float64, device=interior.device)
    g = grid.ng
    full[:, g:-g, g:-g, g:-g] = interior
    return full


def _interior(grid: G.Grid, full: torch.Tensor) -> torch.Tensor:
    g = grid.ng
    return full[:, g:-g, g:-g, g:-g]


class _Evolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, prim0, gamma, grid, params, scheme, dt, nsteps, every, metric, keep_last):
        p = dataclasses.replace(params, gamma=float(gamma.item()))
        full = _embed(grid, prim0.detach())
        G.fill_ghosts(grid, p.bc, full)
        cons = G.prim2con(grid, p, full, metric)
        ws = G.workspace(grid, scheme, full.device)
        ckpt = {0: (cons.clone(), full.clone())}
        # the last segment starts at the last checkpoint; with keep_last its
        # steps are recorded now, for the backward pass
        last = ((nsteps - 1) // every) * every if nsteps > 0 else 0
        record = keep_last and any(ctx.needs_input_grad[:2])
        tail = []
        ns = G.stage_count(scheme)
        for s in range(nsteps):
            if record and s >= last:
                stages = torch.empty((ns, 8) + grid.shape, dtype=torch.float64, device=full.device)
                tail.append((cons.clone(), full.clone(), stages))
                G.rk_step_record(grid, p, scheme, dt, cons, full, stages, metric, None, ws)
            else:
                G.rk_step(grid, p, scheme, dt, cons, full, metric, None, ws)
            if (s + 1) % every == 0 and s + 1 < nsteps:
                ckpt[s + 1] = (cons.clone(), full.clone())
        ctx.tail = (last, tail) if record else None
        ctx.grid, ctx.params, ctx.scheme, ctx.dt, ctx.nsteps, ctx.every = grid, p, scheme, dt, nsteps, every
        ctx.metric = metric
        ctx.ckpt = ckpt
        return _interior(grid, full).clone()

    @staticmethod
    def backward(ctx, grad_out):
        grid, p, scheme, dt = ctx.grid, ctx.params, ctx.scheme, ctx.dt
        metric = ctx.metric
        dev = grad_out.device
        pbar = _embed(grid, grad_out.contiguous())
        ubar = torch.zeros_like(pbar)
        gbar = torch.zeros(1, dtype=torch.float64, device=dev)
        ws = G.workspace(grid, scheme, dev)
        wsa = G.adjoint_workspace(grid, scheme, dev)
        starts = sorted(ctx.ckpt)
        for k in reversed(range(len(starts))):
            s0 = starts[k]
            s1 = starts[k + 1] if k + 1 < len(starts) else ctx.nsteps
            if ctx.tail is not None and s0 == ctx.tail[0] and len(ctx.tail[1]) == s1 - s0:
                states = ctx.tail[1]  # recorded by the forward pass
            else:
                cons, prim = (t.clone() for t in ctx.ckpt[s0])
                states = []
                ns = G.stage_count(scheme)
                for s in range(s0, s1):
                    stages = torch.empty((ns, 8) + grid.shape, dtype=torch.float64, device=dev)
                    states.append((cons.clone(), prim.clone(), stages))
                    G.rk_step_record(grid, p, scheme, dt, cons, prim, stages, metric, None, ws)
            for cons_s, prim_s, stages in reversed(states):
                G.rk_step_adjoint(grid, p, scheme, dt, cons_s, prim_s, ubar, pbar, gbar, metric, None, wsa,
                                  stage_prims=stages)
        # initial data: P_full = ghost_fill(P0), U0 = prim2con(P_full)
        _, prim_init = ctx.ckpt[0]
        G.fill_ghosts_adjoint(grid, p.bc, pbar)
        G.prim2con_adjoint(grid, p, prim_init, ubar, pbar, gbar, metric)
        ctx.tail = None
        return (_interior(grid, pbar).clone(), gbar.reshape(()).clone(), None, None, None, None, None, None, None,
                None)


class _DensityL2(torch.autograd.Function):
    @staticmethod
    def forward(ctx, prim, grid, metric):
        full = _embed(grid, prim.detach())
        loss = torch.zeros(1, dtype=torch.float64, device=prim.device)
        G.density_l2(grid, full, metric, 0.0, loss, None)
        ctx.save_for_backward(full)
        ctx.grid, ctx.metric = grid, metric
        return loss.reshape(())

    @staticmethod
    def backward(ctx, gL):
        (full,) = ctx.saved_tensors
        pbar = torch.zeros_like(full)
        G.density_l2(ctx.grid, full, ctx.metric, float(gL.item()), None, pbar)
        return _interior(ctx.grid, pbar).clone(), None, None


def evolve(prim0, gamma, grid: G.Grid, params: G.Params, scheme: int, dt: float, nsteps: int,
           checkpoint_every: int = 5, metric=None, keep_last_segment: bool = True, deterministic: bool = False):
    """Interior primitives after nsteps steps (differentiable in prim0 and gamma).
    keep_last_segment=False recomputes the last segment in the backward pass
    too (no memory beyond the checkpoints).  deterministic=True sets
    GRMHD_DETERMINISTIC for the reverse calls: the gradients are then the
    same to the bit from run to run."""
    if deterministic:
        params = dataclasses.replace(params, flags=params.flags | G.DETERMINISTIC)
    return _Evolve.apply(prim0, gamma, grid, params, scheme, dt, nsteps, checkpoint_every, metric,
                         keep_last_segment)


def density_l2(prim, grid: G.Grid, metric=None):
    """sum over the interior of rho^2 sqrt(gamma) dV (differentiable)."""
    return _DensityL2.apply(prim, grid, metric)

"""Differentiable rollout of PolyPIC transfer steps.

``rollout(ctx, x0, mass, c0, n_steps, dt, ...)`` runs ``n_steps`` single-phase
steps (sort, P2G, grid update without projection, G2P with advection) through
the C library and returns the last step's grid velocity and mass.  Gradients of
a loss on that velocity flow back to the initial coefficients ``c0`` (every
mode, including the particle velocity c_0) and the initial positions ``x0``
through the library's hand-written adjoints: polypic_g2p_adjoint,
polypic_grid_update_adjoint and polypic_p2g_adjoint, chained step by step in
reverse.

Memory: particle states are checkpointed every ``checkpoint_every`` steps; the
backward pass recomputes each segment forward from its checkpoint (keeping that
segment's states, permutations and grids) and then walks it in reverse.

Particle order: every step writes its output state in its own slot order, so
the adjoint of step n arrives in step n's slot order, which is exactly the
storage order of step n+1's input; the library's adjoint entry points map it
back through step n's permutation.  The returned gradients are in the order of
the caller's initial arrays.
"""
from __future__ import annotations

from typing import List, Optional

import torch

from . import polypic as pp


def _copy_state(ctx: pp.Context, s: pp.ParticleState) -> pp.ParticleState:
    out = ctx.new_particles(s.count, device=s.x.device)
    out.x.copy_(s.x)
    out.mass.copy_(s.mass)
    out.coeff.copy_(s.coeff)
    return out


def _zeros_like_grid(g: pp.GridState) -> pp.GridState:
    z = lambda ts: [torch.zeros_like(t) for t in ts]
    return pp.GridState(mass=z(g.vel), mom=z(g.vel), vel=z(g.vel))


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(fctx, c0: torch.Tensor, x0: torch.Tensor, mass: torch.Tensor, ctx: pp.Context,
                n_steps: int, dt: float, gravity, k: int):
        if ctx.coeff_format != "f32":
            raise pp.PolyPICError(2, "rollout: only FP32 coefficients are differentiable")
        P = x0.shape[1]
        state = ctx.new_particles(P, device=x0.device)
        state.x.copy_(x0)
        state.mass.copy_(mass)
        state.coeff.copy_(c0)
        ws = ctx.workspace(P, device=x0.device)
        params = pp.UpdateSettings(dt=dt, gravity=tuple(gravity))
        grid = ctx.new_grid(device=x0.device)
        nxt = ctx.new_particles(P, device=x0.device)
        checkpoints = {}
        for n in range(n_steps):
            if n % k == 0:
                checkpoints[n] = _copy_state(ctx, state)
            pp.polypic_step(ctx, state, nxt, grid, params, ws)
            state, nxt = nxt, state
        st = pp.polypic_check_device_status(ctx)
        if st != 0:
            raise pp.PolyPICError(st, "rollout forward")
        fctx.ctx_ = ctx
        fctx.n_steps, fctx.dt, fctx.k = n_steps, dt, k
        fctx.params = params
        fctx.checkpoints = checkpoints
        fctx.ws = ws
        vel = [v.clone() for v in grid.vel]
        gmass = [m.clone() for m in grid.mass]
        for m in gmass:
            fctx.mark_non_differentiable(m)
        return (*vel, *gmass)

    @staticmethod
    def backward(fctx, gv0, gv1, gv2, _gm0, _gm1, _gm2):
        ctx: pp.Context = fctx.ctx_
        N, dt, k = fctx.n_steps, fctx.dt, fctx.k
        params, ws = fctx.params, fctx.ws
        grads_v = [g if g is not None else None for g in (gv0, gv1, gv2)]
        some = next(g for g in grads_v if g is not None)
        dev = some.device
        first = fctx.checkpoints[0]
        P = first.count
        R = ctx.num_modes
        # adjoint of the state after the last step (it does not reach the loss)
        lam_next = ctx.new_particles(P, device=dev)
        lam_next.x.zero_()
        lam_next.coeff.zero_()
        for seg_start in sorted(fctx.checkpoints.keys(), reverse=True):
            seg_end = min(seg_start + k, N)
            # recompute the segment, keeping each step's input state and grid
            states: List[pp.ParticleState] = []
            grids: List[pp.GridState] = []
            cur = _copy_state(ctx, fctx.checkpoints[seg_start])
            for n in range(seg_start, seg_end):
                g = ctx.new_grid(device=dev)
                out = ctx.new_particles(P, device=dev)
                pp.polypic_step(ctx, cur, out, g, params, ws)
                states.append(cur)
                grids.append(g)
                cur = out
            for i in range(seg_end - seg_start - 1, -1, -1):
                n = seg_start + i
                s, g = states[i], grids[i]
                bar_grid = _zeros_like_grid(g)
                if n == N - 1:
                    for a in range(3):
                        if grads_v[a] is not None:
                            bar_grid.vel[a].copy_(grads_v[a])
                lam = ctx.new_particles(P, device=dev)
                lam.x.zero_()
                lam.coeff.zero_()
                pp.polypic_g2p_adjoint(ctx, g, s, dt, lam_next, bar_grid, lam, ws, accumulate=True)
                pp.polypic_grid_update_adjoint(ctx, g, params, bar_grid, bar_grid)
                pp.polypic_p2g_adjoint(ctx, s, bar_grid, lam, ws, accumulate=True)
                lam_next = lam
        st = pp.polypic_check_device_status(ctx)
        if st != 0:
            raise pp.PolyPICError(st, "rollout backward")
        return lam_next.coeff, lam_next.x, None, None, None, None, None, None


def rollout(ctx: pp.Context, x0: torch.Tensor, mass: torch.Tensor, c0: torch.Tensor,
            n_steps: int, dt: float, gravity=(0.0, -9.81, 0.0), checkpoint_every: int = 8):
    """Differentiable n-step rollout.  Returns (vel[3], mass[3]) of the last
    step's grid; vel carries gradients to c0 (3, R, P) and x0 (3, P)."""
    out = _Rollout.apply(c0, x0, mass, ctx, int(n_steps), float(dt), tuple(gravity),
                         int(checkpoint_every))
    return list(out[:3]), list(out[3:])


def taylor_green_loss(vel: List[torch.Tensor], gmass: List[torch.Tensor],
                      target: List[torch.Tensor]) -> torch.Tensor:
    """L = 1/2 sum over faces with m > 0 of (v~ - u_TG)^2."""
    loss = 0.0
    for v, m, u in zip(vel, gmass, target):
        d = torch.where(m > 0, v - u, torch.zeros_like(v))
        loss = loss + 0.5 * (d * d).sum()
    return loss

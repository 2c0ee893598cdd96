"""Differentiable rollout of PolyPIC transfer steps.

``rollout(ctx, x0, mass, c0, n_steps, dt, ...)`` runs ``n_steps`` steps (sort,
P2G, grid update, G2P with advection) through the C library and returns the
last step's fluid grid velocity and mass.  Gradients of a loss on that
velocity flow back to the initial coefficients ``c0`` (every mode, including
the particle velocity c_0) and the initial positions ``x0`` through the
library's hand-written adjoints: polypic_g2p_adjoint,
polypic_grid_update_adjoint and polypic_p2g_adjoint, chained step by step in
reverse.

Options: ``project=True`` adds the pressure projection to every step (its
adjoint is the projection of the wall-zeroed adjoint velocity, the
walls-then-projection map being an orthogonal projector); ``solid=(xs0,
ms, mabs, cs0)`` adds a solid phase (Eqs 18-20: weight m_s + m_abs) coupled
to the fluid by the implicit drag of strength ``drag_k``, and the gradient
then also reaches ``cs0`` and ``xs0``.  The fluid-cell set of the projection
and the stencil decisions are piecewise constant: they pass no gradient.

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
    out = ctx.new_particles(s.count, solid=s.mass_abs is not None, device=s.x.device)
    out.x.copy_(s.x)
    out.mass.copy_(s.mass)
    out.coeff.copy_(s.coeff)
    if s.mass_abs is not None:
        out.mass_abs.copy_(s.mass_abs)
    return out


def _zeros_like_grid(g: pp.GridState) -> pp.GridState:
    z = lambda ts: [torch.zeros_like(t) for t in ts]
    return pp.GridState(mass=z(g.vel), mom=z(g.vel), vel=z(g.vel))


def _new_state(ctx, x, mass, coeff, mass_abs=None):
    s = ctx.new_particles(x.shape[1], solid=mass_abs is not None, device=x.device)
    s.x.copy_(x)
    s.mass.copy_(mass)
    s.coeff.copy_(coeff)
    if mass_abs is not None:
        s.mass_abs.copy_(mass_abs)
    return s


def _zero_adjoint(ctx, P, dev):
    lam = ctx.new_particles(P, device=dev)
    lam.x.zero_()
    lam.coeff.zero_()
    return lam


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(fctx, c0, x0, cs0, xs0, mass, ms, mabs, ctx: pp.Context, n_steps: int,
                params: pp.UpdateSettings, k: int):
        if ctx.coeff_format != "f32":
            raise pp.PolyPICError(2, "rollout: only FP32 coefficients are differentiable")
        two = cs0 is not None
        P = x0.shape[1]
        Ps = xs0.shape[1] if two else 0
        dev = x0.device
        state = _new_state(ctx, x0, mass, c0)
        sstate = _new_state(ctx, xs0, ms, cs0, mabs) if two else None
        ws = ctx.workspace(P, Ps, device=dev)
        grid = ctx.new_grid(device=dev)
        sgrid = ctx.new_grid(device=dev) if two else None
        nxt = ctx.new_particles(P, device=dev)
        snxt = ctx.new_particles(Ps, solid=True, device=dev) if two else None
        checkpoints = {}
        for n in range(n_steps):
            if n % k == 0:
                checkpoints[n] = (_copy_state(ctx, state),
                                  _copy_state(ctx, sstate) if two else None)
            pp.polypic_step(ctx, state, nxt, grid, params, ws, solid_in=sstate, solid_out=snxt,
                            gs=sgrid)
            state, nxt = nxt, state
            if two:
                sstate, snxt = snxt, sstate
        st = pp.polypic_check_device_status(ctx)
        if st != 0:
            raise pp.PolyPICError(st, "rollout forward")
        fctx.ctx_ = ctx
        fctx.n_steps, fctx.k, fctx.two = n_steps, k, two
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
        N, k, two = fctx.n_steps, fctx.k, fctx.two
        params, ws = fctx.params, fctx.ws
        dt = params.dt
        grads_v = [gv0, gv1, gv2]
        dev = next(g for g in grads_v if g is not None).device
        first, sfirst = fctx.checkpoints[0]
        P = first.count
        Ps = sfirst.count if two else 0
        # adjoints of the states after the last step (they do not reach the loss)
        lam_next = _zero_adjoint(ctx, P, dev)
        slam_next = _zero_adjoint(ctx, Ps, dev) if two else None
        for seg_start in sorted(fctx.checkpoints.keys(), reverse=True):
            seg_end = min(seg_start + k, N)
            # recompute the segment, keeping each step's input states and grids
            steps = []
            cur = _copy_state(ctx, fctx.checkpoints[seg_start][0])
            scur = _copy_state(ctx, fctx.checkpoints[seg_start][1]) if two else None
            for n in range(seg_start, seg_end):
                g = ctx.new_grid(device=dev)
                gs = ctx.new_grid(device=dev) if two else None
                out = ctx.new_particles(P, device=dev)
                sout = ctx.new_particles(Ps, solid=True, device=dev) if two else None
                pp.polypic_step(ctx, cur, out, g, params, ws, solid_in=scur, solid_out=sout,
                                gs=gs)
                steps.append((cur, scur, g, gs))
                cur, scur = out, sout
            for i in range(seg_end - seg_start - 1, -1, -1):
                n = seg_start + i
                s, ss, g, gs = steps[i]
                bar_g = _zeros_like_grid(g)
                bar_gs = _zeros_like_grid(gs) if two else None
                if n == N - 1:
                    for a in range(3):
                        if grads_v[a] is not None:
                            bar_g.vel[a].copy_(grads_v[a])
                lam = _zero_adjoint(ctx, P, dev)
                pp.polypic_g2p_adjoint(ctx, g, s, dt, lam_next, bar_g, lam, ws, accumulate=True)
                slam = None
                if two:
                    slam = _zero_adjoint(ctx, Ps, dev)
                    pp.polypic_g2p_adjoint(ctx, gs, ss, dt, slam_next, bar_gs, slam, ws,
                                           accumulate=True)
                pp.polypic_grid_update_adjoint(ctx, g, params, bar_g, bar_g, solid=gs,
                                               bar_solid_out=bar_gs, bar_solid_in=bar_gs,
                                               fluid_particles=s, ws=ws)
                pp.polypic_p2g_adjoint(ctx, s, bar_g, lam, ws, accumulate=True)
                if two:
                    pp.polypic_p2g_adjoint(ctx, ss, bar_gs, slam, ws, accumulate=True)
                lam_next, slam_next = lam, slam
        st = pp.polypic_check_device_status(ctx)
        if st != 0:
            raise pp.PolyPICError(st, "rollout backward")
        return (lam_next.coeff, lam_next.x, slam_next.coeff if two else None,
                slam_next.x if two else None, None, None, None, None, None, None, None)


def rollout(ctx: pp.Context, x0: torch.Tensor, mass: torch.Tensor, c0: torch.Tensor,
            n_steps: int, dt: float, gravity=(0.0, -9.81, 0.0), checkpoint_every: int = 8,
            project: bool = False, solid=None, drag_k: float = 0.0, pcg_rtol: float = 1e-6,
            pcg_maxiter: int = 2000):
    """Differentiable n-step rollout.  Returns (vel[3], mass[3]) of the last
    step's fluid grid; vel carries gradients to c0 (3, R, P) and x0 (3, P),
    and with solid = (xs0, ms, mabs, cs0) to cs0 and xs0 as well."""
    params = pp.UpdateSettings(dt=float(dt), gravity=tuple(gravity), drag_k=float(drag_k),
                               project=bool(project), pcg_rtol=float(pcg_rtol),
                               pcg_maxiter=int(pcg_maxiter))
    if solid is not None:
        xs0, ms, mabs, cs0 = solid
    else:
        xs0 = ms = mabs = cs0 = None
    out = _Rollout.apply(c0, x0, cs0, xs0, mass, ms, mabs, ctx, int(n_steps), params,
                         int(checkpoint_every))
    return list(out[:3]), list(out[3:])


def taylor_green_loss(vel: List[torch.Tensor], gmass: List[torch.Tensor],
                      target: List[torch.Tensor], min_mass: float = 0.0) -> torch.Tensor:
    """L = 1/2 sum over faces with m > min_mass of (v~ - u_TG)^2."""
    loss = 0.0
    for v, m, u in zip(vel, gmass, target):
        d = torch.where(m > min_mass, v - u, torch.zeros_like(v))
        loss = loss + 0.5 * (d * d).sum()
    return loss

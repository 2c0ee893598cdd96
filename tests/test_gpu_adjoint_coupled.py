"""The differentiable rollout with every part of the grid update: a fluid
half box (random velocities and modes) and a fabric sheet inside it (solid
phase, Eqs 18-20, with absorbed mass), coupled by the implicit drag, and the
pressure projection on the fluid cells every step.  N = 8 steps with a
checkpoint every 4 on 16^3; the loss is the L2 distance of the final fluid
grid velocity to the Taylor-Green field; gradients with respect to the
initial modes of both phases.

The GPU gradient (torch.autograd through the hand-written adjoints) is
compared with the FP64 oracle's chained adjoint, element by element, and
with FP64 central differences of the oracle's forward on random directions
in velocity units (the median direction within 1e-4, the worst within
2e-4).  The loss is only piecewise smooth (the guard band of the degenerate
quadratic fit, the faces holding mass, and here also the set of fluid cells
the projection runs on), so a direction whose differences at h and h/2
disagree crossed a jump and is drawn again."""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2308_01060_gb300 import autograd as pag
from paper_2308_01060_gb300 import polypic as pp
from paper_2308_01060_gb300 import scenes
from gpu_util import assert_close, np_

pytestmark = pytest.mark.gpu

STEPS, EVERY, K_DRAG, RTOL = 8, 4, 0.05, 1e-12
G = (0.0, -9.81, 0.0)
TOL_VECTOR, TOL_FD_MEDIAN, TOL_FD_WORST = 2e-4, 1e-4, 2e-4


def _scene(n, R, seed):
    sc = scenes.random_velocity_scene(n=n, R=R, seed=seed, sigma_v=0.3, dt=1e-3, steps=STEPS)
    rng = np.random.default_rng(seed + 100)
    xs, ms, _ = scenes.sheet_particles(16, 0.6, 0.3)
    cs = scenes.random_modes(R, xs.shape[1], sc.dx, rng)
    cs[:, 0] = rng.normal(0.0, 0.1, (3, xs.shape[1]))
    mabs = (rng.uniform(0.0, 1.0, xs.shape[1]) * ms).astype(np.float32)
    return sc, xs, ms, mabs, cs.astype(np.float32)


def _fluid_cells(x, n, dx):
    k = np.floor(x.astype(np.float32) * np.float32(1.0 / dx)).astype(int)
    fl = np.zeros((n[2], n[1], n[0]), dtype=bool)
    fl[k[2], k[1], k[0]] = True
    return fl


def _forward(st, n, dx, dt, steps, keep):
    """The oracle's coupled step: P2G of both phases, the update with drag,
    the projection on the cells holding fluid particles, G2P of both."""
    xf, mf, cf, xs, ms, mabs, cs = st
    R = cf.shape[1]
    out = []
    for _ in range(steps):
        gm, gp = oracle.p2g(xf, mf, cf, n, dx)
        sgm, sgp = oracle.p2g(xs, ms, cs, n, dx, mass_abs=mabs)
        gv, sv = oracle.grid_update(n, dt, G, gm, gp, sgm, sgp, drag_k=K_DRAG)
        fl = _fluid_cells(xf, n, dx)
        gv, _, _ = oracle.pcg_project(n, dx, dt, 1000.0, fl, gv, rtol=RTOL, maxiter=5000)
        rec = (xf, cf, xs, cs, gm, gp, sgm, sgp, gv, sv, fl)
        out = out + [rec] if keep else [rec]
        cf, xf = oracle.g2p(xf, gv, R, n, dx, dt)
        cs, xs = oracle.g2p(xs, sv, R, n, dx, dt)
    return out


def _loss(recs, target):
    gm, gv = recs[-1][4], recs[-1][8]
    return sum(0.5 * np.sum(np.where(gm[a] > 0, gv[a] - target[a], 0.0) ** 2) for a in range(3))


def _gradient(recs, mf, ms, mabs, n, dx, dt, target):
    """The oracle's FP64 adjoint of its own forward, chained step by step:
    (dL/dcf0, dL/dcs0)."""
    R = recs[0][1].shape[1]
    P, Ps = mf.shape[0], ms.shape[0]
    lcf, lxf = np.zeros((3, R, P)), np.zeros((3, P))
    lcs, lxs = np.zeros((3, R, Ps)), np.zeros((3, Ps))
    for i in range(len(recs) - 1, -1, -1):
        xf, cf, xs, cs, gm, gp, sgm, sgp, gv, sv, fl = recs[i]
        if i == len(recs) - 1:
            lvf = [np.where(gm[a] > 0, gv[a] - target[a], 0.0) for a in range(3)]
            lvs = [np.zeros_like(a) for a in sv]
            lxf0, lxs0 = np.zeros((3, P)), np.zeros((3, Ps))
        else:
            lvf, lxf0 = oracle.g2p_adjoint(xf, gv, R, n, dx, dt, lcf, lxf)
            lvs, lxs0 = oracle.g2p_adjoint(xs, sv, R, n, dx, dt, lcs, lxs)
        lm, lp, lsm, lsp = oracle.grid_update_adjoint(n, gm, gp, lvf, dt=dt, gravity=G, sm=sgm,
                                                      sp=sgp, lsv=lvs, drag_k=K_DRAG, fluid=fl,
                                                      rtol=RTOL)
        c1, x1 = oracle.p2g_adjoint(xf, mf, cf, n, dx, lm, lp)
        c2, x2 = oracle.p2g_adjoint(xs, ms, cs, n, dx, lsm, lsp, mass_abs=mabs)
        lcf, lxf = c1, lxf0 + x1
        lcs, lxs = c2, lxs0 + x2
    return lcf, lcs


def _gate(n, R, directions, seed):
    sc, xs, ms, mabs, cs = _scene(n, R, seed)
    f = sc.fluid
    dx, dt = sc.dx, sc.dt
    ctx = pp.Context(sc.n, dx, R)
    target = [scenes.taylor_green(scenes.face_positions(a, sc.n, dx), a) for a in range(3)]
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    c0 = dev(f.coeff).requires_grad_(True)
    cs0 = dev(cs).requires_grad_(True)
    vel, gmass = pag.rollout(ctx, dev(f.x), dev(f.mass), c0, STEPS, dt, checkpoint_every=EVERY,
                             project=True, drag_k=K_DRAG,
                             solid=(dev(xs), dev(ms), dev(mabs), cs0))
    tgt = [torch.from_numpy(t.astype(np.float32)).cuda() for t in target]
    loss = pag.taylor_green_loss(vel, gmass, tgt)
    loss.backward()
    gf = np_(c0.grad).astype(np.float64)
    gs = np_(cs0.grad).astype(np.float64)
    assert pp.polypic_check_device_status(ctx) == 0

    st0 = tuple(a.astype(np.float64) for a in (f.x, f.mass, f.coeff, xs, ms, mabs, cs))
    oracle.set_threads(os.cpu_count() or 1)
    try:
        recs = _forward(st0, sc.n, dx, dt, STEPS, keep=True)
        L0 = _loss(recs, target)
        assert abs(loss.item() - L0) <= 1e-4 * abs(L0)
        of, os_ = _gradient(recs, st0[1], st0[4], st0[5], sc.n, dx, dt, target)
        del recs
        assert_close(gf, of, TOL_VECTOR, "dL/dc0 of the fluid against the oracle's adjoint")
        assert_close(gs, os_, TOL_VECTOR, "dL/dc0 of the sheet against the oracle's adjoint")
        assert np.linalg.norm(os_) > 0          # the drag carries gradient to the sheet
        rng = np.random.default_rng(2)
        deg = scenes.mode_degrees(R).astype(np.float64)
        w = 1.0 / (dx ** deg)[None, :, None]
        scale = np.linalg.norm(np.concatenate([(of * w).ravel(), (os_ * w).ravel()]))

        def fd(df, ds, h):
            def L(s):
                st = list(st0)
                st[2] = st0[2] + s * df
                st[6] = st0[6] + s * ds
                return _loss(_forward(tuple(st), sc.n, dx, dt, STEPS, keep=False), target)
            return (L(h) - L(-h)) / (2 * h)

        errs, redrawn = [], 0
        while len(errs) < directions:
            uf = rng.standard_normal(st0[2].shape)
            us = rng.standard_normal(st0[6].shape)
            nrm = np.sqrt(np.sum(uf ** 2) + np.sum(us ** 2))
            df, ds = uf / nrm * w, us / nrm * w
            h = 1e-2
            f1, f2 = fd(df, ds, h), fd(df, ds, h / 2)
            if abs(f1 - f2) > 1e-3 * max(abs(f2), 1e-3 * scale):
                redrawn += 1
                assert redrawn <= max(2, directions // 4), "too many directions cross a jump"
                continue
            an = float(np.sum(gf * df) + np.sum(gs * ds))
            errs.append((abs(f2 - an) / max(abs(f2), 1e-3 * scale), f2, an))
        worst = max(errs)
        med = float(np.median([e[0] for e in errs]))
        print(f"coupled rollout, {directions} directions: worst {worst[0]:.3e} "
              f"(fd {worst[1]:.6e}, adjoint {worst[2]:.6e}), median {med:.3e}, "
              f"redrawn {redrawn}")
        assert med <= TOL_FD_MEDIAN, errs
        assert worst[0] <= TOL_FD_WORST, worst
    finally:
        oracle.set_threads(1)


def test_coupled_projected_rollout_gate_16cube_8_steps():
    _gate(16, 27, 16, seed=6)

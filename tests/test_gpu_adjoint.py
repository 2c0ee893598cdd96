"""GPU adjoints against the FP64 oracle.

  * each adjoint entry point (G2P, grid update, P2G) against the oracle's
    transposed transfer on identical seeded inputs;
  * the differentiable rollout's gradient (loss = L2 distance of the last
    grid velocity to a Taylor-Green field) against the oracle's chained FP64
    adjoint and against FP64 central finite differences of the oracle's own
    forward on random directions (tolerance 1e-4 relative).
"""
import numpy as np
import pytest
import torch

import oracle
import slot_layout
from paper_2308_01060_gb300 import autograd as pag
from paper_2308_01060_gb300 import polypic as pp
from paper_2308_01060_gb300 import scenes
from gpu_util import assert_close, grid_from_host, np_, random_grid_velocity, rel, sorted_particles

pytestmark = pytest.mark.gpu


def _scene(n=16, R=27, seed=0):
    return scenes.random_velocity_scene(n=n, R=R, seed=seed, sigma_v=0.3, dt=2e-3, steps=4)


@pytest.mark.parametrize("R", [1, 4, 8, 27])
def test_p2g_adjoint_matches_oracle(R):
    sc = _scene(R=R, seed=R)
    f = sc.fluid
    ctx = pp.Context(sc.n, sc.dx, R)
    ps, ws = sorted_particles(ctx, f)
    rng = np.random.default_rng(100 + R)
    lm = [rng.standard_normal(oracle.face_shape(a, sc.n)).astype(np.float32) for a in range(3)]
    lp = [rng.standard_normal(oracle.face_shape(a, sc.n)).astype(np.float32) for a in range(3)]
    bar_grid = grid_from_host(ctx, mass=lm, mom=lp)
    bar_in = ctx.new_particles(ps.count)
    pp.polypic_p2g_adjoint(ctx, ps, bar_grid, bar_in, ws)
    lc_or, lx_or = oracle.p2g_adjoint(f.x, f.mass, f.coeff, sc.n, sc.dx, lm, lp)
    assert_close(np_(bar_in.coeff), lc_or, 1e-5)
    assert_close(np_(bar_in.x), lx_or, 1e-4)
    assert pp.polypic_check_device_status(ctx) == 0


@pytest.mark.parametrize("R", [1, 4, 8, 27])
def test_g2p_adjoint_matches_oracle(R):
    sc = _scene(R=R, seed=10 + R)
    f = sc.fluid
    ctx = pp.Context(sc.n, sc.dx, R)
    ps, ws = sorted_particles(ctx, f)
    gv = random_grid_velocity(sc.n, sc.dx, seed=R)
    g = grid_from_host(ctx, vel=gv)
    rng = np.random.default_rng(200 + R)
    deg = scenes.mode_degrees(R)
    lc_out = (rng.standard_normal((3, R, f.n)) * (sc.dx ** deg)[None, :, None]).astype(np.float32)
    lx_out = rng.standard_normal((3, f.n)).astype(np.float32)
    perm = slot_layout.library_order(f.x, sc.n, sc.dx)[0]
    bar_out = ctx.new_particles(f.n)                       # slot order
    bar_out.coeff.copy_(torch.from_numpy(np.ascontiguousarray(lc_out[:, :, perm])))
    bar_out.x.copy_(torch.from_numpy(np.ascontiguousarray(lx_out[:, perm])))
    bar_grid = ctx.new_grid()
    bar_in = ctx.new_particles(f.n)
    dt = 2e-3
    pp.polypic_g2p_adjoint(ctx, g, ps, dt, bar_out, bar_grid, bar_in, ws)
    lv_or, lx_or = oracle.g2p_adjoint(f.x, gv, R, sc.n, sc.dx, dt, lc_out, lx_out)
    for a in range(3):
        assert_close(np_(bar_grid.vel[a]), lv_or[a], 1e-5)
    assert_close(np_(bar_in.x), lx_or, 1e-4)
    # determinism of the scatter
    bar_grid2 = ctx.new_grid()
    pp.polypic_g2p_adjoint(ctx, g, ps, dt, bar_out, bar_grid2, bar_in, ws)
    for a in range(3):
        assert torch.equal(bar_grid.vel[a], bar_grid2.vel[a])


def test_grid_update_adjoint_matches_oracle():
    n = (12, 10, 8)
    rng = np.random.default_rng(5)
    ctx = pp.Context(n, 1 / 12, 1)
    shapes = [oracle.face_shape(a, n) for a in range(3)]
    fm = [(rng.uniform(0, 2, s) * (rng.uniform(size=s) > 0.3)).astype(np.float32) for s in shapes]
    fp = [rng.standard_normal(s).astype(np.float32) for s in shapes]
    lv = [rng.standard_normal(s).astype(np.float32) for s in shapes]
    g = grid_from_host(ctx, mass=fm, mom=fp)
    bar = grid_from_host(ctx, vel=lv)
    out = ctx.new_grid()
    pp.polypic_grid_update_adjoint(ctx, g, pp.UpdateSettings(dt=1e-3), bar, out)
    lm_or, lp_or = oracle.grid_update_adjoint(n, fm, fp, lv)
    for a in range(3):
        assert_close(np_(out.mass[a]), lm_or[a], 1e-6)
        assert_close(np_(out.mom[a]), lp_or[a], 1e-6)


# ------------------------------------------------------------------ rollout gradient

def _tg_target(n, dx):
    return [scenes.taylor_green(scenes.face_positions(a, n, dx), a) for a in range(3)]


def _oracle_forward(x, mass, c, n, dx, dt, steps, g=(0.0, -9.81, 0.0)):
    states = []
    for _ in range(steps):
        gm, gp = oracle.p2g(x, mass, c, n, dx)
        gv = oracle.grid_update(n, dt, g, gm, gp)
        states.append((x, c, gm, gp, gv))
        c, x = oracle.g2p(x, gv, c.shape[1], n, dx, dt)
    return states


def _oracle_loss(states, target):
    _, _, gm, _, gv = states[-1]
    return sum(0.5 * np.sum(np.where(gm[a] > 0, gv[a] - target[a], 0.0) ** 2) for a in range(3))


def _oracle_gradient(states, mass, n, dx, dt, target):
    """Chained FP64 adjoint of the oracle forward: dL/dc0, dL/dx0."""
    R = states[0][1].shape[1]
    P = mass.shape[0]
    lc_next = np.zeros((3, R, P))
    lx_next = np.zeros((3, P))
    for i in range(len(states) - 1, -1, -1):
        x, c, gm, gp, gv = states[i]
        if i == len(states) - 1:
            lv = [np.where(gm[a] > 0, gv[a] - target[a], 0.0) for a in range(3)]
            lx = np.zeros((3, P))
        else:
            lv, lx = oracle.g2p_adjoint(x, gv, R, n, dx, dt, lc_next, lx_next)
        lm, lp = oracle.grid_update_adjoint(n, gm, gp, lv)
        lc, lx2 = oracle.p2g_adjoint(x, mass, c, n, dx, lm, lp)
        lc_next, lx_next = lc, lx + lx2
    return lc_next, lx_next


@pytest.mark.parametrize("R", [4, 27])
def test_rollout_gradient_matches_oracle_and_finite_differences(R):
    sc = scenes.random_velocity_scene(n=16, R=R, seed=3, sigma_v=0.3, dt=2e-3, steps=4)
    f = sc.fluid
    n, dx, dt, steps = sc.n, sc.dx, sc.dt, 4
    ctx = pp.Context(n, dx, R)
    x0 = torch.from_numpy(f.x).cuda()
    m0 = torch.from_numpy(f.mass).cuda()
    c0 = torch.from_numpy(f.coeff).cuda().requires_grad_(True)
    target = _tg_target(n, dx)
    tgt = [torch.from_numpy(t.astype(np.float32)).cuda() for t in target]
    vel, gmass = pag.rollout(ctx, x0, m0, c0, steps, dt, checkpoint_every=2)
    loss = pag.taylor_green_loss(vel, gmass, tgt)
    loss.backward()
    g_gpu = np_(c0.grad).astype(np.float64)

    x64, c64, m64 = f.x.astype(np.float64), f.coeff.astype(np.float64), f.mass.astype(np.float64)
    states = _oracle_forward(x64, m64, c64, n, dx, dt, steps)
    L0 = _oracle_loss(states, target)
    assert abs(loss.item() - L0) <= 1e-4 * abs(L0)
    g_or, _ = _oracle_gradient(states, m64, n, dx, dt, target)
    assert_close(g_gpu, g_or, 1e-4)

    rng = np.random.default_rng(1)
    deg = scenes.mode_degrees(R)
    for _ in range(4):
        d = rng.standard_normal(c64.shape) / (dx ** deg)[None, :, None]
        d /= np.linalg.norm(d)
        h = 1e-3 * np.linalg.norm(c64) / np.sqrt(c64.size) * np.sqrt(d.size)
        Lp = _oracle_loss(_oracle_forward(x64, m64, c64 + h * d, n, dx, dt, steps), target)
        Lm = _oracle_loss(_oracle_forward(x64, m64, c64 - h * d, n, dx, dt, steps), target)
        fd = (Lp - Lm) / (2 * h)
        an = float(np.sum(g_gpu * d))
        assert abs(fd - an) <= 1e-4 * max(abs(fd), 1e-3 * np.linalg.norm(g_or)), (fd, an)


def test_adjoints_at_64cube_match_oracle():
    """Both particle adjoints on the full-size workload of the rollout (64^3
    half box, 864,000 particles, 27 modes), every tile interior or seam,
    element by element against the oracle on all host cores."""
    import os
    sc = scenes.random_velocity_scene(n=64, R=27, seed=3, sigma_v=0.3, dt=1e-3, steps=1)
    f = sc.fluid
    ctx = pp.Context(sc.n, sc.dx, 27)
    ps, ws = sorted_particles(ctx, f)
    rng = np.random.default_rng(301)
    lm = [rng.standard_normal(oracle.face_shape(a, sc.n)).astype(np.float32) for a in range(3)]
    lp = [rng.standard_normal(oracle.face_shape(a, sc.n)).astype(np.float32) for a in range(3)]
    bar_grid = grid_from_host(ctx, mass=lm, mom=lp)
    bar_in = ctx.new_particles(ps.count)
    pp.polypic_p2g_adjoint(ctx, ps, bar_grid, bar_in, ws)
    gv = random_grid_velocity(sc.n, sc.dx, seed=302)
    g = grid_from_host(ctx, vel=gv)
    deg = scenes.mode_degrees(27)
    lc_out = (rng.standard_normal((3, 27, f.n)) * (sc.dx ** deg)[None, :, None]).astype(np.float32)
    lx_out = rng.standard_normal((3, f.n)).astype(np.float32)
    perm = slot_layout.library_order(f.x, sc.n, sc.dx)[0]
    bar_out = ctx.new_particles(f.n)
    bar_out.coeff.copy_(torch.from_numpy(np.ascontiguousarray(lc_out[:, :, perm])))
    bar_out.x.copy_(torch.from_numpy(np.ascontiguousarray(lx_out[:, perm])))
    bar_v = ctx.new_grid()
    bar_x = ctx.new_particles(f.n)
    pp.polypic_g2p_adjoint(ctx, g, ps, sc.dt, bar_out, bar_v, bar_x, ws)
    assert pp.polypic_check_device_status(ctx) == 0
    oracle.set_threads(os.cpu_count() or 1)
    try:
        lc_or, lx_or = oracle.p2g_adjoint(f.x, f.mass, f.coeff, sc.n, sc.dx, lm, lp)
        lv_or, lx2_or = oracle.g2p_adjoint(f.x, gv, 27, sc.n, sc.dx, sc.dt, lc_out, lx_out)
    finally:
        oracle.set_threads(1)
    assert_close(np_(bar_in.coeff), lc_or, 1e-5, "P2G adjoint, coefficients")
    assert_close(np_(bar_in.x), lx_or, 1e-4, "P2G adjoint, positions")
    for a in range(3):
        assert_close(np_(bar_v.vel[a]), lv_or[a], 1e-5, f"G2P adjoint, grid {a}")
    assert_close(np_(bar_x.x), lx2_or, 1e-4, "G2P adjoint, positions")

"""polypic_g2p2g, the fused transfer (G2P of step n and P2G of step n + 1 in
one pass), against the FP64 oracle: the oracle's G2P (fit and advection)
followed by its P2G of the new state with the new coefficients.  The new
positions must carry the same bits as polypic_g2p's, the movers' coefficients
too; the grid of step n + 1 agrees element by element.  Velocities large
enough that a good share of the particles change cell exercise the spill
path (compaction, sort, P2G added onto the grid)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2308_01060_gb300 import polypic as pp
from paper_2308_01060_gb300 import scenes
from gpu_util import assert_close, grid_from_host, np_, random_grid_velocity, sorted_particles, u32

pytestmark = pytest.mark.gpu

N = (32, 32, 32)
DX = 1.0 / 32


def _setup(R, seed, solid=False, amp=3.0):
    sc = scenes.parity_scene(n=32, R=R, seed=seed, random_mode_init=True)
    f = sc.fluid
    mabs = None
    if solid:
        mabs = (np.random.default_rng(seed + 1).uniform(0, 1, f.n) * f.mass).astype(np.float32)
    ctx = pp.Context(N, DX, R)
    host = scenes.ParticleSet(x=f.x, mass=f.mass, coeff=f.coeff, mass_abs=mabs, num_modes=R)
    ps, ws = sorted_particles(ctx, host)
    gv = random_grid_velocity(N, DX, seed=seed + 2, amp=amp)
    g = grid_from_host(ctx, vel=gv)
    return ctx, f, mabs, ps, ws, g, gv


def _spill(ctx, P, solid):
    return ctx.new_particles(P, solid=solid)


@pytest.mark.parametrize("R", [27, 4, 1])
def test_g2p2g_matches_oracle_and_g2p(R):
    ctx, f, mabs, ps, ws, g, gv = _setup(R, 41)
    dt = 2e-3                                   # |v| dt / dx ~ 0.2-0.5: many movers
    out = ctx.new_particles(ps.count)
    spill = _spill(ctx, ps.count, False)
    gn = ctx.new_grid(vel=False)
    pp.polypic_g2p2g(ctx, g, ps, out, spill, gn, dt, ws)
    assert pp.polypic_check_device_status(ctx) == 0
    # the unfused G2P of the same state: positions bit for bit, movers' modes too
    ref = ctx.new_particles(ps.count)
    pp.polypic_g2p(ctx, g, ps, ref, dt, ws)
    assert torch.equal(out.x, ref.x) and torch.equal(out.mass, ref.mass)
    perm = u32(ps.perm)
    x0 = f.x[:, perm]
    k0 = np.floor(x0 * np.float32(1 / DX)).astype(int)
    k1 = np.floor(np_(out.x) * np.float32(1 / DX)).astype(int)
    movers = np.any(k0 != k1, axis=0)
    assert 0.05 * ps.count < movers.sum() < 0.95 * ps.count, movers.sum()
    assert torch.equal(out.coeff[:, :, torch.from_numpy(movers).cuda()],
                       ref.coeff[:, :, torch.from_numpy(movers).cuda()])
    # the grid of step n + 1 against the oracle's G2P then P2G
    c1, x1 = oracle.g2p(f.x, gv, R, N, DX, dt)
    gm, gp = oracle.p2g(x1, f.mass, c1, N, DX)
    for a in range(3):
        assert_close(np_(gn.mass[a]), gm[a], 1e-5, f"mass {a}")
        assert_close(np_(gn.mom[a]), gp[a], 1e-5, f"momentum {a}")
    assert_close(np_(out.x), x1[:, perm], 1e-6, "positions")
    # and against the unfused P2G of the GPU's own new state (other sum order)
    pp.polypic_sort(ctx, ref, ws)
    gr = ctx.new_grid(vel=False)
    pp.polypic_p2g(ctx, ref, gr, ws)
    for a in range(3):
        assert_close(np_(gn.mom[a]), np_(gr.mom[a]), 1e-5, f"vs unfused {a}")


def test_g2p2g_solid_phase_and_determinism():
    ctx, f, mabs, ps, ws, g, gv = _setup(8, 42, solid=True)
    dt = 2e-3
    outs = []
    for _ in range(2):
        out = ctx.new_particles(ps.count, solid=True)
        spill = _spill(ctx, ps.count, True)
        gn = ctx.new_grid(vel=False)
        pp.polypic_g2p2g(ctx, g, ps, out, spill, gn, dt, ws)
        outs.append((out, gn))
    assert pp.polypic_check_device_status(ctx) == 0
    for a in range(3):
        assert torch.equal(outs[0][1].mass[a], outs[1][1].mass[a])
        assert torch.equal(outs[0][1].mom[a], outs[1][1].mom[a])
    c1, x1 = oracle.g2p(f.x, gv, 8, N, DX, dt)
    gm, gp = oracle.p2g(x1, f.mass, c1, N, DX, mass_abs=mabs)
    for a in range(3):
        assert_close(np_(outs[0][1].mass[a]), gm[a], 1e-5, f"mass {a}")
        assert_close(np_(outs[0][1].mom[a]), gp[a], 1e-5, f"momentum {a}")
    assert np.array_equal(np_(outs[0][0].mass_abs), mabs[u32(ps.perm)])


def test_g2p2g_refuses_a_spill_set_too_small():
    ctx, f, mabs, ps, ws, g, gv = _setup(4, 43)
    out = ctx.new_particles(ps.count)
    spill = _spill(ctx, 16, False)
    gn = ctx.new_grid(vel=False)
    with pytest.raises(pp.PolyPICError) as ei:
        pp.polypic_g2p2g(ctx, g, ps, out, spill, gn, 2e-3, ws)
    assert ei.value.name == "WORKSPACE"
    assert pp.polypic_check_device_status(ctx) == 0


def test_g2p2g_without_movers_and_unsupported_formats():
    ctx, f, mabs, ps, ws, g, gv = _setup(4, 44)
    out = ctx.new_particles(ps.count)
    spill = _spill(ctx, 0, False)               # dt = 0: nobody moves, no spill needed
    gn = ctx.new_grid(vel=False)
    pp.polypic_g2p2g(ctx, g, ps, out, spill, gn, 0.0, ws)
    c1, x1 = oracle.g2p(f.x, gv, 4, N, DX, 0.0)
    gm, gp = oracle.p2g(x1, f.mass, c1, N, DX)
    for a in range(3):
        assert_close(np_(gn.mom[a]), gp[a], 1e-5, f"momentum {a}")
    c16 = pp.Context(N, DX, 4, coeff_format="bf16")
    with pytest.raises(pp.PolyPICError) as ei:
        pp.polypic_g2p2g(c16, g, ps, out, spill, gn, 0.0, ws)
    assert ei.value.name == "UNSUPPORTED"


def test_fused_rollout_matches_the_stepped_rollout():
    """Ten steps of sort + g2p2g + grid update against ten polypic_step calls
    from the same state (G2P, then the next step's P2G): the same grid
    velocity up to the rounding of the different sum order."""
    sc = scenes.dam_break_scene(n=32, R=27, seed=45)
    f = sc.fluid
    ctx = pp.Context(sc.n, sc.dx, 27)
    prm = pp.UpdateSettings(dt=sc.dt)
    a = pp.upload_particles(ctx, f.x, f.mass, np.zeros((3, 27, f.n), np.float32))
    b = ctx.new_particles(f.n)
    ws = ctx.workspace(f.n)
    g = ctx.new_grid()
    for _ in range(3):                          # get some motion first
        pp.polypic_step(ctx, a, b, g, prm, ws)
        a, b = b, a
    fa = ctx.new_particles(f.n)
    fa.x.copy_(a.x), fa.mass.copy_(a.mass), fa.coeff.copy_(a.coeff)
    fb = ctx.new_particles(f.n)
    spill = ctx.new_particles(f.n)
    # stepped: 10 polypic_step calls
    for _ in range(10):
        pp.polypic_step(ctx, a, b, g, prm, ws)
        a, b = b, a
    # fused: P2G + update of the start state, then 10 x (g2p2g, update) with
    # the G2P of the last step left out (it is the stepped run's 11th G2P)
    gf, gn = ctx.new_grid(), ctx.new_grid()
    pp.polypic_sort(ctx, fa, ws)
    pp.polypic_p2g(ctx, fa, gf, ws)
    pp.polypic_grid_update(ctx, gf, prm)
    for _ in range(9):
        pp.polypic_g2p2g(ctx, gf, fa, fb, spill, gn, sc.dt, ws)
        pp.polypic_grid_update(ctx, gn, prm)
        gf, gn = gn, gf
        fa, fb = fb, fa
        pp.polypic_sort(ctx, fa, ws)
    assert pp.polypic_check_device_status(ctx) == 0
    for k in range(3):
        assert_close(np_(gf.vel[k]), np_(g.vel[k]), 1e-5, f"grid velocity {k} after 10 steps")

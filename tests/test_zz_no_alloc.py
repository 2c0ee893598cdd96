"""polypic_p2g_noalloc: P2G for callers that cannot allocate device memory
while they run (an application that reserves the GPU's memory up front, or
code that must not enter an allocator where it issues the transfer).  It
uses a fixed scratch array built into the library instead of a workspace.

Its grids are checked element by element against the FP64 oracle (and
against polypic_p2g, which uses a caller workspace) on two calls in a row:
a dense scene first, then a sparse one on the same grid, so that the second
call runs on the leftovers of the first in the shared built-in array (tiles
live only in the first call must not leak into the second).  BF16 and FP16
codes are compared with the oracle fed the decoded coefficients, and a
solid phase (absorbed mass, Eq 18) goes through the same entry point.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test."""
import numpy as np
import pytest

import oracle
from paper_2308_01060_gb300 import polypic as pp
from paper_2308_01060_gb300 import scenes
from gpu_util import (assert_close, decoded, grid_from_host, np_, random_grid_velocity,
                      sorted_particles)

TOL = 1e-5
N = 32


def _dense(R, seed):
    return scenes.parity_scene(n=N, R=R, seed=seed, random_mode_init=True).fluid


def _sparse(R, seed):
    """A small ball of fluid (radius 3 cells) near one corner: few live tiles."""
    rng = np.random.default_rng(seed)
    dx = 1.0 / N
    c0 = np.array([7.3, 20.6, 9.1]) * dx
    u = rng.uniform(-1, 1, (3, 6000))
    u = u[:, np.sum(u * u, axis=0) <= 1.0]
    x = (c0[:, None] + 3 * dx * u).astype(np.float32)
    P = x.shape[1]
    mass = np.full(P, 1000.0 * dx ** 3 / 8, np.float32)
    c = scenes.random_modes(R, P, dx, rng)
    c[:, 0] = rng.normal(0, 0.5, (3, P))
    return scenes.ParticleSet(x=x, mass=mass, coeff=c.astype(np.float32), num_modes=R)


def _state(ctx, fmt, f, seed):
    """Sorted device particles in format fmt, and the FP32 coefficients the
    oracle must see: the scene's own for FP32; for the 16-bit formats the
    codes G2P writes (from a seeded grid velocity), decoded on the host."""
    if fmt == "f32":
        ps, ws = sorted_particles(ctx, f)
        return ps, ws, f.coeff, f.x, f.mass
    R = ctx.num_modes
    ps0, ws = sorted_particles(ctx, scenes.ParticleSet(x=f.x, mass=f.mass, coeff=None,
                                                       num_modes=R))
    g = grid_from_host(ctx, vel=random_grid_velocity(ctx.n, ctx.dx, seed=seed))
    ps = ctx.new_particles(ps0.count)
    pp.polypic_g2p(ctx, g, ps0, ps, 0.0, ws)        # dt = 0: positions unchanged
    pp.polypic_sort(ctx, ps, ws)
    return ps, ws, decoded(ps, R, ctx.dx), np_(ps.x), np_(ps.mass)


@pytest.mark.gpu
@pytest.mark.parametrize("R,fmt", [(27, "f32"), (8, "f32"), (27, "bf16"), (27, "f16")])
def test_noalloc_p2g_matches_oracle_on_two_calls(R, fmt):
    ctx = pp.Context((N, N, N), 1.0 / N, R, coeff_format=fmt)
    prev_live = None
    for call, f in enumerate([_dense(R, 31), _sparse(R, 32)]):
        ps, ws, coeff, x, mass = _state(ctx, fmt, f, seed=40 + call)
        g = ctx.new_grid(vel=False)
        for a in range(3):                      # the call overwrites every face
            g.mass[a].fill_(3.0)
            g.mom[a].fill_(3.0)
        pp.polypic_p2g_noalloc(ctx, ps, g)
        gm, gp = oracle.p2g(x, mass, coeff, ctx.n, ctx.dx)
        ref = ctx.new_grid(vel=False)
        pp.polypic_p2g(ctx, ps, ref, ws)
        for a in range(3):
            assert_close(np_(g.mass[a]), gm[a], TOL, f"call {call} mass {a}")
            assert_close(np_(g.mom[a]), gp[a], TOL, f"call {call} momentum {a}")
            # faces no particle reaches are exactly zero, also where the
            # previous call's tiles were live
            empty = gm[a] == 0
            assert np.all(np_(g.mass[a])[empty] == 0) and np.all(np_(g.mom[a])[empty] == 0)
            if prev_live is not None:
                assert np.any(prev_live[a] & empty)
            # the workspace entry point gives the same grids
            assert_close(np_(g.mom[a]), np_(ref.mom[a]), TOL, f"call {call} vs workspace")
        prev_live = [gm[a] != 0 for a in range(3)]
    assert pp.polypic_check_device_status(ctx) == 0


@pytest.mark.gpu
def test_noalloc_p2g_solid_phase():
    """Eq 18: the solid's weight is m_s + m_abs."""
    sc = scenes.parity_scene(n=N, R=8, seed=33, random_mode_init=True)
    f = sc.fluid
    mabs = np.random.default_rng(34).uniform(0, 2, f.n).astype(np.float32) * f.mass
    sol = scenes.ParticleSet(x=f.x, mass=f.mass, coeff=f.coeff, mass_abs=mabs, num_modes=8)
    ctx = pp.Context(sc.n, sc.dx, 8)
    ps, _ = sorted_particles(ctx, sol)
    assert ps.mass_abs is not None
    for _ in range(2):
        g = ctx.new_grid(vel=False)
        pp.polypic_p2g_noalloc(ctx, ps, g)
        gm, gp = oracle.p2g(f.x, f.mass, f.coeff, sc.n, sc.dx, mass_abs=mabs)
        for a in range(3):
            assert_close(np_(g.mass[a]), gm[a], TOL, f"mass {a}")
            assert_close(np_(g.mom[a]), gp[a], TOL, f"momentum {a}")
    assert pp.polypic_check_device_status(ctx) == 0


@pytest.mark.gpu
def test_noalloc_p2g_rejects_grids_beyond_its_scratch():
    ctx = pp.Context((128, 128, 128), 1 / 128, 4)          # 8192 tiles > 2048
    ps = ctx.new_particles(0)
    g = ctx.new_grid(vel=False)
    with pytest.raises(pp.PolyPICError) as ei:
        pp.polypic_p2g_noalloc(ctx, ps, g)
    assert ei.value.name == "WORKSPACE"

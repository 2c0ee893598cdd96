"""GPU tests of the transfer variants of the 4-mode (APIC) set against the
FP64 oracle.

  * Eq 10's gradient form of the linear modes in G2P (apic_grad_w): FP32
    coefficients and positions, and the BF16 codes through a P2G round trip;
  * Eq 12's affine map in P2G (map_affine; 4, 8 and 27 modes): momentum with
    linear modes large enough that the map changes it well beyond the
    tolerance; the identity
    fallback when det(I + dt C) vanishes; dt = 0 equal bit for bit to the
    constant map; a whole step with both variants;
  * the configurations that are not built return their documented status.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import slot_layout
from paper_2308_01060_gb300 import polypic as pp
from paper_2308_01060_gb300 import scenes
from gpu_util import assert_close, max_rel, grid_from_host, np_, random_grid_velocity, rel, sorted_particles, u32

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _scene(seed, n=32):
    return scenes.parity_scene(n=n, R=4, seed=seed, random_mode_init=False)


def _linear_heavy(f, seed, sigma_c=30.0):
    """The scene's particles with velocities ~ N(0, 0.3^2) and linear-mode
    coefficients ~ N(0, sigma_c^2) 1/s (the velocity gradient C_p)."""
    rng = np.random.default_rng(seed)
    c = np.zeros((3, 4, f.n), np.float32)
    c[:, 0] = rng.normal(0.0, 0.3, (3, f.n))
    c[:, 1:] = rng.normal(0.0, sigma_c, (3, 3, f.n))
    return scenes.ParticleSet(x=f.x, mass=f.mass, coeff=c, num_modes=4)


# ------------------------------------------------------------------ Eq 10

def test_g2p_grad_w_matches_oracle():
    sc = _scene(seed=41)
    f = sc.fluid
    ctx = pp.Context(sc.n, sc.dx, 4, apic_grad_w=True)
    ps, ws = sorted_particles(ctx, f)
    gv = random_grid_velocity(sc.n, sc.dx, seed=5)
    g = grid_from_host(ctx, vel=gv)
    out = ctx.new_particles(ps.count)
    dt = 1e-3
    pp.polypic_g2p(ctx, g, ps, out, dt, ws)
    c_or, x_or = oracle.g2p(f.x, gv, 4, sc.n, sc.dx, dt, apic_grad=True)
    c_fit, _ = oracle.g2p(f.x, gv, 4, sc.n, sc.dx, dt)
    perm = slot_layout.library_order(f.x, sc.n, sc.dx)[0]
    c_or, x_or, c_fit = c_or[:, :, perm], x_or[:, perm], c_fit[:, :, perm]
    c_gpu = np_(out.coeff).astype(np.float64)
    assert_close(c_gpu[:, 0], c_or[:, 0], TOL)
    assert_close(c_gpu[:, 1:], c_or[:, 1:], TOL)
    assert rel(c_or[:, 1:], c_fit[:, 1:]) > 100 * TOL     # the two forms differ here
    assert np.max(np.abs(np_(out.x) - x_or)) < 2e-7
    assert pp.polypic_check_device_status(ctx) == 0


def test_g2p_grad_w_16bit_round_trip():
    """BF16 codes of the gradient form, decoded by P2G, against the oracle's
    P2G of its own unquantised gradient-form coefficients."""
    sc = _scene(seed=42)
    f = sc.fluid
    ctx = pp.Context(sc.n, sc.dx, 4, coeff_format="bf16", apic_grad_w=True)
    ps, ws = sorted_particles(ctx, scenes.ParticleSet(x=f.x, mass=f.mass, coeff=None))
    gv = random_grid_velocity(sc.n, sc.dx, seed=6)
    g = grid_from_host(ctx, vel=gv)
    mid = ctx.new_particles(ps.count)
    pp.polypic_g2p(ctx, g, ps, mid, 0.0, ws)
    pp.polypic_sort(ctx, mid, ws)
    g2 = ctx.new_grid(vel=False)
    pp.polypic_p2g(ctx, mid, g2, ws)
    c_or, _ = oracle.g2p(f.x, gv, 4, sc.n, sc.dx, 0.0, apic_grad=True)
    gm, gp = oracle.p2g(f.x, f.mass, c_or, sc.n, sc.dx)
    errs = [(rel(np_(g2.mom[a]), gp[a]), max_rel(np_(g2.mom[a]), gp[a])) for a in range(3)]
    assert max(max(e) for e in errs) < 1e-3, errs
    assert pp.polypic_check_device_status(ctx) == 0


# ------------------------------------------------------------------ Eq 12

@pytest.mark.parametrize("R", [4, 8, 27])
def test_p2g_affine_map_matches_oracle(R):
    """4 modes: the linear-coefficient transform; 8 and 27: per-node
    evaluation of the mapped modes."""
    sc = scenes.parity_scene(n=32, R=R, seed=43, random_mode_init=True)
    f = sc.fluid
    c = f.coeff.copy()
    c[:, 1:4] = np.random.default_rng(1).normal(0.0, 30.0, (3, 3, f.n)).astype(np.float32)
    f = scenes.ParticleSet(x=f.x, mass=f.mass, coeff=c, num_modes=R)
    dt = 2e-3
    ctx = pp.Context(sc.n, sc.dx, R, map_affine=True)
    ps, ws = sorted_particles(ctx, f)
    g = ctx.new_grid(vel=False)
    pp.polypic_p2g_mapped(ctx, ps, g, dt, ws)
    gm, gp = oracle.p2g(f.x, f.mass, f.coeff, sc.n, sc.dx, map_affine=True, dt=dt)
    _, gp_const = oracle.p2g(f.x, f.mass, f.coeff, sc.n, sc.dx)
    for a in range(3):
        assert_close(np_(g.mass[a]), gm[a], TOL)
        assert_close(np_(g.mom[a]), gp[a], TOL)
        assert rel(gp[a], gp_const[a]) > 100 * TOL        # the map matters here
    assert pp.polypic_check_device_status(ctx) == 0


def test_p2g_affine_map_identity_where_singular():
    """Particles with C_p = -I / dt have det(I + dt C_p) = 0 (to rounding in
    FP32 and FP64 alike): both sides fall back to the identity map."""
    sc = _scene(seed=44)
    f = _linear_heavy(sc.fluid, seed=2)
    dt = 2e-3
    c = f.coeff.copy()
    sing = np.arange(0, f.n, 7)
    c[:, 1:, sing] = 0.0
    for a in range(3):
        c[a, 1 + a, sing] = np.float32(-1.0 / dt)
    f = scenes.ParticleSet(x=f.x, mass=f.mass, coeff=c, num_modes=4)
    ctx = pp.Context(sc.n, sc.dx, 4, map_affine=True)
    ps, ws = sorted_particles(ctx, f)
    g = ctx.new_grid(vel=False)
    pp.polypic_p2g_mapped(ctx, ps, g, dt, ws)
    _, gp = oracle.p2g(f.x, f.mass, f.coeff, sc.n, sc.dx, map_affine=True, dt=dt)
    for a in range(3):
        assert_close(np_(g.mom[a]), gp[a], TOL)
    assert pp.polypic_check_device_status(ctx) == 0


def test_p2g_affine_map_at_zero_dt_is_the_constant_map():
    sc = _scene(seed=45)
    f = _linear_heavy(sc.fluid, seed=3)
    c_aff = pp.Context(sc.n, sc.dx, 4, map_affine=True)
    c_con = pp.Context(sc.n, sc.dx, 4)
    pa, wa = sorted_particles(c_aff, f)
    pc, wc = sorted_particles(c_con, f)
    ga, gc = c_aff.new_grid(vel=False), c_con.new_grid(vel=False)
    pp.polypic_p2g_mapped(c_aff, pa, ga, 0.0, wa)
    pp.polypic_p2g(c_con, pc, gc, wc)
    for a in range(3):
        assert torch.equal(ga.mass[a], gc.mass[a])
        assert torch.equal(ga.mom[a], gc.mom[a])


def test_step_with_affine_map_and_grad_w():
    """One polypic_step with both variants against the oracle's P2G (mapped),
    grid update and G2P (gradient form) composed."""
    sc = _scene(seed=46)
    f = _linear_heavy(sc.fluid, seed=4, sigma_c=10.0)
    dt = 2e-3
    ctx = pp.Context(sc.n, sc.dx, 4, map_affine=True, apic_grad_w=True)
    fi, ws = sorted_particles(ctx, f)
    fo = ctx.new_particles(fi.count)
    g = ctx.new_grid()
    prm = pp.UpdateSettings(dt=dt)
    pp.polypic_step(ctx, fi, fo, g, prm, ws)
    gm, gp = oracle.p2g(f.x, f.mass, f.coeff, sc.n, sc.dx, map_affine=True, dt=dt)
    fv = oracle.grid_update(sc.n, dt, prm.gravity, gm, gp)
    for a in range(3):
        assert_close(np_(g.vel[a]), fv[a], TOL)
    c_or, x_or = oracle.g2p(f.x, fv, 4, sc.n, sc.dx, dt, apic_grad=True)
    perm = u32(fi.perm)
    assert np.array_equal(perm, slot_layout.library_order(f.x, sc.n, sc.dx)[0])
    c_gpu = np_(fo.coeff).astype(np.float64)
    assert_close(c_gpu[:, 0], c_or[:, 0, perm], TOL)
    assert_close(c_gpu[:, 1:], c_or[:, 1:, perm], 3 * TOL)
    assert np.max(np.abs(np_(fo.x) - x_or[:, perm])) < 2e-7
    assert pp.polypic_check_device_status(ctx) == 0


# ------------------------------------------------------------------ status codes

def _create_status(**kw):
    L = pp.load_library()
    cfg = pp.Config()
    for a in range(3):
        cfg.n[a] = 16
    cfg.dx = 1.0 / 16
    cfg.num_modes = kw.get("R", 4)
    cfg.coeff_format = pp.COEFF_FORMATS[kw.get("fmt", "f32")]
    cfg.map = kw.get("map", 0)
    cfg.apic_variant = kw.get("apic", 0)
    h = ctypes.c_void_p()
    st = L.polypic_create(ctypes.byref(cfg), ctypes.byref(h))
    if st == 0:
        L.polypic_destroy(h)
    return st


def test_variant_configurations_report_their_status():
    assert _create_status(R=4, map=1) == 0
    assert _create_status(R=1, map=1) == 0
    assert _create_status(R=8, map=1) == 0
    assert _create_status(R=27, map=1) == 0
    assert _create_status(R=4, apic=1) == 0
    assert _create_status(R=4, apic=1, fmt="bf16") == 0
    assert pp.STATUS_NAMES[_create_status(R=4, map=1, fmt="bf16")] == "UNSUPPORTED"
    assert pp.STATUS_NAMES[_create_status(R=8, apic=1)] == "INVALID_ARG"
    assert pp.STATUS_NAMES[_create_status(R=4, map=2)] == "INVALID_ARG"

    sc = _scene(seed=47, n=16)
    f = _linear_heavy(sc.fluid, seed=5)
    ctx = pp.Context(sc.n, sc.dx, 4, map_affine=True)
    ps, ws = sorted_particles(ctx, f)
    g = ctx.new_grid()
    with pytest.raises(pp.PolyPICError, match="INVALID_ARG|invalid"):
        pp.polypic_p2g(ctx, ps, g, ws)                    # the map needs dt
    with pytest.raises(pp.PolyPICError, match="INVALID_ARG|invalid"):
        pp.polypic_p2g_noalloc(ctx, ps, g)
    bar = ctx.new_particles(ps.count)
    with pytest.raises(pp.PolyPICError, match="UNSUPPORTED|unsupported"):
        pp.polypic_p2g_adjoint(ctx, ps, g, bar, ws)
    cg = pp.Context(sc.n, sc.dx, 4, apic_grad_w=True)
    pg, wg = sorted_particles(cg, f)
    gg = cg.new_grid()
    with pytest.raises(pp.PolyPICError, match="UNSUPPORTED|unsupported"):
        pp.polypic_g2p_adjoint(cg, gg, pg, 1e-3, cg.new_particles(pg.count), cg.new_grid(),
                               cg.new_particles(pg.count), wg)

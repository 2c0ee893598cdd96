"""GPU parity: the CUDA library (called through its C ABI) against the FP64
oracle on identical seeded inputs.

Tolerances (stated by the task for the FP32 form): grid momentum and particle
velocity within 1e-5 relative, norm-wise (||a - b|| / ||b||).  Higher-mode
coefficients are compared in the dimensionless form c dx^L (velocity units),
norm-wise, at 1e-5 as well.  The sort is compared bit-exactly.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2308_01060_gb300 import polypic as pp
from paper_2308_01060_gb300 import scenes
import slot_layout
from gpu_util import (assert_close, grid_from_host, max_rel, np_, random_grid_velocity, rel, sorted_particles,
                      u32, upload)

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _scene(n=32, R=27, seed=0, random_modes=True):
    return scenes.parity_scene(n=n, R=R, seed=seed, random_mode_init=random_modes)


# ------------------------------------------------------------------ sort

@pytest.mark.parametrize("shuffle", [False, True])
def test_sort_bit_exact(shuffle):
    sc = _scene()
    f = sc.fluid
    if shuffle:
        pr = np.random.default_rng(3).permutation(f.n)
        f = scenes.ParticleSet(x=np.ascontiguousarray(f.x[:, pr]), mass=f.mass[pr],
                               coeff=np.ascontiguousarray(f.coeff[:, :, pr]), num_modes=27)
    ctx = pp.Context(sc.n, sc.dx, 27)
    ps, _ = sorted_particles(ctx, f)
    # the method's part: every cell's particle list equals the oracle's stable one
    assert slot_layout.per_cell_lists_match(u32(ps.perm), f.x, sc.n, sc.dx)
    # the library's documented layout on top of it
    perm, cs, key = slot_layout.library_order(f.x, sc.n, sc.dx)
    assert ctx.num_keys == slot_layout.num_keys(sc.n)
    assert np.array_equal(u32(ps.key), key)
    assert np.array_equal(u32(ps.perm), perm)
    assert np.array_equal(u32(ps.cell_start), cs)
    assert pp.polypic_check_device_status(ctx) == 0


@pytest.mark.parametrize("count", [0, 1, 31, 4097, 20000])
def test_sort_ragged_and_odd_grid(count):
    n = (20, 12, 10)       # not multiples of the 8x8x4 tile
    dx = 1.0 / 20
    rng = np.random.default_rng(count)
    x = np.stack([rng.uniform(1.0, n[b] - 1.0, count) * dx for b in range(3)]).astype(np.float32)
    ctx = pp.Context(n, dx, 4)
    ps = pp.upload_particles(ctx, x, np.ones(count, np.float32))
    ws = ctx.workspace(count)
    pp.polypic_sort(ctx, ps, ws)
    assert slot_layout.per_cell_lists_match(u32(ps.perm), x, n, dx)
    perm, cs, key = slot_layout.library_order(x, n, dx)
    assert np.array_equal(u32(ps.perm), perm)
    assert np.array_equal(u32(ps.cell_start), cs)
    if count:
        assert np.array_equal(u32(ps.key), key)


@pytest.mark.parametrize("crowd", [[64, 65, 300, 5000], [70000, 1, 65]])
def test_sort_crowded_cells_bit_exact(crowd):
    """Cells above and at the per-lane selection limit (64 particles) next to
    sparse ones, in shuffled input order; 70000 particles need three 8-bit
    digit passes over the particle index, fewer than 65536 need two."""
    n = (16, 16, 8)
    dx = 1 / 16
    rng = np.random.default_rng(len(crowd))
    cells = [(3, 4, 2), (4, 4, 2), (5, 9, 3), (12, 2, 6)]
    parts = [(np.array(c)[:, None] + rng.uniform(0, 1, (3, m))) * dx for c, m in zip(cells, crowd)]
    parts.append(rng.uniform(1.0, 7.0, (3, 3000)) * dx * np.array([[2.0], [2.0], [1.0]]))
    x = np.concatenate(parts, axis=1)
    x = np.ascontiguousarray(x[:, rng.permutation(x.shape[1])]).astype(np.float32)
    ctx = pp.Context(n, dx, 1)
    ps = pp.upload_particles(ctx, x, np.ones(x.shape[1], np.float32))
    ws = ctx.workspace(x.shape[1])
    for _ in range(2):                      # the second call reuses the workspace
        pp.polypic_sort(ctx, ps, ws)
        assert slot_layout.per_cell_lists_match(u32(ps.perm), x, n, dx)
        perm, cs, _ = slot_layout.library_order(x, n, dx)
        assert np.array_equal(u32(ps.cell_start), cs)
        assert np.array_equal(u32(ps.perm), perm)
    assert pp.polypic_check_device_status(ctx) == 0


def test_sort_flags_out_of_domain():
    n = (16, 16, 16)
    dx = 1 / 16
    x = np.full((3, 40), 0.5, np.float32)
    x[1, 7] = 0.01             # below 1 dx
    ctx = pp.Context(n, dx, 1)
    ps = pp.upload_particles(ctx, x, np.ones(40, np.float32))
    ws = ctx.workspace(40)
    pp.polypic_sort(ctx, ps, ws)
    assert pp.polypic_check_device_status(ctx) == 3  # OUT_OF_DOMAIN
    assert pp.polypic_check_device_status(ctx) == 0  # cleared


# ------------------------------------------------------------------ P2G

@pytest.mark.parametrize("R", [1, 4, 8, 27])
def test_p2g_parity_and_determinism(R):
    sc = _scene(R=R, seed=1)
    f = sc.fluid
    ctx = pp.Context(sc.n, sc.dx, R)
    ps, ws = sorted_particles(ctx, f)
    g = ctx.new_grid(vel=False)
    pp.polypic_p2g(ctx, ps, g, ws)
    gm, gp = oracle.p2g(f.x, f.mass, f.coeff, sc.n, sc.dx)
    for a in range(3):
        assert_close(np_(g.mass[a]), gm[a], TOL)
        assert_close(np_(g.mom[a]), gp[a], TOL)
    g2 = ctx.new_grid(vel=False)
    pp.polypic_p2g(ctx, ps, g2, ws)
    for a in range(3):
        assert torch.equal(g.mass[a], g2.mass[a]) and torch.equal(g.mom[a], g2.mom[a])
    assert pp.polypic_check_device_status(ctx) == 0


def test_p2g_solid_absorbed_mass():
    """Eq 18: solid particles weight momentum by m_s + m_abs."""
    sc = _scene(R=8, seed=2)
    f = sc.fluid
    mabs = (np.random.default_rng(5).uniform(0, 1, f.n) * f.mass).astype(np.float32)
    solid = scenes.ParticleSet(x=f.x, mass=f.mass, coeff=f.coeff, mass_abs=mabs, num_modes=8)
    ctx = pp.Context(sc.n, sc.dx, 8)
    ps, ws = sorted_particles(ctx, solid)
    g = ctx.new_grid(vel=False)
    pp.polypic_p2g(ctx, ps, g, ws)
    gm, gp = oracle.p2g(f.x, f.mass, f.coeff, sc.n, sc.dx, mass_abs=mabs)
    for a in range(3):
        assert_close(np_(g.mass[a]), gm[a], TOL)
        assert_close(np_(g.mom[a]), gp[a], TOL)


def test_p2g_empty():
    ctx = pp.Context((16, 16, 16), 1 / 16, 27)
    ps = ctx.new_particles(0)
    ws = ctx.workspace(0)
    pp.polypic_sort(ctx, ps, ws)
    g = ctx.new_grid(vel=False)
    for a in range(3):
        g.mass[a].fill_(7.0)
        g.mom[a].fill_(7.0)
    pp.polypic_p2g(ctx, ps, g, ws)
    for a in range(3):
        assert float(g.mass[a].abs().max()) == 0.0 and float(g.mom[a].abs().max()) == 0.0


def test_p2g_single_particle_and_crowded_cell():
    n = (16, 16, 16)
    dx = 1 / 16
    rng = np.random.default_rng(9)
    x1 = np.array([[0.41], [0.52], [0.33]], np.float32)
    # 300 particles in one cell (a run longer than many 32-particle batches)
    xc = (np.array([7, 8, 6])[:, None] + rng.uniform(0, 1, (3, 300))) * dx
    x = np.concatenate([x1, xc], axis=1).astype(np.float32)
    P = x.shape[1]
    deg = scenes.mode_degrees(27)
    coeff = (rng.standard_normal((3, 27, P)) * 0.1 / dx ** deg[None, :, None]).astype(np.float32)
    mass = rng.uniform(0.5, 1.5, P).astype(np.float32)
    ctx = pp.Context(n, dx, 27)
    ps = pp.upload_particles(ctx, x, mass, coeff)
    ws = ctx.workspace(P)
    pp.polypic_sort(ctx, ps, ws)
    g = ctx.new_grid(vel=False)
    pp.polypic_p2g(ctx, ps, g, ws)
    gm, gp = oracle.p2g(x, mass, coeff, n, dx)
    for a in range(3):
        assert_close(np_(g.mass[a]), gm[a], TOL)
        assert_close(np_(g.mom[a]), gp[a], TOL)


# ------------------------------------------------------------------ grid update

def test_grid_update_parity():
    n = (24, 16, 12)
    dx = 1 / 24
    rng = np.random.default_rng(11)
    ctx = pp.Context(n, dx, 1)
    shapes = [oracle.face_shape(a, n) for a in range(3)]
    fm = [(rng.uniform(0, 2, s) * (rng.uniform(size=s) > 0.3)).astype(np.float32) for s in shapes]
    fp = [rng.standard_normal(s).astype(np.float32) for s in shapes]
    sm = [(rng.uniform(0, 2, s) * (rng.uniform(size=s) > 0.5)).astype(np.float32) for s in shapes]
    sp = [rng.standard_normal(s).astype(np.float32) for s in shapes]
    gf = grid_from_host(ctx, fm, fp)
    gs = grid_from_host(ctx, sm, sp)
    prm = pp.UpdateSettings(dt=1e-3, gravity=(0.0, -9.81, 0.0), drag_k=3.0)
    pp.polypic_grid_update(ctx, gf, prm, solid=gs)
    fv, sv = oracle.grid_update(n, 1e-3, prm.gravity, fm, fp, sm, sp, drag_k=3.0)
    for a in range(3):
        assert max_rel(np_(gf.vel[a]), fv[a]) < 1e-5
        assert max_rel(np_(gs.vel[a]), sv[a]) < 1e-5


# ------------------------------------------------------------------ G2P

@pytest.mark.parametrize("R", [1, 4, 8, 27])
def test_g2p_parity(R):
    sc = _scene(R=R, seed=4)
    f = sc.fluid
    ctx = pp.Context(sc.n, sc.dx, R)
    ps, ws = sorted_particles(ctx, f)
    gv = random_grid_velocity(sc.n, sc.dx, seed=R)
    g = grid_from_host(ctx, vel=gv)
    out = ctx.new_particles(ps.count)
    dt = 1e-3
    pp.polypic_g2p(ctx, g, ps, out, dt, ws)
    c_or, x_or = oracle.g2p(f.x, gv, R, sc.n, sc.dx, dt)
    perm = slot_layout.library_order(f.x, sc.n, sc.dx)[0]
    c_or = c_or[:, :, perm]
    x_or = x_or[:, perm]
    c_gpu = np_(out.coeff).astype(np.float64)
    deg = scenes.mode_degrees(R)
    scale = (sc.dx ** deg)[None, :, None]
    assert_close(c_gpu[:, 0], c_or[:, 0], TOL)                       # particle velocity
    assert_close(c_gpu * scale, c_or * scale, TOL)                  # all modes, c dx^L
    assert np.max(np.abs(np_(out.x) - x_or)) < 2e-7               # positions (FP32 ulp ~ 6e-8)
    assert np.array_equal(np_(out.mass), f.mass[perm])
    assert pp.polypic_check_device_status(ctx) == 0


def test_g2p_flags_non_finite_velocity():
    """A NaN on the grid reaches the particles whose stencil covers it: G2P
    latches NONFINITE in the device status (and the call itself succeeds);
    the others' coefficients stay finite."""
    sc = _scene(R=8, seed=13)
    f = sc.fluid
    ctx = pp.Context(sc.n, sc.dx, 8)
    ps, ws = sorted_particles(ctx, f)
    gv = random_grid_velocity(sc.n, sc.dx, seed=14)
    i, j, k = 8, 5, 9                                  # a face-x node inside the fluid
    gv[0][k, j, i] = np.nan
    g = grid_from_host(ctx, vel=gv)
    out = ctx.new_particles(ps.count)
    pp.polypic_g2p(ctx, g, ps, out, 1e-3, ws)
    assert pp.STATUS_NAMES[pp.polypic_check_device_status(ctx)] == "NONFINITE"
    c = np_(out.coeff)
    bad = ~np.isfinite(c).all(axis=(0, 1))
    assert 0 < bad.sum() < 0.01 * ps.count              # only the particles around the node
    assert pp.polypic_check_device_status(ctx) == 0       # reading clears the latch


def _offset_particles(ctx, count, shift, coeff_shift=None):
    """Output arrays whose first element sits `shift` 4-byte words past an
    allocation start, so that rows begin at every 16-byte phase (the 16-bit
    codes are stored in 4-byte pairs; coeff_shift, in codes, overrides)."""
    def buf(shape, dtype, sh):
        n = int(np.prod(shape))
        return torch.zeros(n + sh, dtype=dtype, device="cuda")[sh:].view(shape)

    ref = ctx.new_particles(count)
    cs = coeff_shift if coeff_shift is not None else shift * (4 // ref.coeff.element_size())
    return pp.ParticleState(
        x=buf((3, count), torch.float32, shift), mass=buf((count,), torch.float32, shift),
        coeff=buf(tuple(ref.coeff.shape), ref.coeff.dtype, cs), key=ref.key, perm=ref.perm,
        cell_start=ref.cell_start,
        scale=None if ref.scale is None else buf((count,), torch.float32, shift))


@pytest.mark.parametrize("fmt", ["f32", "bf16"])
@pytest.mark.parametrize("shift", [1, 3])
def test_g2p_output_alignment_does_not_change_results(fmt, shift):
    """G2P into output arrays at arbitrary 16-byte phases (odd particle count,
    arrays offset by `shift` elements) writes the aligned call's values bit
    for bit."""
    sc = _scene(R=27, seed=12)
    f = sc.fluid
    keep = f.n - 1 if f.n % 2 == 0 else f.n                 # odd particle count
    sub = scenes.ParticleSet(x=np.ascontiguousarray(f.x[:, :keep]), mass=f.mass[:keep],
                             coeff=None, num_modes=27)
    ctx = pp.Context(sc.n, sc.dx, 27, coeff_format=fmt)
    ps, ws = sorted_particles(ctx, sub)
    g = grid_from_host(ctx, vel=random_grid_velocity(sc.n, sc.dx, seed=31))
    ref = ctx.new_particles(ps.count)
    pp.polypic_g2p(ctx, g, ps, ref, 1e-3, ws)
    out = _offset_particles(ctx, ps.count, shift)
    pp.polypic_g2p(ctx, g, ps, out, 1e-3, ws)
    assert torch.equal(out.x, ref.x)
    assert torch.equal(out.mass, ref.mass)
    assert torch.equal(out.coeff.view(torch.int16) if fmt != "f32" else out.coeff,
                       ref.coeff.view(torch.int16) if fmt != "f32" else ref.coeff)
    if fmt != "f32":
        assert torch.equal(out.scale, ref.scale)
        # code pairs that do not start on a 4-byte boundary are refused
        bad = _offset_particles(ctx, ps.count, shift, coeff_shift=1)
        with pytest.raises(pp.PolyPICError, match="INVALID_ARG|invalid"):
            pp.polypic_g2p(ctx, g, ps, bad, 1e-3, ws)
    assert pp.polypic_check_device_status(ctx) == 0


# ------------------------------------------------------------------ full step

@pytest.mark.parametrize("R", [4, 27])
def test_step_parity(R):
    sc = _scene(R=R, seed=6, random_modes=(R == 27))
    f = sc.fluid
    ctx = pp.Context(sc.n, sc.dx, R)
    ps = upload(ctx, f)
    out = ctx.new_particles(ps.count)
    g = ctx.new_grid()
    ws = ctx.workspace(ps.count)
    prm = pp.UpdateSettings(dt=sc.dt)
    pp.polypic_step(ctx, ps, out, g, prm, ws)
    c_or, x_or, (gm, gp, gv) = oracle.step(f.x, f.mass, f.coeff, sc.n, sc.dx, sc.dt)
    perm = slot_layout.library_order(f.x, sc.n, sc.dx)[0]
    assert np.array_equal(u32(ps.perm), perm)
    for a in range(3):
        assert_close(np_(g.mom[a]), gp[a], TOL)
        assert_close(np_(g.mass[a]), gm[a], TOL)
    c_gpu = np_(out.coeff).astype(np.float64)
    c_or = c_or[:, :, perm]
    scale = (sc.dx ** scenes.mode_degrees(R))[None, :, None]
    assert_close(c_gpu[:, 0], c_or[:, 0], TOL)
    assert_close(c_gpu * scale, c_or * scale, 3 * TOL)
    assert np.max(np.abs(np_(out.x) - x_or[:, perm])) < 2e-7
    assert pp.polypic_check_device_status(ctx) == 0


def test_step_with_solid_phase_and_drag():
    sc = scenes.splash_scene(n=32, R_fluid=8, R_solid=8, sheet_verts=24)
    ctx = pp.Context(sc.n, sc.dx, 8)
    fi = upload(ctx, sc.fluid)
    si = upload(ctx, sc.solid)
    fo = ctx.new_particles(fi.count)
    so = ctx.new_particles(si.count, solid=True)
    gf, gs = ctx.new_grid(), ctx.new_grid()
    ws = ctx.workspace(fi.count, si.count)
    prm = pp.UpdateSettings(dt=sc.dt, drag_k=5.0)
    pp.polypic_step(ctx, fi, fo, gf, prm, ws, solid_in=si, solid_out=so, gs=gs)
    f, s = sc.fluid, sc.solid
    fc = f.coeff
    scf = np.zeros((3, 8, s.n))
    gm, gp = oracle.p2g(f.x, f.mass, fc, sc.n, sc.dx)
    sm, sp = oracle.p2g(s.x, s.mass, scf, sc.n, sc.dx, mass_abs=s.mass_abs)
    fv, sv = oracle.grid_update(sc.n, sc.dt, prm.gravity, gm, gp, sm, sp, drag_k=5.0)
    for a in range(3):
        assert_close(np_(gf.vel[a]), fv[a], TOL)
        assert_close(np_(gs.vel[a]), sv[a], TOL)
    cf, xf = oracle.g2p(f.x, fv, 8, sc.n, sc.dx, sc.dt)
    cs_, xs = oracle.g2p(s.x, sv, 8, sc.n, sc.dx, sc.dt)
    pf = slot_layout.library_order(f.x, sc.n, sc.dx)[0]
    psol = slot_layout.library_order(s.x, sc.n, sc.dx)[0]
    assert_close(np_(fo.coeff)[:, 0], cf[:, 0, pf], TOL)
    assert_close(np_(so.coeff)[:, 0], cs_[:, 0, psol], TOL)
    assert np.array_equal(np_(so.mass_abs), s.mass_abs[psol])


# ------------------------------------------------------------------ 16-bit coefficients

@pytest.mark.parametrize("fmt,tol", [("bf16", 1e-3), ("f16", 1e-3)])
def test_16bit_coefficients_round_trip(fmt, tol):
    """G2P writes 16-bit codes with a per-particle scale; P2G decodes them in
    FP32.  Grid momentum against the FP64 oracle fed the unquantised fit."""
    sc = _scene(R=27, seed=8)
    f = sc.fluid
    ctx = pp.Context(sc.n, sc.dx, 27, coeff_format=fmt)
    ps, ws = sorted_particles(ctx, scenes.ParticleSet(x=f.x, mass=f.mass, coeff=None))
    gv = random_grid_velocity(sc.n, sc.dx, seed=21)
    g = grid_from_host(ctx, vel=gv)
    mid = ctx.new_particles(ps.count)
    pp.polypic_g2p(ctx, g, ps, mid, 0.0, ws)
    pp.polypic_sort(ctx, mid, ws)
    g2 = ctx.new_grid(vel=False)
    pp.polypic_p2g(ctx, mid, g2, ws)
    c_or, _ = oracle.g2p(f.x, gv, 27, sc.n, sc.dx, 0.0)
    gm, gp = oracle.p2g(f.x, f.mass, c_or, sc.n, sc.dx)
    errs = [(rel(np_(g2.mom[a]), gp[a]), max_rel(np_(g2.mom[a]), gp[a])) for a in range(3)]
    assert max(max(e) for e in errs) < tol, errs
    for a in range(3):
        assert_close(np_(g2.mass[a]), gm[a], TOL)


# ------------------------------------------------------------------ projection

def test_pcg_projection_matches_oracle():
    """Multigrid-preconditioned CG with FP64 reductions on the cells holding
    fluid particles: same projected field as the oracle's FP64 solve,
    divergence-free."""
    sc = scenes.dam_break_scene(n=24, R=1, dt=1e-3)
    f = sc.fluid
    ctx = pp.Context(sc.n, sc.dx, 1)
    ps, ws = sorted_particles(ctx, scenes.ParticleSet(x=f.x, mass=f.mass, coeff=None, num_modes=1))
    gv = random_grid_velocity(sc.n, sc.dx, seed=77)
    rng = np.random.default_rng(3)
    gm = [(rng.uniform(0.5, 1.5, s)).astype(np.float32) for s in (oracle.face_shape(a, sc.n) for a in range(3))]
    gp = [(gm[a] * gv[a]).astype(np.float32) for a in range(3)]
    g = grid_from_host(ctx, mass=gm, mom=gp)
    prm = pp.UpdateSettings(dt=sc.dt, project=True, pcg_rtol=1e-6, pcg_maxiter=2000)
    pp.polypic_grid_update(ctx, g, prm, fluid_particles=ps, ws=ws)
    assert pp.polypic_check_device_status(ctx) == 0
    fv = oracle.grid_update(sc.n, sc.dt, prm.gravity, gm, gp)
    fluid = np.zeros((sc.n[2], sc.n[1], sc.n[0]), dtype=bool)
    cells = np.floor(f.x.astype(np.float32) * np.float32(1 / sc.dx)).astype(int)
    fluid[cells[2], cells[1], cells[0]] = True
    vp, _, _ = oracle.pcg_project(sc.n, sc.dx, sc.dt, 1000.0, fluid, fv, rtol=1e-10, maxiter=5000)
    for a in range(3):
        assert_close(np_(g.vel[a]), vp[a], 1e-4)
    v = [np_(g.vel[a]).astype(np.float64) for a in range(3)]
    div = (np.diff(v[0], axis=2) + np.diff(v[1], axis=1) + np.diff(v[2], axis=0)) / sc.dx
    div0 = (np.diff(fv[0], axis=2) + np.diff(fv[1], axis=1) + np.diff(fv[2], axis=0)) / sc.dx
    assert np.abs(div[fluid]).max() <= 1e-4 * np.abs(div0[fluid]).max()


@pytest.mark.parametrize("n,maxiter", [((19, 13, 11), 48), ((32, 16, 8), 48), ((512, 4, 4), 2000)])
def test_pcg_projection_odd_and_flat_grids(n, maxiter):
    """The multigrid hierarchy on grids whose sides halve to odd sizes and to
    1: the projected field against the oracle's FP64 solve (convergence
    within 48 iterations on the compact grids)."""
    dx = 1.0 / n[0]
    rng = np.random.default_rng(11)
    cells = np.stack([rng.integers(1, n[b] - 1, 4000) for b in range(3)])
    keep = cells[1] < (2 * n[1]) // 3                        # a lower slab of fluid
    x = ((cells[:, keep] + rng.uniform(0.1, 0.9, (3, keep.sum()))) * dx).astype(np.float32)
    ctx = pp.Context(n, dx, 1)
    ps, ws = sorted_particles(ctx, scenes.ParticleSet(x=x, mass=np.ones(x.shape[1], np.float32),
                                                      coeff=None, num_modes=1))
    gv = random_grid_velocity(n, dx, seed=79)
    gm = [np.ones_like(v) for v in gv]
    g = grid_from_host(ctx, mass=gm, mom=gv)
    prm = pp.UpdateSettings(dt=1e-3, project=True, pcg_rtol=1e-6, pcg_maxiter=maxiter)
    pp.polypic_grid_update(ctx, g, prm, fluid_particles=ps, ws=ws)
    assert pp.polypic_check_device_status(ctx) == 0
    fv = oracle.grid_update(n, prm.dt, prm.gravity, gm, gv)
    fluid = np.zeros((n[2], n[1], n[0]), dtype=bool)
    c32 = np.floor(x * np.float32(1 / dx)).astype(int)
    fluid[c32[2], c32[1], c32[0]] = True
    vp, _, _ = oracle.pcg_project(n, dx, prm.dt, 1000.0, fluid, fv, rtol=1e-10, maxiter=5000)
    for a in range(3):
        assert_close(np_(g.vel[a]), vp[a], 1e-4)


def test_pcg_reports_not_converged():
    sc = scenes.dam_break_scene(n=24, R=1, dt=1e-3)
    f = sc.fluid
    ctx = pp.Context(sc.n, sc.dx, 1)
    ps, ws = sorted_particles(ctx, scenes.ParticleSet(x=f.x, mass=f.mass, coeff=None, num_modes=1))
    gv = random_grid_velocity(sc.n, sc.dx, seed=78)
    g = grid_from_host(ctx, mass=[np.ones_like(v) for v in gv], mom=gv)
    prm = pp.UpdateSettings(dt=sc.dt, project=True, pcg_rtol=1e-12, pcg_maxiter=3)
    with pytest.raises(pp.PolyPICError) as ei:
        pp.polypic_grid_update(ctx, g, prm, fluid_particles=ps, ws=ws)
    assert ei.value.name == "NOT_CONVERGED"
    assert pp.polypic_check_device_status(ctx) == 5


def test_step_replays_bit_identically_from_a_cuda_graph():
    """polypic_step captured into a CUDA graph (stream-ordered, no host
    synchronisation without the projection) and replayed gives the eager
    step's results bit for bit."""
    sc = _scene(R=8, seed=17)
    f = sc.fluid
    ctx = pp.Context(sc.n, sc.dx, 8)
    prm = pp.UpdateSettings(dt=sc.dt)
    a, b = upload(ctx, f), ctx.new_particles(f.n)
    g, ws = ctx.new_grid(), ctx.workspace(f.n)
    pp.polypic_step(ctx, a, b, g, prm, ws, stream=torch.cuda.current_stream())
    torch.cuda.synchronize()
    ref_x, ref_c, ref_v = b.x.clone(), b.coeff.clone(), [v.clone() for v in g.vel]
    a2, b2 = upload(ctx, f), ctx.new_particles(f.n)
    g2 = ctx.new_grid()
    gr = torch.cuda.CUDAGraph()
    with torch.cuda.graph(gr):
        pp.polypic_step(ctx, a2, b2, g2, prm, ws, stream=torch.cuda.current_stream())
    gr.replay()
    torch.cuda.synchronize()
    assert torch.equal(b2.x, ref_x) and torch.equal(b2.coeff, ref_c)
    for k in range(3):
        assert torch.equal(g2.vel[k], ref_v[k])
    assert pp.polypic_check_device_status(ctx) == 0


def test_g2p_guard_band_matches_oracle():
    """Particles in the band where a quadratic mode degenerates (q = 1 - 4t^2
    < 2^-10, t within ~2e-4 of -1/2): on cell faces (centre grids) and cell
    centres (the face grid) along each axis in turn.  The FP32 guard decision
    and the zeroed quadratic coefficients agree with the oracle."""
    sc = _scene(R=27, seed=19)
    f = sc.fluid
    rng = np.random.default_rng(20)
    x = f.x.astype(np.float64).copy()
    n = f.n
    for axis in range(3):
        sel = rng.choice(n, n // 8, replace=False)
        cells = np.floor(x[axis, sel] / sc.dx)
        off = np.where(rng.uniform(size=sel.size) < 0.5, 1.0, 0.5) + 1e-4
        x[axis, sel] = (np.minimum(cells, sc.n[axis] - 3) + off) * sc.dx
    x = x.astype(np.float32)
    g_on = [np.count_nonzero(oracle.particle_modes(x[:, p], a, 27, sc.dx)[4])
            for p in range(0, n, 97) for a in range(3)]
    assert sum(g_on) > 0                                  # the band is populated
    fg = scenes.ParticleSet(x=x, mass=f.mass, coeff=f.coeff, num_modes=27)
    ctx = pp.Context(sc.n, sc.dx, 27)
    ps, ws = sorted_particles(ctx, fg)
    gv = random_grid_velocity(sc.n, sc.dx, seed=21)
    g = grid_from_host(ctx, vel=gv)
    out = ctx.new_particles(ps.count)
    pp.polypic_g2p(ctx, g, ps, out, 1e-3, ws)
    c_or, x_or = oracle.g2p(x, gv, 27, sc.n, sc.dx, 1e-3)
    perm = slot_layout.library_order(x, sc.n, sc.dx)[0]
    c_or, x_or = c_or[:, :, perm], x_or[:, perm]
    c_gpu = np_(out.coeff).astype(np.float64)
    scale = (sc.dx ** scenes.mode_degrees(27))[None, :, None]
    assert np.array_equal(c_gpu == 0.0, c_or == 0.0)       # the same coefficients zeroed
    assert_close(c_gpu * scale, c_or * scale, TOL)
    assert np.max(np.abs(np_(out.x) - x_or)) < 2e-7
    assert pp.polypic_check_device_status(ctx) == 0

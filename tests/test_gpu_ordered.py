"""GPU tests of ordered phases (polypic_order, polypic_step_ordered).

  * polypic_order against the oracle's grouped slot order, bit-exactly, and
    its gathered arrays against the inputs;
  * one ordered step against the FP64 oracle step (values compared through
    the particle identities that the two perms give), including particles
    that move more than a cell (the path that reads the grid directly);
  * several ordered steps, the projection, a 16-bit format and a phase with
    absorbed mass against the block-interleaved polypic_step;
  * the next order written by the step checked against the properties that
    define the grouped order, on the step's own keys.
"""
import numpy as np
import pytest

import oracle
from paper_2308_01060_gb300 import polypic as pp
from paper_2308_01060_gb300 import scenes
from gpu_util import np_, rel, u32, upload

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _ordered(ctx, host):
    """(unordered upload, ordered phase, its workspace)."""
    src = upload(ctx, host)
    dst = ctx.new_particles(src.count, solid=host.mass_abs is not None)
    ws = ctx.workspace(src.count)
    pp.polypic_order(ctx, src, dst, ws)
    return src, dst, ws


def _check_grouped_order(key, perm_prev, cs):
    """The grouped slot order's defining properties on (key, cell_start) of an
    ordered phase; the stable order inside a cell is ascending perm_prev."""
    nk = cs.shape[0] - 1
    counts = np.bincount(key.astype(np.int64), minlength=nk)
    assert np.array_equal(np.diff(cs.astype(np.int64)), counts)
    for t in range(nk // 256):
        lo, hi = cs[256 * t], cs[256 * t + 256]
        kk = key[lo:hi].astype(np.int64)
        assert np.all((kk >= 256 * t) & (kk < 256 * t + 256))
        if hi == lo:
            continue
        _, first = np.unique(kk, return_index=True)
        ranked = kk[np.sort(first)]
        q = np.minimum(counts[ranked], 31)
        assert np.all((q[:-1] > q[1:]) | ((q[:-1] == q[1:]) & (ranked[:-1] < ranked[1:])))
        rank = {int(k): i for i, k in enumerate(ranked)}
        grp = np.array([rank[int(k)] // 32 for k in kk])
        lane = np.array([rank[int(k)] % 32 for k in kk])
        assert np.all(np.diff(grp) >= 0)
        prev = perm_prev[lo:hi].astype(np.int64)
        rnd = np.zeros(hi - lo, np.int64)
        for k in np.unique(kk):
            m = np.nonzero(kk == k)[0]
            assert np.all(np.diff(prev[m]) > 0)          # stable: ascending old index
            rnd[m] = np.arange(m.size)
        for g in np.unique(grp):
            m = grp == g
            assert np.all(np.diff(rnd[m] * 32 + lane[m]) > 0)


@pytest.mark.parametrize("case", ["parity", "crowded", "odd_grid"])
def test_order_matches_oracle_bit_exactly(case):
    rng = np.random.default_rng(7)
    if case == "parity":
        sc = scenes.parity_scene(n=32, R=8, seed=3, random_mode_init=True)
        f, n, dx = sc.fluid, sc.n, sc.dx
        pr = rng.permutation(f.n)
        f = scenes.ParticleSet(x=np.ascontiguousarray(f.x[:, pr]), mass=f.mass[pr],
                               coeff=np.ascontiguousarray(f.coeff[:, :, pr]), num_modes=8)
    else:
        n = (16, 16, 8) if case == "crowded" else (20, 12, 10)
        dx = 1 / 16 if case == "crowded" else 1 / 20
        x = np.stack([rng.uniform(1.0, n[b] - 1.0, 4000) * dx for b in range(3)])
        if case == "crowded":
            x[:, :300] = (np.array([3, 4, 2])[:, None] + rng.uniform(0, 1, (3, 300))) * dx
            x[:, 300:340] = (np.array([7, 9, 5])[:, None] + rng.uniform(0, 1, (3, 40))) * dx
        x = x.astype(np.float32)
        c = (rng.standard_normal((3, 8, x.shape[1])) * 0.1).astype(np.float32)
        f = scenes.ParticleSet(x=x, mass=rng.uniform(0.5, 1.5, x.shape[1]).astype(np.float32),
                               coeff=c, num_modes=8)
    ctx = pp.Context(n, dx, 8)
    _, dst, _ = _ordered(ctx, f)
    perm, cs = oracle.ordered_particle_order(f.x, n, dx)
    assert np.array_equal(u32(dst.perm), perm)
    assert np.array_equal(u32(dst.cell_start), cs)
    assert np.array_equal(u32(dst.key), oracle.keys(f.x, n, dx)[perm])
    assert np.array_equal(np_(dst.x), f.x[:, perm])
    assert np.array_equal(np_(dst.mass), f.mass[perm])
    assert np.array_equal(np_(dst.coeff), f.coeff[:, :, perm])
    assert pp.polypic_check_device_status(ctx) == 0


def _oracle_compare(sc, f, R, dt, ordered, out, g, gravity=(0.0, -9.81, 0.0)):
    """out (slot j) against the oracle step of f (input order)."""
    c_or, x_or, (gm, gp, _) = oracle.step(f.x, f.mass, f.coeff, sc.n, sc.dx, dt, gravity)
    for a in range(3):
        assert rel(np_(g.mass[a]), gm[a]) < TOL
        assert rel(np_(g.mom[a]), gp[a]) < TOL
    ident = u32(ordered.perm)[u32(out.perm)]              # input index of out slot j
    assert np.array_equal(np.sort(ident), np.arange(f.n))
    scale = (sc.dx ** scenes.mode_degrees(R))[None, :, None]
    c_gpu = np_(out.coeff).astype(np.float64)
    assert rel(c_gpu[:, 0], c_or[:, 0, ident]) < TOL
    assert rel(c_gpu * scale, c_or[:, :, ident] * scale) < 3 * TOL
    assert np.max(np.abs(np_(out.x) - x_or[:, ident])) < 2e-7
    assert np.array_equal(np_(out.mass), f.mass[ident])
    _check_grouped_order(u32(out.key), u32(out.perm), u32(out.cell_start))


@pytest.mark.parametrize("R", [4, 27])
def test_step_ordered_matches_oracle(R):
    sc = scenes.parity_scene(n=32, R=R, seed=6, random_mode_init=(R == 27))
    f = sc.fluid
    ctx = pp.Context(sc.n, sc.dx, R)
    _, ordered, ws = _ordered(ctx, f)
    out = ctx.new_particles(f.n)
    g = ctx.new_grid()
    pp.polypic_step_ordered(ctx, ordered, out, g, pp.UpdateSettings(dt=sc.dt), ws)
    _oracle_compare(sc, f, R, sc.dt, ordered, out, g)
    assert pp.polypic_check_device_status(ctx) == 0


def test_step_ordered_particles_moving_several_cells():
    """A vortex fast enough to carry particles 2-5 cells in one step: their
    old cells lie outside the staged halo of their new tile."""
    sc = scenes.parity_scene(n=32, R=8, seed=11, random_mode_init=False)
    f = sc.fluid
    v, _ = scenes.vortex_velocity(f.x.astype(np.float64), omega=30.0)
    coeff = np.zeros((3, 8, f.n), np.float32)
    coeff[:, 0] = v.astype(np.float32)
    f = scenes.ParticleSet(x=f.x, mass=f.mass, coeff=coeff, num_modes=8)
    dt, gravity = 0.01, (0.0, 0.0, 0.0)
    ctx = pp.Context(sc.n, sc.dx, 8)
    _, ordered, ws = _ordered(ctx, f)
    out = ctx.new_particles(f.n)
    g = ctx.new_grid()
    pp.polypic_step_ordered(ctx, ordered, out, g, pp.UpdateSettings(dt=dt, gravity=gravity), ws)
    ident = u32(ordered.perm)[u32(out.perm)]
    moved = np.abs(np_(out.x) - f.x[:, ident]).max(axis=0) / sc.dx
    assert np.sum(moved > 2.0) > 100                     # the far path is exercised
    _oracle_compare(sc, f, 8, dt, ordered, out, g, gravity)


def _general_steps(ctx, f, steps, prm):
    a = upload(ctx, f)
    b = ctx.new_particles(a.count, solid=f.mass_abs is not None)
    g = ctx.new_grid()
    ws = ctx.workspace(a.count)
    ident = np.arange(f.n)
    for _ in range(steps):
        pp.polypic_step(ctx, a, b, g, prm, ws)
        ident = ident[u32(a.perm)]
        a, b = b, a
    return a, g, ident


def _ordered_steps(ctx, f, steps, prm):
    _, a, ws = _ordered(ctx, f)
    b = ctx.new_particles(a.count, solid=f.mass_abs is not None)
    g = ctx.new_grid()
    ident = u32(a.perm).astype(np.int64)
    for _ in range(steps):
        pp.polypic_step_ordered(ctx, a, b, g, prm, ws)
        ident = ident[u32(b.perm)]
        a, b = b, a
    return a, g, ident


def _inverse(ident):
    inv = np.empty(ident.size, np.int64)
    inv[ident] = np.arange(ident.size)
    return inv


@pytest.mark.parametrize("variant", ["steps", "project", "bf16", "absorbed"])
def test_step_ordered_matches_block_step(variant):
    R = 27 if variant in ("steps", "bf16") else 8
    fmt = "bf16" if variant == "bf16" else "f32"
    sc = scenes.random_velocity_scene(n=32, R=R, seed=21, sigma_v=0.3, dt=2e-3, steps=4)
    f = sc.fluid
    if variant == "absorbed":
        mabs = (np.random.default_rng(3).uniform(0, 1, f.n) * f.mass).astype(np.float32)
        f = scenes.ParticleSet(x=f.x, mass=f.mass, coeff=f.coeff, mass_abs=mabs, num_modes=R)
    if fmt != "f32":
        f = scenes.ParticleSet(x=f.x, mass=f.mass, coeff=None, num_modes=R)
    prm = pp.UpdateSettings(dt=sc.dt, project=(variant == "project"))
    steps = 3 if variant in ("steps", "bf16") else 1
    ctx = pp.Context(sc.n, sc.dx, R, coeff_format=fmt)
    a, ga, ia = _general_steps(ctx, f, steps, prm)
    b, gb, ib = _ordered_steps(ctx, f, steps, prm)
    inv_a, inv_b = _inverse(ia), _inverse(ib)
    tol = 1e-3 if fmt != "f32" else 1e-5 * steps
    for k in range(3):
        assert rel(np_(gb.vel[k]), np_(ga.vel[k])) < tol
    assert np.max(np.abs(np_(b.x)[:, inv_b] - np_(a.x)[:, inv_a])) < 1e-6
    va = np_(a.coeff.float()).astype(np.float64)[:, 0][:, inv_a]
    vb = np_(b.coeff.float()).astype(np.float64)[:, 0][:, inv_b]
    if fmt != "f32":                                     # 16-bit codes times the scale
        va = va * np_(a.scale)[inv_a][None]
        vb = vb * np_(b.scale)[inv_b][None]
    assert rel(vb, va) < tol
    if variant == "absorbed":
        assert np.array_equal(np_(b.mass_abs)[inv_b], f.mass_abs)
    assert pp.polypic_check_device_status(ctx) == 0

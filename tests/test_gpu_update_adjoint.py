"""polypic_grid_update_adjoint with the two-phase drag and the pressure
projection, through the C ABI, against the oracle's FP64 adjoint (whose
steps are each the written-out transpose, pinned by central differences of
the oracle's forward).  The GPU side takes the projection's transpose as the
forward projection of the wall-zeroed adjoint (P W is an orthogonal
projector); agreement with the oracle's literal transpose checks that
reading too."""
import numpy as np
import pytest

import oracle
from paper_2308_01060_gb300 import polypic as pp
from paper_2308_01060_gb300 import scenes
from gpu_util import assert_close, grid_from_host, np_, sorted_particles

pytestmark = pytest.mark.gpu

DT = 1e-3
G = (0.0, -9.81, 0.0)


def _random_grids(n, rng, zero_frac):
    shapes = [oracle.face_shape(a, n) for a in range(3)]
    m = [(rng.uniform(0.5, 2.0, s) * (rng.uniform(size=s) > zero_frac)).astype(np.float32)
         for s in shapes]
    p = [rng.standard_normal(s).astype(np.float32) for s in shapes]
    return m, p


@pytest.mark.parametrize("n", [(16, 16, 16), (20, 12, 10)])
def test_two_phase_drag_adjoint_matches_oracle(n):
    rng = np.random.default_rng(21)
    ctx = pp.Context(n, 1.0 / n[0], 1)
    fm, fp = _random_grids(n, rng, 0.2)
    sm, sp = _random_grids(n, rng, 0.4)
    lfv = [rng.standard_normal(a.shape).astype(np.float32) for a in fm]
    lsv = [rng.standard_normal(a.shape).astype(np.float32) for a in sm]
    K = 500.0
    prm = pp.UpdateSettings(dt=DT, drag_k=K)
    g, gs = grid_from_host(ctx, mass=fm, mom=fp), grid_from_host(ctx, mass=sm, mom=sp)
    bf, bs = grid_from_host(ctx, vel=lfv), grid_from_host(ctx, vel=lsv)
    of, os_ = ctx.new_grid(), ctx.new_grid()
    pp.polypic_grid_update_adjoint(ctx, g, prm, bf, of, solid=gs, bar_solid_out=bs,
                                   bar_solid_in=os_)
    lm, lp, lsm, lsp = oracle.grid_update_adjoint(n, fm, fp, lfv, dt=DT, gravity=G, sm=sm, sp=sp,
                                                  lsv=lsv, drag_k=K)
    for a in range(3):
        assert_close(np_(of.mom[a]), lp[a], 1e-5, f"fluid momentum adjoint {a}")
        assert_close(np_(of.mass[a]), lm[a], 1e-5, f"fluid mass adjoint {a}")
        assert_close(np_(os_.mom[a]), lsp[a], 1e-5, f"solid momentum adjoint {a}")
        assert_close(np_(os_.mass[a]), lsm[a], 1e-5, f"solid mass adjoint {a}")
        # faces holding no mass pass nothing, exactly
        assert np.all(np_(of.mom[a])[fm[a] == 0] == 0)
        assert np.all(np_(os_.mass[a])[sm[a] == 0] == 0)
    # in place: the outputs may alias the adjoint velocity's grid
    pp.polypic_grid_update_adjoint(ctx, g, prm, bf, bf, solid=gs, bar_solid_out=bs,
                                   bar_solid_in=bs)
    for a in range(3):
        assert np.array_equal(np_(bf.mom[a]), np_(of.mom[a]))
        assert np.array_equal(np_(bs.mass[a]), np_(os_.mass[a]))


def _fluid_scene(n, seed):
    """Particles in a lower block plus a lone clump: the fluid cells the
    projection runs on (cells holding particles)."""
    rng = np.random.default_rng(seed)
    dx = 1.0 / n[0]
    lo = np.array([1, 1, 1])
    hi = np.array([n[0] * 2 // 3, n[1] // 2, n[2] - 2])
    cells = np.stack([rng.integers(lo[b], hi[b], 6000) for b in range(3)])
    extra = np.array([[n[0] - 3], [n[1] - 3], [2]]) + rng.integers(0, 2, (3, 40))
    cells = np.concatenate([cells, extra], axis=1)
    x = ((cells + rng.uniform(0.05, 0.95, cells.shape)) * dx).astype(np.float32)
    fluid = np.zeros((n[2], n[1], n[0]), dtype=bool)
    c32 = np.floor(x * np.float32(1 / dx)).astype(int)
    fluid[c32[2], c32[1], c32[0]] = True
    return x, fluid


@pytest.mark.parametrize("n", [(24, 24, 24), (19, 13, 11)])
def test_projection_adjoint_matches_oracle(n):
    rng = np.random.default_rng(22)
    dx = 1.0 / n[0]
    x, fluid = _fluid_scene(n, 23)
    ctx = pp.Context(n, dx, 1)
    ps, ws = sorted_particles(ctx, scenes.ParticleSet(x=x, mass=np.ones(x.shape[1], np.float32),
                                                      coeff=None, num_modes=1))
    fm, fp = _random_grids(n, rng, 0.1)
    lfv = [rng.standard_normal(a.shape).astype(np.float32) for a in fm]
    prm = pp.UpdateSettings(dt=DT, project=True, pcg_rtol=1e-6, pcg_maxiter=2000)
    g, bf, out = grid_from_host(ctx, mass=fm, mom=fp), grid_from_host(ctx, vel=lfv), ctx.new_grid()
    pp.polypic_grid_update_adjoint(ctx, g, prm, bf, out, fluid_particles=ps, ws=ws)
    assert pp.polypic_check_device_status(ctx) == 0
    lm, lp = oracle.grid_update_adjoint(n, fm, fp, lfv, dt=DT, gravity=G, fluid=fluid,
                                        rtol=1e-10)
    unprojected = oracle.grid_update_adjoint(n, fm, fp, lfv, dt=DT, gravity=G)[1]
    for a in range(3):
        assert_close(np_(out.mom[a]), lp[a], 1e-4, f"projected momentum adjoint {a}")
        assert_close(np_(out.mass[a]), lm[a], 1e-4, f"projected mass adjoint {a}")
    # the projection changed the adjoint substantially (the check is not vacuous)
    num = sum(np.linalg.norm(lp[a] - unprojected[a]) for a in range(3))
    assert num > 0.1 * sum(np.linalg.norm(lp[a]) for a in range(3))


def test_projection_and_drag_adjoint_matches_oracle():
    n = (16, 16, 16)
    rng = np.random.default_rng(24)
    dx = 1.0 / n[0]
    x, fluid = _fluid_scene(n, 25)
    ctx = pp.Context(n, dx, 1)
    ps, ws = sorted_particles(ctx, scenes.ParticleSet(x=x, mass=np.ones(x.shape[1], np.float32),
                                                      coeff=None, num_modes=1))
    fm, fp = _random_grids(n, rng, 0.1)
    sm, sp = _random_grids(n, rng, 0.5)
    lfv = [rng.standard_normal(a.shape).astype(np.float32) for a in fm]
    lsv = [rng.standard_normal(a.shape).astype(np.float32) for a in sm]
    K = 300.0
    prm = pp.UpdateSettings(dt=DT, drag_k=K, project=True, pcg_rtol=1e-6, pcg_maxiter=2000)
    g, gs = grid_from_host(ctx, mass=fm, mom=fp), grid_from_host(ctx, mass=sm, mom=sp)
    bf, bs = grid_from_host(ctx, vel=lfv), grid_from_host(ctx, vel=lsv)
    of, os_ = ctx.new_grid(), ctx.new_grid()
    pp.polypic_grid_update_adjoint(ctx, g, prm, bf, of, solid=gs, bar_solid_out=bs,
                                   bar_solid_in=os_, fluid_particles=ps, ws=ws)
    assert pp.polypic_check_device_status(ctx) == 0
    ref = oracle.grid_update_adjoint(n, fm, fp, lfv, dt=DT, gravity=G, sm=sm, sp=sp, lsv=lsv,
                                     drag_k=K, fluid=fluid, rtol=1e-10)
    outs = [of.mass, of.mom, os_.mass, os_.mom]
    names = ["fluid mass", "fluid momentum", "solid mass", "solid momentum"]
    for r, o, nm in zip(ref, outs, names):
        for a in range(3):
            assert_close(np_(o[a]), r[a], 1e-4, f"{nm} adjoint {a}")


def test_update_adjoint_argument_checks():
    n = (16, 16, 16)
    ctx = pp.Context(n, 1.0 / 16, 1)
    g, b, o = ctx.new_grid(), ctx.new_grid(), ctx.new_grid()
    # the projection needs the fluid particles' cell_start and a workspace
    with pytest.raises(pp.PolyPICError) as ei:
        pp.polypic_grid_update_adjoint(ctx, g, pp.UpdateSettings(dt=DT, project=True), b, o)
    assert ei.value.name == "INVALID_ARG"
    # a solid grid without its adjoint grids
    with pytest.raises(pp.PolyPICError) as ei:
        pp.polypic_grid_update_adjoint(ctx, g, pp.UpdateSettings(dt=DT, drag_k=1.0), b, o,
                                       solid=ctx.new_grid())
    assert ei.value.name == "INVALID_ARG"

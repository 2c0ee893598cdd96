"""The fabric and absorption stand-ins through the C ABI against the FP64
oracle: polypic_fabric_forces (mass-spring lattice on the sheet's vertex
particles), polypic_absorb (per-cell transfer of fluid mass into m_abs), and
polypic_step_coupled (sort, absorption, forces, P2G of both phases, update
with drag and projection, G2P of both, lattice ids carried along)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2308_01060_gb300 import polypic as pp
from paper_2308_01060_gb300 import scenes
from gpu_util import assert_close, np_, u32

pytestmark = pytest.mark.gpu

N = (32, 32, 32)
DX = 1.0 / 32
FAB = dict(k_stretch=40.0, k_shear=15.0, k_bend=4.0, damping=0.02)


def _sheet(m, side, height, seed, jitter=0.15, R=4):
    """A jittered sheet (vertex + element particles) in a shuffled order with
    lattice ids, random velocities and higher modes, random absorbed mass."""
    rng = np.random.default_rng(seed)
    x, mass, nv = scenes.sheet_particles(m, side, height)
    h = side / (m - 1)
    x = (x + jitter * h * rng.standard_normal(x.shape)).astype(np.float32)
    P = x.shape[1]
    ids = np.arange(P, dtype=np.uint32)
    order = rng.permutation(P)
    x, mass, ids = np.ascontiguousarray(x[:, order]), mass[order], ids[order]
    mabs = (rng.uniform(0, 1, P) * mass).astype(np.float32)
    c = np.zeros((3, R, P), np.float32)
    c[:, 0] = rng.normal(0, 0.2, (3, P))
    c[:, 1:] = rng.normal(0, 1.0, (3, R - 1, P))
    return x, mass, mabs, c, ids, h


def test_fabric_forces_match_oracle():
    m = 48
    x, mass, mabs, c, ids, h = _sheet(m, 0.6, 0.5, seed=1)
    ctx = pp.Context(N, DX, 4)
    ps = pp.upload_particles(ctx, x, mass, c, mabs, ids=ids)
    ws = ctx.workspace(0, ps.count)
    fab = pp.FabricSettings(verts_per_side=m, rest_length=h, **FAB)
    dt = 1e-3
    pp.polypic_fabric_forces(ctx, ps, fab, dt, ws)
    got = np_(ps.coeff).astype(np.float64)
    want = oracle.fabric_forces(x, mass, c, ids, m, h, FAB["k_stretch"], FAB["k_shear"],
                                FAB["k_bend"], FAB["damping"], dt, mass_abs=mabs)
    # the velocity changes, element by element; everything else untouched
    assert_close(got[:, 0] - c[:, 0], want[:, 0] - c[:, 0], 1e-4, "dv")
    assert np.array_equal(np_(ps.coeff)[:, 1:], c[:, 1:])
    el = ids >= m * m
    assert np.array_equal(np_(ps.coeff)[:, 0, el], c[:, 0, el])
    assert np.abs(want[:, 0] - c[:, 0]).max() > 1e-3            # the forces act


def test_absorb_matches_oracle():
    rng = np.random.default_rng(2)
    fluid = scenes.dam_break_scene(n=32, R=4, seed=3).fluid
    xf = fluid.x
    fm = (fluid.mass * rng.uniform(0.5, 1.5, fluid.n)).astype(np.float32)
    x, ms, mabs, c, ids, h = _sheet(40, 0.5, 0.3, seed=4)
    ctx = pp.Context(N, DX, 4)
    pf = pp.upload_particles(ctx, xf, fm, None)
    psol = pp.upload_particles(ctx, x, ms, c, mabs, ids=ids)
    ws = ctx.workspace(pf.count, psol.count)
    pp.polypic_sort(ctx, pf, ws)
    pp.polypic_sort(ctx, psol, ws)
    fab = pp.FabricSettings(verts_per_side=40, rest_length=h, absorb_rate=20.0,
                            absorb_capacity=1.5, absorb_max_fraction=0.3)
    dt = 1e-2
    for _ in range(3):                      # three calls: the capacity starts to bind
        pp.polypic_absorb(ctx, pf, psol, fab, dt)
    fm_w, ma_w = fm.astype(np.float64), mabs.astype(np.float64)
    for _ in range(3):
        fm_w, ma_w = oracle.absorb(xf, fm_w, x, ms, ma_w, N, DX, dt, 20.0, 1.5, 0.3)
    assert_close(np_(pf.mass), fm_w, 1e-6, "fluid masses")
    assert_close(np_(psol.mass_abs), ma_w, 1e-5, "absorbed masses")
    total0 = fm.astype(np.float64).sum() + mabs.astype(np.float64).sum()
    total = np_(pf.mass).astype(np.float64).sum() + np_(psol.mass_abs).astype(np.float64).sum()
    assert abs(total - total0) <= 1e-6 * total0
    assert ma_w.sum() - mabs.sum() > 1e-3 * ms.sum()          # something was absorbed
    assert np.any(ma_w >= 1.5 * ms * (1 - 1e-9))              # and some particle is full


@pytest.mark.parametrize("project", [False, True])
def test_step_coupled_matches_oracle(project):
    R = 4
    rng = np.random.default_rng(5)
    fluid = scenes.dam_break_scene(n=32, R=R, seed=6).fluid
    xf, fm = fluid.x, fluid.mass
    cf = np.zeros((3, R, fluid.n), np.float32)
    cf[:, 0] = rng.normal(0, 0.3, (3, fluid.n))
    m = 40
    x, ms, mabs, cs, ids, h = _sheet(m, 0.5, 0.3, seed=7, R=R)
    ctx = pp.Context(N, DX, R)
    fi = pp.upload_particles(ctx, xf, fm, cf)
    fo = ctx.new_particles(fi.count)
    si = pp.upload_particles(ctx, x, ms, cs, mabs, ids=ids)
    so = ctx.new_particles(si.count, solid=True, ids=True)
    gf, gs = ctx.new_grid(), ctx.new_grid()
    ws = ctx.workspace(fi.count, si.count)
    dt, K = 1e-3, 0.05
    prm = pp.UpdateSettings(dt=dt, drag_k=K, project=project, pcg_rtol=1e-6, pcg_maxiter=2000)
    fab = pp.FabricSettings(verts_per_side=m, rest_length=h, absorb_rate=50.0,
                            absorb_capacity=2.0, absorb_max_fraction=0.3, **FAB)
    pp.polypic_step_coupled(ctx, fi, fo, si, so, gf, gs, prm, fab, ws)
    assert pp.polypic_check_device_status(ctx) == 0

    # the oracle's step in the input order
    fm2, ma2 = oracle.absorb(xf, fm, x, ms, mabs, N, DX, dt, 50.0, 2.0, 0.3)
    cs2 = oracle.fabric_forces(x, ms, cs, ids, m, h, FAB["k_stretch"], FAB["k_shear"],
                               FAB["k_bend"], FAB["damping"], dt, mass_abs=ma2)
    gm, gp = oracle.p2g(xf, fm2, cf, N, DX)
    sgm, sgp = oracle.p2g(x, ms, cs2, N, DX, mass_abs=ma2)
    gv, sv = oracle.grid_update(N, dt, prm.gravity, gm, gp, sgm, sgp, drag_k=K)
    if project:
        fl = np.zeros((N[2], N[1], N[0]), dtype=bool)
        k = np.floor(xf * np.float32(1 / DX)).astype(int)
        fl[k[2], k[1], k[0]] = True
        gv, _, _ = oracle.pcg_project(N, DX, dt, 1000.0, fl, gv, rtol=1e-10, maxiter=5000)
    for a in range(3):
        assert_close(np_(gf.vel[a]), gv[a], 1e-4 if project else 1e-5, f"fluid grid v {a}")
        assert_close(np_(gs.vel[a]), sv[a], 1e-5, f"solid grid v {a}")
    c_f, x_f = oracle.g2p(xf, gv, R, N, DX, dt)
    c_s, x_s = oracle.g2p(x, sv, R, N, DX, dt)
    pf, psl = u32(fi.perm), u32(si.perm)
    assert np.array_equal(u32(so.id), ids[psl])               # ids follow their particles
    assert_close(np_(fo.mass), fm2[pf], 1e-6, "fluid masses after absorption")
    assert_close(np_(so.mass_abs), ma2[psl], 1e-5, "absorbed masses")
    assert_close(np_(so.coeff), c_s[:, :, psl], 1e-4 if project else 1e-5, "sheet modes")
    assert_close(np_(fo.coeff), c_f[:, :, pf], 1e-4 if project else 1e-5, "fluid modes")
    assert_close(np_(so.x), x_s[:, psl], 1e-6, "sheet positions")

"""Pins of the oracle's fabric stand-in (mass-spring lattice on the sheet's
vertex particles) and absorption stand-in (per-cell transfer of fluid mass
into the solid's absorbed mass m_abs of Eqs 18-20).  The paper takes both
from Fei et al. and gives no formulas, so these pin the stated stand-ins to
physics they must obey (no force at rest, momentum conservation, force =
minus the gradient of the spring energy, dissipation by the damper, mass
conservation, the capacity) and to hand-computed values."""
import numpy as np
import pytest

import oracle

M, H = 6, 0.05


def _lattice(rng, jitter=0.0):
    """An M x M lattice at spacing H in the plane y = 0.5, its ids in a
    shuffled particle order, plus 5 element particles (ids >= M^2)."""
    k, i = np.meshgrid(np.arange(M), np.arange(M), indexing="ij")
    x = np.stack([0.3 + H * i.ravel(), np.full(M * M, 0.5), 0.3 + H * k.ravel()])
    x = x + jitter * rng.standard_normal(x.shape)
    ids = np.arange(M * M, dtype=np.uint32)
    xe = rng.uniform(0.3, 0.5, (3, 5))
    x = np.concatenate([x, xe], axis=1)
    ids = np.concatenate([ids, np.arange(M * M, M * M + 5, dtype=np.uint32)])
    order = rng.permutation(x.shape[1])
    return x[:, order], ids[order]


def _state(rng, jitter, vel=0.0, R=4):
    x, ids = _lattice(rng, jitter)
    P = x.shape[1]
    mass = rng.uniform(0.5, 1.5, P) * 1e-3
    mabs = rng.uniform(0.0, 1.0, P) * mass
    c = np.zeros((3, R, P))
    c[:, 0, :] = vel * rng.standard_normal((3, P))
    c[:, 1:, :] = rng.standard_normal((3, R - 1, P))
    return x, ids, mass, mabs, c


def _energy(x, ids, ks):
    """Spring energy sum 1/2 k (L - L0)^2 over the lattice's springs (each once)."""
    pos = np.zeros((M * M, 3))
    for p, v in enumerate(ids):
        if v < M * M:
            pos[v] = x[:, p]
    E = 0.0
    for (di, dk), k, L0 in [((1, 0), ks[0], H), ((0, 1), ks[0], H), ((1, 1), ks[1], H * 2 ** 0.5),
                            ((1, -1), ks[1], H * 2 ** 0.5), ((2, 0), ks[2], 2 * H),
                            ((0, 2), ks[2], 2 * H)]:
        for kk in range(M):
            for ii in range(M):
                i2, k2 = ii + di, kk + dk
                if 0 <= i2 < M and 0 <= k2 < M:
                    L = np.linalg.norm(pos[k2 * M + i2] - pos[kk * M + ii])
                    E += 0.5 * k * (L - L0) ** 2
    return E


def test_no_force_at_rest():
    rng = np.random.default_rng(1)
    x, ids, mass, mabs, c = _state(rng, 0.0)
    out = oracle.fabric_forces(x, mass, c, ids, M, H, 50.0, 20.0, 5.0, 0.3, 1e-3, mass_abs=mabs)
    assert np.allclose(out, c, rtol=0, atol=1e-12)


def test_forces_conserve_momentum_and_leave_elements_and_higher_modes():
    rng = np.random.default_rng(2)
    x, ids, mass, mabs, c = _state(rng, 0.01, vel=0.2)
    dt = 1e-3
    out = oracle.fabric_forces(x, mass, c, ids, M, H, 50.0, 20.0, 5.0, 0.3, dt, mass_abs=mabs)
    mt = mass + mabs
    dp = ((out[:, 0, :] - c[:, 0, :]) * mt).sum(axis=1)
    scale = (np.abs(out[:, 0, :] - c[:, 0, :]) * mt).sum()
    assert scale > 0
    assert np.all(np.abs(dp) <= 1e-12 * scale)
    el = ids >= M * M
    assert np.array_equal(out[:, :, el], c[:, :, el])
    assert np.array_equal(out[:, 1:, :], c[:, 1:, :])


@pytest.mark.parametrize("ks", [(50.0, 0.0, 0.0), (0.0, 20.0, 0.0), (0.0, 0.0, 5.0),
                                (50.0, 20.0, 5.0)])
def test_elastic_force_is_minus_the_energy_gradient(ks):
    """With no damping, m dv / dt at each vertex equals -dE/dx by central
    differences of the spring energy: each spring family alone and together
    (stiffness, rest length and sign of each)."""
    rng = np.random.default_rng(3)
    x, ids, mass, mabs, c = _state(rng, 0.01)
    dt = 1e-3
    out = oracle.fabric_forces(x, mass, c, ids, M, H, *ks, 0.0, dt, mass_abs=mabs)
    f = (out[:, 0, :] - c[:, 0, :]) * (mass + mabs) / dt
    for p in rng.choice(np.flatnonzero(ids < M * M), 8, replace=False):
        for a in range(3):
            e = 1e-7
            xp, xm = x.copy(), x.copy()
            xp[a, p] += e
            xm[a, p] -= e
            g = (_energy(xp, ids, ks) - _energy(xm, ids, ks)) / (2 * e)
            assert abs(f[a, p] + g) <= 1e-6 * (abs(g) + 1e-3 * np.abs(f).max()), (p, a, f[a, p], g)


def test_damping_dissipates_exactly_its_power():
    """Stiffness 0: sum_i m_i v_i . dv_i / dt = -c sum over springs of
    ((v_j - v_i) . e)^2 (each spring once), which is <= 0."""
    rng = np.random.default_rng(4)
    x, ids, mass, mabs, c = _state(rng, 0.01, vel=0.3)
    dt, cd = 1e-3, 0.4
    out = oracle.fabric_forces(x, mass, c, ids, M, H, 0.0, 0.0, 0.0, cd, dt, mass_abs=mabs)
    mt = mass + mabs
    power = np.sum(mt * np.sum(c[:, 0, :] * (out[:, 0, :] - c[:, 0, :]), axis=0)) / dt
    slot = {int(v): p for p, v in enumerate(ids)}
    want = 0.0
    for kk in range(M):
        for ii in range(M):
            for di, dk in [(1, 0), (0, 1), (1, 1), (1, -1), (2, 0), (0, 2)]:
                i2, k2 = ii + di, kk + dk
                if 0 <= i2 < M and 0 <= k2 < M:
                    p, q = slot[kk * M + ii], slot[k2 * M + i2]
                    d = x[:, q] - x[:, p]
                    e = d / np.linalg.norm(d)
                    want -= cd * np.dot(c[:, 0, q] - c[:, 0, p], e) ** 2
    assert want < 0
    assert abs(power - want) <= 1e-10 * abs(want)


def test_forces_do_not_depend_on_particle_order():
    rng = np.random.default_rng(5)
    x, ids, mass, mabs, c = _state(rng, 0.01, vel=0.2)
    out = oracle.fabric_forces(x, mass, c, ids, M, H, 50.0, 20.0, 5.0, 0.3, 1e-3, mass_abs=mabs)
    perm = rng.permutation(x.shape[1])
    out2 = oracle.fabric_forces(x[:, perm], mass[perm], c[:, :, perm], ids[perm], M, H, 50.0, 20.0,
                                5.0, 0.3, 1e-3, mass_abs=mabs[perm])
    assert np.allclose(out2, out[:, :, perm], rtol=1e-14, atol=1e-15)


# ------------------------------------------------------------------ absorption

N = (4, 4, 4)
DX = 0.25


def _at(cell, k, rng):
    """k FP32 positions inside cell (i, j, l)."""
    return ((np.array(cell)[:, None] + rng.uniform(0.2, 0.8, (3, k))) * DX).astype(np.float32)


def test_absorption_hand_computed_cell():
    """One cell: fluid masses 1 and 3, a solid particle of mass 1 with m_abs 0;
    rate dt = 0.5, capacity 2, at most a quarter of the cell's fluid per step:
    the solid asks 0.5, the cell gives min(0.5, 1) = 0.5, the fluid loses it
    in proportion (1 - 0.125, 3 - 0.375).  With the fluid cut to 0.4 the cell
    gives 0.1 instead, split over two solid particles by their demand."""
    rng = np.random.default_rng(6)
    xf, xs = _at((1, 1, 1), 2, rng), _at((1, 1, 1), 1, rng)
    fm, ma = oracle.absorb(xf, [1.0, 3.0], xs, [1.0], [0.0], N, DX, dt=0.5, rate=1.0, capacity=2.0,
                           max_fraction=0.25)
    assert np.allclose(fm, [0.875, 2.625], rtol=1e-15)
    assert np.allclose(ma, [0.5], rtol=1e-15)
    xs2 = _at((1, 1, 1), 2, rng)
    fm, ma = oracle.absorb(xf, [0.1, 0.3], xs2, [1.0, 3.0], [0.0, 2.9], N, DX, dt=0.5, rate=1.0,
                           capacity=1.0, max_fraction=0.25)
    # demands: min(0.5, 1) = 0.5 and min(1.5, 3 - 2.9) = 0.1; the cell gives 0.1
    assert np.allclose(ma, [0.1 * 0.5 / 0.6, 2.9 + 0.1 * 0.1 / 0.6], rtol=1e-14)
    assert np.allclose(fm, [0.1 * 0.75, 0.3 * 0.75], rtol=1e-14)


def test_absorption_needs_fluid_and_solid_in_the_same_cell():
    rng = np.random.default_rng(7)
    xf, xs = _at((1, 1, 1), 3, rng), _at((2, 1, 1), 2, rng)
    fm, ma = oracle.absorb(xf, [1.0, 1.0, 1.0], xs, [1.0, 1.0], [0.0, 0.0], N, DX, dt=0.1,
                           rate=1.0, capacity=2.0, max_fraction=0.5)
    assert np.array_equal(fm, [1.0, 1.0, 1.0]) and np.array_equal(ma, [0.0, 0.0])


def test_absorption_conserves_mass_and_respects_capacity():
    rng = np.random.default_rng(8)
    n, dx = (8, 8, 8), 1 / 8
    xf = rng.uniform(1.1 * dx, 6.9 * dx, (3, 3000)).astype(np.float32)
    xs = rng.uniform(1.1 * dx, 6.9 * dx, (3, 400)).astype(np.float32)
    fm0 = rng.uniform(0.5, 1.5, 3000)
    sm = rng.uniform(0.5, 1.5, 400)
    ma0 = rng.uniform(0.0, 1.0, 400) * sm
    fm, ma = fm0, ma0
    for _ in range(20):
        fm, ma = oracle.absorb(xf, fm, xs, sm, ma, n, dx, dt=0.05, rate=2.0, capacity=1.2,
                               max_fraction=0.3)
    total0 = fm0.sum() + ma0.sum()
    assert abs(fm.sum() + ma.sum() - total0) <= 1e-12 * total0
    assert np.all(ma <= 1.2 * sm * (1 + 1e-12)) and np.all(ma >= ma0)
    assert np.all(fm > 0) and np.all(fm <= fm0)
    assert ma.sum() - ma0.sum() > 1e-3 * total0          # something was absorbed

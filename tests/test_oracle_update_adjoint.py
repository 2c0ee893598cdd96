"""Pins of the oracle's grid-update adjoint with the two-phase drag and the
pressure projection (the adjoint of the whole update: division by mass,
gravity, implicit drag between the fluid and solid grids, walls, projection).

Each check ties the adjoint to something other than itself: central
differences of the oracle's FORWARD (grid_update, then pcg_project solved to
1e-13), reductions to the single-phase adjoint, and the projector's symmetry
(P W is an orthogonal projection, so its transpose is itself).  The random
directions touch every term, so a dropped term, a wrong sign or a swapped
phase fails one of them."""
import numpy as np
import pytest

import oracle

N = (7, 6, 5)
DT = 1e-3
G = (0.0, -9.81, 0.0)


def _grids(rng, lo, hi, zero_frac=0.0):
    out = []
    for a in range(3):
        m = rng.uniform(lo, hi, oracle.face_shape(a, N))
        if zero_frac:
            m[rng.uniform(size=m.shape) < zero_frac] = 0.0
        out.append(m)
    return out


def _normal(rng):
    return [rng.standard_normal(oracle.face_shape(a, N)) for a in range(3)]


def _fluid_mask():
    """A fluid block touching the floor and one wall, plus a lone cell; air
    elsewhere, so the Poisson problem is non-singular."""
    fl = np.zeros((N[2], N[1], N[0]), dtype=bool)
    fl[0:3, 0:4, 0:5] = True
    fl[4, 4, 5] = True
    return fl


def _forward(fm, fp, sm, sp, drag_k, fluid):
    if sm is None:
        fv = oracle.grid_update(N, DT, G, fm, fp)
        sv = None
    else:
        fv, sv = oracle.grid_update(N, DT, G, fm, fp, sm, sp, drag_k=drag_k)
    if fluid is not None:
        fv, _, _ = oracle.pcg_project(N, 1.0 / N[0], DT, 1000.0, fluid, fv, rtol=1e-13,
                                      maxiter=5000)
    return fv, sv


def _directional(fm, fp, sm, sp, drag_k, fluid, lfv, lsv, d, h=1e-6):
    """Central difference of L = <lfv, v~_f> + <lsv, v~_s> along d = (dfm, dfp,
    dsm, dsp)."""
    def L(s):
        a = [x + s * y for x, y in zip(fm, d[0])]
        b = [x + s * y for x, y in zip(fp, d[1])]
        c = None if sm is None else [x + s * y for x, y in zip(sm, d[2])]
        e = None if sm is None else [x + s * y for x, y in zip(sp, d[3])]
        fv, sv = _forward(a, b, c, e, drag_k, fluid)
        out = sum(np.sum(lfv[k] * fv[k]) for k in range(3))
        if sv is not None:
            out += sum(np.sum(lsv[k] * sv[k]) for k in range(3))
        return out
    return (L(h) - L(-h)) / (2 * h)


def _dot(adj, d):
    return sum(np.sum(x * y) for A, D in zip(adj, d) for x, y in zip(A, D))


@pytest.mark.parametrize("part", ["all", "fluid_mass", "solid_mass", "momenta"])
def test_two_phase_drag_adjoint_matches_central_differences(part):
    """Implicit drag with dt K / m ~ 0.5: the transposed 2x2 Jacobian and the
    mass derivatives (through the mean, the weights and the drag factor)
    against central differences, one group of inputs at a time."""
    rng = np.random.default_rng(11)
    fm, sm = _grids(rng, 0.5, 2.0, 0.15), _grids(rng, 0.5, 2.0, 0.15)
    fp, sp = _normal(rng), _normal(rng)
    lfv, lsv = _normal(rng), _normal(rng)
    K = 500.0
    adj = oracle.grid_update_adjoint(N, fm, fp, lfv, dt=DT, gravity=G, sm=sm, sp=sp, lsv=lsv,
                                     drag_k=K)
    lm, lp, lsm, lsp = adj
    # mass perturbations only where the mass is positive (m = 0 is a branch)
    d = [[rng.standard_normal(a.shape) * (a > 0) for a in fm], _normal(rng),
         [rng.standard_normal(a.shape) * (a > 0) for a in sm], _normal(rng)]
    zero = lambda g: [np.zeros_like(a) for a in g]
    if part == "fluid_mass":
        d = [d[0], zero(fp), zero(sm), zero(sp)]
    elif part == "solid_mass":
        d = [zero(fm), zero(fp), d[2], zero(sp)]
    elif part == "momenta":
        d = [zero(fm), d[1], zero(sm), d[3]]
    fd = _directional(fm, fp, sm, sp, K, None, lfv, lsv, d)
    an = _dot([lm, lp, lsm, lsp], d)
    assert abs(fd - an) <= 1e-7 * abs(an), (fd, an)


def test_drag_adjoint_at_zero_k_is_two_single_phase_adjoints():
    rng = np.random.default_rng(12)
    fm, sm = _grids(rng, 0.5, 2.0, 0.1), _grids(rng, 0.5, 2.0, 0.1)
    fp, sp = _normal(rng), _normal(rng)
    lfv, lsv = _normal(rng), _normal(rng)
    lm, lp, lsm, lsp = oracle.grid_update_adjoint(N, fm, fp, lfv, dt=DT, gravity=G, sm=sm,
                                                  sp=sp, lsv=lsv, drag_k=0.0)
    lm1, lp1 = oracle.grid_update_adjoint(N, fm, fp, lfv)
    lsm1, lsp1 = oracle.grid_update_adjoint(N, sm, sp, lsv)
    for a in range(3):
        assert np.array_equal(lm[a], lm1[a]) and np.array_equal(lp[a], lp1[a])
        assert np.array_equal(lsm[a], lsm1[a]) and np.array_equal(lsp[a], lsp1[a])


def test_drag_adjoint_conserves_the_mass_weighted_mean():
    """The drag keeps m_f v_f + m_s v_s on each face.  So with the adjoint
    inputs lfv = m_f l and lsv = m_s l (fixed numbers), L = sum l (m_f v_f' +
    m_s v_s') = sum l (m_f v_f + m_s v_s): the momentum adjoints are l on both
    grids, and differentiating the conservation law in m_f gives the fluid
    mass adjoint l (v_f - v_f') - l (mv)_f / m_f (likewise for the solid)."""
    rng = np.random.default_rng(13)
    fm, sm = _grids(rng, 0.5, 2.0), _grids(rng, 0.5, 2.0)
    fp, sp = _normal(rng), _normal(rng)
    l = _normal(rng)
    K = 800.0
    lfv = [fm[a] * l[a] for a in range(3)]
    lsv = [sm[a] * l[a] for a in range(3)]
    lm, lp, lsm, lsp = oracle.grid_update_adjoint(N, fm, fp, lfv, dt=DT, gravity=G, sm=sm,
                                                  sp=sp, lsv=lsv, drag_k=K)
    fv, sv = oracle.grid_update(N, DT, G, fm, fp, sm, sp, drag_k=K)
    for a in range(3):
        interior = np.ones_like(fm[a], dtype=bool)
        idx = [slice(None)] * 3
        idx[2 - a] = 0
        interior[tuple(idx)] = False
        idx[2 - a] = -1
        interior[tuple(idx)] = False
        assert np.allclose(lp[a][interior], l[a][interior], rtol=1e-12, atol=1e-12)
        assert np.allclose(lsp[a][interior], l[a][interior], rtol=1e-12, atol=1e-12)
        vf = fp[a] / fm[a] + DT * G[a]
        vs = sp[a] / sm[a] + DT * G[a]
        want_f = l[a] * (vf - fv[a]) - l[a] * fp[a] / fm[a]
        want_s = l[a] * (vs - sv[a]) - l[a] * sp[a] / sm[a]
        assert np.allclose(lm[a][interior], want_f[interior], rtol=1e-9, atol=1e-12)
        assert np.allclose(lsm[a][interior], want_s[interior], rtol=1e-9, atol=1e-12)
        # the drag does act on these faces (the check is not vacuous)
        assert np.abs((fv[a] - vf)[interior]).max() > 1e-3


def test_projection_adjoint_matches_central_differences():
    """The update followed by the projection, differentiated in the momenta
    and masses of the fluid grid: L = <lfv, P(v~)>."""
    rng = np.random.default_rng(14)
    fl = _fluid_mask()
    fm = _grids(rng, 0.5, 2.0, 0.1)
    fp, lfv = _normal(rng), _normal(rng)
    lm, lp = oracle.grid_update_adjoint(N, fm, fp, lfv, dt=DT, gravity=G, fluid=fl)
    d = [[rng.standard_normal(a.shape) * (a > 0) for a in fm], _normal(rng)]
    fd = _directional(fm, fp, None, None, 0.0, fl, lfv, None, d + [None, None])
    an = _dot([lm, lp], d)
    assert abs(fd - an) <= 1e-7 * abs(an), (fd, an)


def test_projection_adjoint_is_the_projector_itself():
    """P W (walls, then projection) is the orthogonal projection onto the
    discretely divergence-free fields on the fluid cells, hence symmetric:
    its transpose applied to w equals the forward projection of W w.  With
    unit masses and dt = 0 the update adjoint's momentum output is exactly
    that transpose."""
    rng = np.random.default_rng(15)
    fl = _fluid_mask()
    ones = [np.ones(oracle.face_shape(a, N)) for a in range(3)]
    w = _normal(rng)
    _, lp = oracle.grid_update_adjoint(N, ones, _normal(rng), w, dt=0.0, gravity=G, fluid=fl)
    ww = []
    for a in range(3):
        x = w[a].copy()
        idx = [slice(None)] * 3
        idx[2 - a] = 0
        x[tuple(idx)] = 0
        idx[2 - a] = -1
        x[tuple(idx)] = 0
        ww.append(x)
    pw, _, _ = oracle.pcg_project(N, 1.0 / N[0], 1e-3, 1000.0, fl, ww, rtol=1e-13, maxiter=5000)
    for a in range(3):
        assert np.allclose(lp[a], pw[a], rtol=0, atol=1e-10 * np.abs(pw[a]).max())
    # and it is not the identity on this mask (the solve did something)
    assert max(np.abs(pw[a] - ww[a]).max() for a in range(3)) > 1e-2


def test_projection_and_drag_adjoint_matches_central_differences():
    """The whole coupled update: two phases with drag, then the projection of
    the fluid velocity; every input perturbed at once."""
    rng = np.random.default_rng(16)
    fl = _fluid_mask()
    fm, sm = _grids(rng, 0.5, 2.0, 0.1), _grids(rng, 0.5, 2.0, 0.3)
    fp, sp = _normal(rng), _normal(rng)
    lfv, lsv = _normal(rng), _normal(rng)
    K = 300.0
    adj = oracle.grid_update_adjoint(N, fm, fp, lfv, dt=DT, gravity=G, sm=sm, sp=sp, lsv=lsv,
                                     drag_k=K, fluid=fl)
    d = [[rng.standard_normal(a.shape) * (a > 0) for a in fm], _normal(rng),
         [rng.standard_normal(a.shape) * (a > 0) for a in sm], _normal(rng)]
    fd = _directional(fm, fp, sm, sp, K, fl, lfv, lsv, d)
    an = _dot(list(adj), d)
    assert abs(fd - an) <= 1e-7 * abs(an), (fd, an)

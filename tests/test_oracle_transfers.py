"""Pins of the oracle's transfers against what the paper and the mathematics fix
(host only, no GPU).

  * stable sort == numpy's stable argsort; key layout properties
  * P2G conserves mass and linear momentum (Eqs 1-5, 13)
  * round-trips: constant / affine / multilinear / triquadratic / arbitrary
    fields are reproduced by G2P then P2G for the mode counts that span them
    (Section 3.3; the lossless claim of the abstract and Section 5)
  * N_r = 1 is PIC (Eqs 1-8) and N_r = 4 is APIC with B_p D_p^-1 (Eq 9),
    both written independently below
  * brute-force all-pairs evaluation on tiny grids
  * free fall, energy non-increase, adjoint identities, two-phase drag,
    absorbed mass (Eqs 18-20), pressure projection
"""

import numpy as np
import pytest

import oracle
from oracle import bruteforce
from paper_2308_01060_gb300 import scenes


def _safe_positions(rng, P, n, lo=3, hi=None, eps=0.06):
    """Positions whose fractional cell offset avoids the degenerate bands of
    both grid offsets (frac near 0 or near 1/2), so no guard fires."""
    hi = (n - 3) if hi is None else hi
    out = []
    while len(out) < P:
        v = rng.uniform(lo, hi, size=3)
        f = v - np.floor(v)
        if np.all((np.abs(f - 0.5) > eps) & (f > eps) & (f < 1 - eps)):
            out.append(v)
    return np.array(out).T / n


def _modes(R):
    return [oracle.mode_abc(r) for r in range(R)]


# --------------------------------------------------------------------- sort

def test_stable_sort_matches_numpy():
    rng = np.random.default_rng(0)
    n = (16, 24, 12)
    dx = 1.0 / 16
    x = np.stack([rng.uniform(0, n[b] * dx, 5000) for b in range(3)]).astype(np.float32)
    key = oracle.keys(x, n, dx)
    nc = oracle.num_cells(n)
    perm, cs = oracle.stable_sort(key, nc)
    assert np.array_equal(perm, np.argsort(key, kind="stable").astype(np.uint32))
    assert np.array_equal(cs, np.searchsorted(np.sort(key), np.arange(nc + 1)).astype(np.uint32))


def test_key_is_the_plain_cell_index():
    """The oracle's key is (k n_y + j) n_x + i of the FP32-decided cell, on a
    grid whose axes all differ, against integer arithmetic done here."""
    rng = np.random.default_rng(12)
    n = (7, 5, 6)
    dx = 1.0 / 7
    ijk = np.stack([rng.integers(0, n[b], 400) for b in range(3)])
    x = ((ijk + rng.uniform(0.05, 0.95, ijk.shape)) * dx).astype(np.float32)
    key = oracle.keys(x, n, dx)
    assert np.array_equal(key, (ijk[2] * n[1] + ijk[1]) * n[0] + ijk[0])
    perm, cs, k2 = oracle.cell_sort(x, n, dx)
    assert np.array_equal(k2, key)
    for c in range(oracle.num_cells(n)):
        members = np.flatnonzero(key == c)
        assert np.array_equal(perm[cs[c]:cs[c + 1]], members)


def test_key_uses_fp32_product():
    n = (32, 32, 32)
    dx = 1.0 / 32
    x = np.array([[np.nextafter(np.float32(0.5), np.float32(0))], [0.3], [0.3]], np.float32)
    key = oracle.keys(x, n, dx)
    i = int(np.floor(np.float32(x[0, 0] * np.float32(32.0))))
    assert i == 15                          # the FP32 product rounds below 16
    assert key[0] == (9 * 32 + 9) * 32 + i


def test_key_clamps_positions_outside_the_grid():
    """The cell is clamp(floor(x inv_dx), 0, n - 1) per axis: positions below
    0, at or beyond n dx, and NaN land in the edge cells (0 for NaN)."""
    n = (6, 5, 7)
    dx = 0.25
    inside = np.float32(2.5 * dx)
    cases = [(-0.3 * dx, 0), (-5 * dx, 0), (np.nan, 0)]
    for b in range(3):
        cases_b = cases + [(n[b] * dx, n[b] - 1), ((n[b] + 3) * dx, n[b] - 1),
                           ((n[b] - 0.5) * dx, n[b] - 1)]
        x = np.full((3, len(cases_b)), inside, np.float32)
        x[b] = np.array([c[0] for c in cases_b], np.float32)
        want = np.full((3, len(cases_b)), 2)
        want[b] = [c[1] for c in cases_b]
        key = oracle.keys(x, n, dx)
        assert np.array_equal(key, (want[2] * n[1] + want[1]) * n[0] + want[0]), b


def test_key_rounds_the_product_in_fp32_on_a_non_power_of_two_grid():
    """On a 48-cell axis, the largest FP32 position below each cell boundary
    k / 48 whose FP32 product with inv_dx = 48 rounds up to k lies in cell k,
    although the exact product is below k: the cell is the floor of the
    product rounded once in FP32, not of the exact or FP64 quotient."""
    from fractions import Fraction
    n = (48, 8, 8)
    dx = 1.0 / 48
    inv = np.float32(48.0)
    xs, ks = [], []
    for k in range(2, 47):
        x = np.float32(k / 48)
        while Fraction(float(x)) >= Fraction(k, 48):
            x = np.nextafter(x, np.float32(0))
        if np.floor(x * inv) == k:                 # FP32 product rounds up
            assert Fraction(float(x)) * 48 < k     # the exact one does not
            xs.append(x)
            ks.append(k)
    assert len(xs) >= 10
    P = len(xs)
    y, z = np.float32(4.5 / 48), np.float32(3.5 / 48)
    x = np.stack([np.array(xs, np.float32), np.full(P, y), np.full(P, z)])
    key = oracle.keys(x, n, dx)
    j, kz = int(np.floor(y * inv)), int(np.floor(z * inv))
    assert (j, kz) == (4, 3)
    assert np.array_equal(key, (kz * n[1] + j) * n[0] + np.array(ks))


# --------------------------------------------------------------------- P2G

@pytest.mark.parametrize("R", [1, 4, 8, 27])
def test_p2g_conserves_mass_and_momentum(R):
    sc = scenes.parity_scene(n=16, R=R, seed=3, random_mode_init=True)
    f = sc.fluid
    gm, gp = oracle.p2g(f.x, f.mass, f.coeff, sc.n, sc.dx)
    msum = f.mass.astype(np.float64).sum()
    for a in range(3):
        assert abs(gm[a].sum() - msum) <= 1e-13 * msum
        mom = np.dot(f.mass.astype(np.float64), f.coeff[a, 0].astype(np.float64))
        scale = np.dot(f.mass.astype(np.float64), np.abs(f.coeff[a, 0].astype(np.float64)))
        assert abs(gp[a].sum() - mom) <= 1e-12 * scale


def test_p2g_absorbed_mass_eq18_20():
    """Eq 18: solid momentum weight is m_s + m_abs; Eq 20: its velocity divides
    by the node total of (m_s + m_abs) w."""
    sc = scenes.parity_scene(n=12, R=8, seed=4, random_mode_init=True)
    f = sc.fluid
    mabs = np.random.default_rng(0).uniform(0, 2, f.n).astype(np.float32) * f.mass
    gm1, gp1 = oracle.p2g(f.x, f.mass, f.coeff, sc.n, sc.dx, mass_abs=mabs)
    gm2, gp2 = oracle.p2g(f.x, f.mass.astype(np.float64) + mabs, f.coeff, sc.n, sc.dx)
    for a in range(3):
        assert np.allclose(gm1[a], gm2[a], rtol=1e-14, atol=0)
        assert np.allclose(gp1[a], gp2[a], rtol=1e-13, atol=1e-18)
    gv = oracle.grid_update(sc.n, 0.0, (0, 0, 0), gm1, gp1)
    for a in range(3):
        sel = gm1[a] > 0
        idx = [slice(None)] * 3
        idx[2 - a] = slice(1, -1)
        inside = np.zeros_like(sel)
        inside[tuple(idx)] = True
        sel &= inside
        assert np.allclose(gv[a][sel], gp1[a][sel] / gm1[a][sel], rtol=1e-14)


def test_bruteforce_matches_stencil_oracle():
    rng = np.random.default_rng(5)
    n = (6, 6, 6)
    dx = 1 / 6
    for R in (1, 4, 8, 27):
        P = 12
        x = _safe_positions(rng, P, 6, lo=1.1, hi=4.9)
        mass = rng.uniform(0.5, 1.5, P)
        deg = scenes.mode_degrees(R)
        coeff = rng.standard_normal((3, R, P)) / (dx ** deg)[None, :, None]
        gm, gp = oracle.p2g(x, mass, coeff, n, dx)
        bm, bp = bruteforce.p2g(x, mass, coeff, n, dx, _modes(R))
        for a in range(3):
            assert np.allclose(gm[a], bm[a], rtol=1e-13, atol=1e-15)
            assert np.allclose(gp[a], bp[a], rtol=1e-12, atol=1e-12 * np.abs(bp[a]).max())
        gv = [rng.standard_normal(oracle.face_shape(a, n)) for a in range(3)]
        c, _ = oracle.g2p(x, gv, R, n, dx, 0.0)
        cb = bruteforce.g2p_fit(x, gv, n, dx, _modes(R))
        assert np.allclose(c, cb, rtol=1e-10, atol=1e-10 * np.abs(cb).max())


# --------------------------------------------------------------------- round trips

def _field(kind, rng, xf):
    """A scalar field of the given polynomial class evaluated at positions xf."""
    x, y, z = xf
    if kind == "constant":
        return np.full_like(x, rng.standard_normal())
    if kind == "affine":
        a = rng.standard_normal(4)
        return a[0] + a[1] * x + a[2] * y + a[3] * z
    if kind == "multilinear":
        a = rng.standard_normal(8)
        return sum(a[4 * i + 2 * j + k] * x ** i * y ** j * z ** k
                   for i in range(2) for j in range(2) for k in range(2))
    if kind == "triquadratic":
        a = rng.standard_normal(27)
        return sum(a[9 * i + 3 * j + k] * x ** i * y ** j * z ** k
                   for i in range(3) for j in range(3) for k in range(3))
    return rng.standard_normal(x.shape)  # arbitrary


@pytest.mark.parametrize("R,kind", [(1, "constant"), (4, "constant"), (4, "affine"),
                                    (8, "affine"), (8, "multilinear"), (27, "multilinear"),
                                    (27, "triquadratic"), (27, "arbitrary")])
def test_round_trip_reproduces_spanned_fields(R, kind):
    """G2P then P2G at fixed positions returns v~ on every face with m > 0
    whenever the field lies in the span of the first R modes (27 modes span
    every field on the 3x3x3 stencil: the lossless transfer)."""
    rng = np.random.default_rng(100 * R + ["constant", "affine", "multilinear",
                                           "triquadratic", "arbitrary"].index(kind))
    n = (10, 10, 10)
    dx = 0.1
    P = 300
    x = _safe_positions(rng, P, 10)
    mass = rng.uniform(0.5, 1.5, P)
    gv = [_field(kind, rng, scenes.face_positions(a, n, dx)) for a in range(3)]
    c, _ = oracle.g2p(x, gv, R, n, dx, 0.0)
    gm, gp = oracle.p2g(x, mass, c, n, dx)
    for a in range(3):
        m = gm[a] > 0
        v = gp[a][m] / gm[a][m]
        assert np.allclose(v, gv[a][m], rtol=1e-11, atol=1e-11 * np.abs(gv[a]).max())


def test_round_trip_fails_outside_span():
    """Control: an affine-only transfer does not reproduce a quadratic field."""
    rng = np.random.default_rng(9)
    n = (10, 10, 10)
    dx = 0.1
    x = _safe_positions(rng, 200, 10)
    mass = np.ones(200)
    gv = [_field("triquadratic", rng, scenes.face_positions(a, n, dx)) for a in range(3)]
    c, _ = oracle.g2p(x, gv, 4, n, dx, 0.0)
    gm, gp = oracle.p2g(x, mass, c, n, dx)
    m = gm[0] > 0
    assert np.max(np.abs(gp[0][m] / gm[0][m] - gv[0][m])) > 1e-4


@pytest.mark.parametrize("R", [1, 4, 8, 27])
def test_grid_energy_never_increases(R):
    rng = np.random.default_rng(20 + R)
    n = (10, 10, 10)
    dx = 0.1
    P = 400
    x = _safe_positions(rng, P, 10)
    mass = rng.uniform(0.5, 1.5, P)
    gm, _ = oracle.p2g(x, mass, np.zeros((3, R, P)), n, dx)
    gv = [rng.standard_normal(gm[a].shape) * (gm[a] > 0) for a in range(3)]
    ke0 = sum(0.5 * np.sum(gm[a] * gv[a] ** 2) for a in range(3))
    c, _ = oracle.g2p(x, gv, R, n, dx, 0.0)
    _, gp = oracle.p2g(x, mass, c, n, dx)
    ke1 = sum(0.5 * np.sum(gp[a][gm[a] > 0] ** 2 / gm[a][gm[a] > 0]) for a in range(3))
    if R == 27:
        assert abs(ke1 - ke0) <= 1e-11 * ke0
    else:
        assert ke1 <= ke0 * (1 + 1e-13)
        assert ke1 < ke0


# --------------------------------------------------------------------- PIC / APIC truncation

def _all_faces(n, dx, alpha, x):
    """Independent all-faces weights: w (P, faces), offsets (P, faces, 3)."""
    fx = np.stack([f.ravel() for f in scenes.face_positions(alpha, n, dx)], axis=1)
    d = x.T[:, None, :] - fx[None, :, :]
    w = np.prod(bruteforce.bspline2(d / dx), axis=2)
    return w, -d


def test_single_mode_is_pic():
    """N_r = 1 reduces to PIC: Eqs 1-5 for P2G and Eqs 6-8 (per component) for G2P."""
    rng = np.random.default_rng(30)
    n = (8, 8, 8)
    dx = 1 / 8
    P = 60
    x = _safe_positions(rng, P, 8)
    mass = rng.uniform(0.5, 1.5, P)
    vp = rng.standard_normal((3, P))
    gm, gp = oracle.p2g(x, mass, vp[:, None, :], n, dx)
    gv = [rng.standard_normal(oracle.face_shape(a, n)) for a in range(3)]
    c, xn = oracle.g2p(x, gv, 1, n, dx, 1e-3)
    for a in range(3):
        w, _ = _all_faces(n, dx, a, x)
        assert np.allclose(gm[a].ravel(), (mass[:, None] * w).sum(0), rtol=1e-13, atol=1e-16)
        assert np.allclose(gp[a].ravel(), (mass[:, None] * w * vp[a][:, None]).sum(0),
                           rtol=1e-12, atol=1e-14)
        v_pic = w @ gv[a].ravel()
        assert np.allclose(c[a, 0], v_pic, rtol=1e-12, atol=1e-13)
        assert np.allclose(xn[a], x[a] + 1e-3 * v_pic, rtol=0, atol=1e-15)


def test_four_modes_are_apic():
    """N_r = 4 reduces to APIC (Eq 9 / Jiang et al.): v_p = sum w v~,
    C_p = B_p D_p^-1 with B_p = sum w v~ (x_i - x_p)^T, D_p = dx^2/4 I, and
    (mv)_i = sum m w (v_p + C_p (x_i - x_p))."""
    rng = np.random.default_rng(31)
    n = (8, 8, 8)
    dx = 1 / 8
    P = 60
    x = _safe_positions(rng, P, 8)
    mass = rng.uniform(0.5, 1.5, P)
    gv = [rng.standard_normal(oracle.face_shape(a, n)) for a in range(3)]
    c, _ = oracle.g2p(x, gv, 4, n, dx, 0.0)
    for a in range(3):
        w, z = _all_faces(n, dx, a, x)
        v = w @ gv[a].ravel()
        B = np.einsum("pf,f,pfb->pb", w, gv[a].ravel(), z)
        C = B / (dx * dx / 4)
        assert np.allclose(c[a, 0], v, rtol=1e-12, atol=1e-13)
        assert np.allclose(c[a, 1:4], C.T, rtol=1e-10, atol=1e-10 * np.abs(C).max())
    gm, gp = oracle.p2g(x, mass, c, n, dx)
    for a in range(3):
        w, z = _all_faces(n, dx, a, x)
        mv = np.einsum("p,pf,pf->f", mass, w, c[a, 0][:, None] + np.einsum("bp,pfb->pf", c[a, 1:4], z))
        assert np.allclose(gp[a].ravel(), mv, rtol=1e-11, atol=1e-12 * np.abs(mv).max())


def test_apic_grad_w_reproduces_affine_and_differs_in_general():
    """Eq 10 (c = sum grad w v~) is exact for affine fields but is not the
    affine truncation for quadratic B-splines in general."""
    rng = np.random.default_rng(32)
    n = (8, 8, 8)
    dx = 1 / 8
    x = _safe_positions(rng, 40, 8)
    A = rng.standard_normal((3, 4))
    gv = [A[a, 0] + sum(A[a, 1 + b] * scenes.face_positions(a, n, dx)[b] for b in range(3))
          for a in range(3)]
    cg, _ = oracle.g2p(x, gv, 4, n, dx, 0.0, apic_grad=True)
    for a in range(3):
        assert np.allclose(cg[a, 1:4], A[a, 1:4][:, None], rtol=1e-10, atol=1e-10)
    gv = [rng.standard_normal(oracle.face_shape(a, n)) for a in range(3)]
    cg, _ = oracle.g2p(x, gv, 4, n, dx, 0.0, apic_grad=True)
    ct, _ = oracle.g2p(x, gv, 4, n, dx, 0.0)
    assert np.allclose(cg[:, 0], ct[:, 0])
    assert np.max(np.abs(cg[:, 1:] - ct[:, 1:])) > 1e-3 * np.max(np.abs(ct[:, 1:]))


# --------------------------------------------------------------------- step-level

def test_free_fall():
    """A resting block away from the walls, no projection: after one step every
    particle has c_0 = dt g exactly and no higher modes; x advances by dt^2 g."""
    n = (16, 16, 16)
    dx = 1 / 16
    rng = np.random.default_rng(40)
    cells = scenes.box_cells(n, (6, 6, 6), (10, 10, 10))
    x = scenes.seed_cells(cells, 8, dx, rng)
    P = x.shape[1]
    mass = np.full(P, 1000 * dx ** 3 / 8)
    dt = 1e-3
    g = (0.0, -9.81, 0.0)
    c, xn, _ = oracle.step(x, mass, np.zeros((3, 27, P)), n, dx, dt, g)
    for a in range(3):
        assert np.allclose(c[a, 0], dt * g[a], rtol=1e-13, atol=1e-16)
        # FP64 cancellation in sum_i w g (small d_2) leaves ~1e-11 relative residue
        assert np.max(np.abs(c[a, 1:]) * dx ** scenes.mode_degrees(27)[1:, None]) < 1e-10 * dt * 9.81
        assert np.allclose(xn[a], x[a].astype(np.float64) + dt * dt * g[a], rtol=0, atol=1e-15)


def test_advection_clamps_to_margin():
    """Particles leaving the domain are clamped to [1.5 dx, (n - 1.5) dx] per
    axis (the paper deletes them instead; a fixed count is kept here)."""
    n = (8, 8, 8)
    dx = 1 / 8
    x = np.array([[1.6 * dx, 6.4 * dx, 4.2 * dx], [4.3 * dx, 4.4 * dx, 1.55 * dx],
                  [6.3 * dx, 2.2 * dx, 4.4 * dx]])
    gv = [np.full(oracle.face_shape(a, n), s) for a, s in enumerate((-50.0, 50.0, -50.0))]
    _, xn = oracle.g2p(x, gv, 1, n, dx, 0.1)
    lo, hi = 1.5 * dx, 6.5 * dx
    assert np.all(xn >= lo - 1e-15) and np.all(xn <= hi + 1e-15)
    # velocities carry x down, y up, z down: every particle ends on a bound
    assert np.allclose(xn[0], lo) and np.allclose(xn[1], hi) and np.allclose(xn[2], lo)


def test_transfers_refuse_particles_outside_the_valid_region():
    """The valid region [dx, (n - 1) dx) per axis (decided in FP32) is where
    every 3-node stencil of every face grid lies inside that grid: at its
    lower and upper edges the stencils touch the first and last nodes, and a
    particle a little outside is refused by P2G, G2P and both adjoints."""
    n = (8, 8, 8)
    dx = 1 / 8
    for face in (0, 1):
        d = 8 + face
        lo = oracle.stencil_1d(dx, dx, face)[0]
        hi = oracle.stencil_1d(np.nextafter(np.float32(7 * dx), np.float32(0)), dx, face)[0]
        assert lo == 0 and hi + 2 == d - 1      # inside, and no room to spare
    inside = np.array([[dx, 4.5 * dx], [4.5 * dx, 4.5 * dx], [4.5 * dx, 6.9 * dx]])
    oracle.p2g(inside, np.ones(2), np.zeros((3, 1, 2)), n, dx)
    gv = [np.zeros(oracle.face_shape(a, n)) for a in range(3)]
    for bad in (0.9 * dx, 7.0 * dx, 7.05 * dx):      # the upper edge itself is outside
        for axis in range(3):
            x = np.full((3, 1), 4.5 * dx)
            x[axis, 0] = bad
            with pytest.raises(oracle.OracleError):
                oracle.p2g(x, np.ones(1), np.zeros((3, 1, 1)), n, dx)
            with pytest.raises(oracle.OracleError):
                oracle.g2p(x, gv, 1, n, dx, 0.0)
            with pytest.raises(oracle.OracleError):
                oracle.p2g_adjoint(x, np.ones(1), np.zeros((3, 1, 1)), n, dx, gv, gv)
            with pytest.raises(oracle.OracleError):
                oracle.g2p_adjoint(x, gv, 1, n, dx, 0.0, np.zeros((3, 1, 1)), np.zeros((3, 1)))


def test_empty_faces_get_zero_velocity_before_gravity():
    """Eq 5 divides only where m > 0; a face holding no mass gets v = 0, so
    after the update its velocity is dt g on interior faces and 0 on walls,
    whatever its momentum entry holds (reading 11: m > 0 exactly)."""
    rng = np.random.default_rng(42)
    n = (6, 5, 7)
    fm = [rng.uniform(0.5, 2, oracle.face_shape(a, n)) for a in range(3)]
    fp = [rng.standard_normal(oracle.face_shape(a, n)) for a in range(3)]
    empty = [rng.uniform(size=m.shape) < 0.3 for m in fm]
    for a in range(3):
        fm[a][empty[a]] = 0.0
    dt, g = 2e-3, (0.5, -9.81, 1.5)
    v = oracle.grid_update(n, dt, g, fm, fp)
    for a in range(3):
        idx = [slice(None)] * 3
        idx[2 - a] = slice(1, -1)
        inner = np.zeros(fm[a].shape, bool)
        inner[tuple(idx)] = True
        assert np.all(v[a][empty[a] & inner] == dt * g[a])
        full = ~empty[a] & inner
        assert np.allclose(v[a][full], fp[a][full] / fm[a][full] + dt * g[a], rtol=1e-15)
        assert np.all(v[a][~inner] == 0.0)


def test_two_phase_drag_solves_implicit_euler():
    rng = np.random.default_rng(41)
    n = (6, 6, 6)
    shapes = [oracle.face_shape(a, n) for a in range(3)]
    fm = [rng.uniform(0.1, 2, s) for s in shapes]
    sm = [rng.uniform(0.1, 2, s) for s in shapes]
    fp = [rng.standard_normal(s) * m for s, m in zip(shapes, fm)]
    sp = [rng.standard_normal(s) * m for s, m in zip(shapes, sm)]
    dt, K = 1e-3, 50.0
    fv, sv = oracle.grid_update(n, dt, (0, 0, 0), fm, fp, sm, sp, drag_k=K)
    for a in range(3):
        idx = [slice(None)] * 3
        idx[2 - a] = slice(1, -1)
        idx = tuple(idx)
        vf0, vs0 = fp[a] / fm[a], sp[a] / sm[a]
        rel = fv[a] - sv[a]
        # m_f (v_f' - v_f) = -dt K (v_f' - v_s'),  m_s (v_s' - v_s) = +dt K (v_f' - v_s')
        assert np.allclose((fm[a] * (fv[a] - vf0))[idx], (-dt * K * rel)[idx], rtol=1e-10, atol=1e-14)
        assert np.allclose((sm[a] * (sv[a] - vs0))[idx], (dt * K * rel)[idx], rtol=1e-10, atol=1e-14)
        # walls hold zero normal velocity
        wall = [slice(None)] * 3
        wall[2 - a] = 0
        assert np.all(fv[a][tuple(wall)] == 0) and np.all(sv[a][tuple(wall)] == 0)


# --------------------------------------------------------------------- adjoints

def _fd_setup(R, seed):
    rng = np.random.default_rng(seed)
    n = (8, 8, 8)
    dx = 1 / 8
    P = 30
    x = _safe_positions(rng, P, 8, eps=0.1)
    mass = rng.uniform(0.5, 1.5, P)
    deg = scenes.mode_degrees(R)
    coeff = rng.standard_normal((3, R, P)) / (dx ** deg)[None, :, None]
    return rng, n, dx, x, mass, coeff


@pytest.mark.parametrize("R", [1, 4, 27])
def test_p2g_adjoint_dot_product_and_position_fd(R):
    rng, n, dx, x, mass, coeff = _fd_setup(R, 50 + R)
    lm = [rng.standard_normal(oracle.face_shape(a, n)) for a in range(3)]
    lp = [rng.standard_normal(oracle.face_shape(a, n)) for a in range(3)]

    def J(xx, cc):
        gm, gp = oracle.p2g(xx, mass, cc, n, dx)
        return sum(np.sum(gm[a] * lm[a]) + np.sum(gp[a] * lp[a]) for a in range(3))

    lc, lx = oracle.p2g_adjoint(x, mass, coeff, n, dx, lm, lp)
    # linear in c: <P2G(c), lp> = <c, P2G^T lp>
    gm, gp = oracle.p2g(x, mass, coeff, n, dx)
    lhs = sum(np.sum(gp[a] * lp[a]) for a in range(3))
    assert abs(lhs - np.sum(lc * coeff)) <= 1e-12 * (abs(lhs) + np.abs(lc * coeff).sum())
    # position terms: central differences
    for _ in range(3):
        dxp = rng.standard_normal(x.shape)
        h = 1e-6 * dx
        fd = (J(x + h * dxp, coeff) - J(x - h * dxp, coeff)) / (2 * h)
        an = np.sum(lx * dxp)
        assert abs(fd - an) <= 1e-6 * max(abs(an), np.abs(lx).sum() * 1e-3)


@pytest.mark.parametrize("R", [1, 4, 27])
def test_g2p_adjoint_dot_product_and_position_fd(R):
    rng, n, dx, x, mass, _ = _fd_setup(R, 60 + R)
    dt = 2e-3
    gv = [rng.standard_normal(oracle.face_shape(a, n)) for a in range(3)]
    deg = scenes.mode_degrees(R)
    mu = rng.standard_normal((3, R, x.shape[1])) * (dx ** deg)[None, :, None]
    nu = rng.standard_normal(x.shape)

    def J(xx, vv):
        c, xo = oracle.g2p(xx, vv, R, n, dx, dt)
        return np.sum(c * mu) + np.sum(xo * nu)

    lv, lx = oracle.g2p_adjoint(x, gv, R, n, dx, dt, mu, nu)
    # linear in v~ (no clamping here): J(v) - J(0) = <v, G2P^T(mu, nu)>
    j0 = J(x, [np.zeros_like(a) for a in gv])
    lhs = J(x, gv) - j0
    rhs = sum(np.sum(lv[a] * gv[a]) for a in range(3))
    assert abs(lhs - rhs) <= 1e-11 * (abs(lhs) + 1e-30 + np.abs(rhs))
    for _ in range(3):
        dxp = rng.standard_normal(x.shape)
        h = 1e-6 * dx
        fd = (J(x + h * dxp, gv) - J(x - h * dxp, gv)) / (2 * h)
        an = np.sum(lx * dxp)
        assert abs(fd - an) <= 1e-6 * max(abs(an), np.abs(lx).sum() * 1e-3)


def test_g2p_adjoint_passes_no_gradient_through_a_clamp():
    """A particle whose advection is clamped to the margin on an axis keeps
    x' = 1.5 dx there whatever x_p and v~ are: the adjoint passes nothing
    through the advection on that axis (the fit's position terms stay),
    against central differences of the clamped forward map."""
    rng = np.random.default_rng(65)
    n = (8, 8, 8)
    dx, dt, R = 1 / 8, 2e-3, 4
    P = 10
    x = _safe_positions(rng, P, 8, eps=0.1)
    x[0] = (1 + rng.uniform(0.62, 0.88, P)) / 8          # cell 1 along x, off the guard
    gv = [rng.standard_normal(oracle.face_shape(a, n)) for a in range(3)]
    gv[0] -= 50.0                                         # x + dt v_x < 1.5 dx: clamped
    c, xo = oracle.g2p(x, gv, R, n, dx, dt)
    assert np.all(xo[0] == 1.5 * dx) and np.all(xo[1:] > 1.5 * dx)
    deg = scenes.mode_degrees(R)
    mu = rng.standard_normal((3, R, P)) * (dx ** deg)[None, :, None]
    nu = rng.standard_normal((3, P))

    def J(xx):
        cc, xx_o = oracle.g2p(xx, gv, R, n, dx, dt)
        return np.sum(cc * mu) + np.sum(xx_o * nu)

    _, lx = oracle.g2p_adjoint(x, gv, R, n, dx, dt, mu, nu)
    for _ in range(3):
        dxp = rng.standard_normal(x.shape)
        h = 1e-6 * dx
        fd = (J(x + h * dxp) - J(x - h * dxp)) / (2 * h)
        an = np.sum(lx * dxp)
        assert abs(fd - an) <= 1e-6 * max(abs(an), np.abs(lx).sum() * 1e-3)


def test_grid_update_adjoint_fd():
    rng = np.random.default_rng(70)
    n = (6, 6, 6)
    fm = [rng.uniform(0.5, 2, oracle.face_shape(a, n)) for a in range(3)]
    fm[0][2, 2, 2] = 0.0
    fp = [rng.standard_normal(oracle.face_shape(a, n)) for a in range(3)]
    lv = [rng.standard_normal(oracle.face_shape(a, n)) for a in range(3)]

    def J(m, p):
        v = oracle.grid_update(n, 1e-3, (0, -9.81, 0), m, p)
        return sum(np.sum(v[a] * lv[a]) for a in range(3))

    lm, lp = oracle.grid_update_adjoint(n, fm, fp, lv)
    dm = [rng.standard_normal(a.shape) * (a > 0) for a in fm]
    dp = [rng.standard_normal(a.shape) for a in fp]
    h = 1e-6
    fd = (J([a + h * b for a, b in zip(fm, dm)], [a + h * b for a, b in zip(fp, dp)])
          - J([a - h * b for a, b in zip(fm, dm)], [a - h * b for a, b in zip(fp, dp)])) / (2 * h)
    an = sum(np.sum(lm[a] * dm[a]) + np.sum(lp[a] * dp[a]) for a in range(3))
    assert abs(fd - an) <= 1e-7 * abs(an)


# --------------------------------------------------------------------- projection

def _laplacian_matrix(n, fluid):
    import scipy.sparse as sp
    nx, ny, nz = n
    idx = -np.ones(fluid.shape, dtype=np.int64)
    cells = np.argwhere(fluid)
    idx[tuple(cells.T)] = np.arange(len(cells))
    rows, cols, vals = [], [], []
    for r, (k, j, i) in enumerate(cells):
        nn = 0
        for dk, dj, di in [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]:
            kk, jj, ii = k + dk, j + dj, i + di
            if not (0 <= kk < nz and 0 <= jj < ny and 0 <= ii < nx):
                continue      # wall: zero normal flux
            nn += 1
            if fluid[kk, jj, ii]:
                rows.append(r); cols.append(idx[kk, jj, ii]); vals.append(-1.0)
        rows.append(r); cols.append(r); vals.append(float(nn))
    return sp.csr_matrix((vals, (rows, cols)), shape=(len(cells), len(cells))), cells


@pytest.mark.parametrize("region", ["interior", "against the walls"])
def test_pcg_projection_matches_direct_solve_and_is_divergence_free(region):
    """The interior region meets air on every side; the corner block (a dam
    break's column) rests on the floor and two side walls, where the walls
    are zero-flux (no neighbour term, no diagonal entry), not p = 0."""
    import scipy.sparse.linalg as spla
    rng = np.random.default_rng(80)
    n = (12, 10, 8)
    dx, dt, rho = 1 / 12, 1e-3, 1000.0
    fluid = np.zeros((n[2], n[1], n[0]), dtype=bool)
    if region == "interior":
        fluid[1:6, 1:8, 2:10] = True
        fluid[6, 3:5, 4:6] = True
    else:
        fluid[0:5, 0:6, 0:7] = True        # z-low, y-low (floor), x-low walls
        fluid[5, 0:2, 0:3] = True
        assert fluid[0].any() and fluid[:, 0].any() and fluid[:, :, 0].any()
    v = [rng.standard_normal(oracle.face_shape(a, n)) for a in range(3)]
    for a in range(3):       # walls carry no normal velocity
        idx = [slice(None)] * 3
        idx[2 - a] = 0
        v[a][tuple(idx)] = 0
        idx[2 - a] = -1
        v[a][tuple(idx)] = 0
    vp, p, it = oracle.pcg_project(n, dx, dt, rho, fluid, v, rtol=1e-12, maxiter=2000)
    assert it > 0
    # divergence of the projected field vanishes in every fluid cell
    div = (np.diff(vp[0], axis=2) + np.diff(vp[1], axis=1) + np.diff(vp[2], axis=0)) / dx
    div0 = (np.diff(v[0], axis=2) + np.diff(v[1], axis=1) + np.diff(v[2], axis=0)) / dx
    assert np.max(np.abs(div[fluid])) <= 1e-9 * np.max(np.abs(div0[fluid]))
    # pressure equals a direct sparse solve of the same Poisson problem
    A, cells = _laplacian_matrix(n, fluid)
    b = -(rho * dx * dx / dt) * div0[fluid]
    p_direct = spla.spsolve(A.tocsc(), b)
    assert np.allclose(p[fluid], p_direct, rtol=1e-8, atol=1e-8 * np.abs(p_direct).max())
    assert np.all(p[~fluid] == 0)
    # idempotent
    vp2, _, _ = oracle.pcg_project(n, dx, dt, rho, fluid, vp, rtol=1e-12, maxiter=2000) \
        if np.abs(div[fluid]).max() > 0 else (vp, None, None)
    for a in range(3):
        assert np.allclose(vp2[a], vp[a], rtol=0, atol=1e-8 * np.abs(vp[a]).max())


def test_affine_map_reduces_to_constant_map_at_zero_dt():
    """Eq 12: xi = x_p + (I + dt C)^-1 (x - x_p) is the identity shift at dt = 0."""
    sc = scenes.parity_scene(n=12, R=8, seed=12, random_mode_init=True)
    f = sc.fluid
    gm0, gp0 = oracle.p2g(f.x, f.mass, f.coeff, sc.n, sc.dx)
    gm1, gp1 = oracle.p2g(f.x, f.mass, f.coeff, sc.n, sc.dx, map_affine=True, dt=0.0)
    gm2, gp2 = oracle.p2g(f.x, f.mass, f.coeff, sc.n, sc.dx, map_affine=True, dt=1e-3)
    for a in range(3):
        assert np.array_equal(gm0[a], gm1[a]) and np.allclose(gp0[a], gp1[a], rtol=0, atol=0)
        assert np.array_equal(gm0[a], gm2[a])          # the map moves modes, not weights
        assert not np.allclose(gp0[a], gp2[a], rtol=1e-12, atol=0)


@pytest.mark.parametrize("R", [4, 8, 27])
def test_affine_map_matches_all_pairs_mapped_evaluation(R):
    """Eq 12: the oracle's stencil P2G with the affine map against an all-pairs
    evaluation at xi = M z, M from numpy's inverse of I + dt C_p."""
    rng = np.random.default_rng(70 + R)
    n, dx, P, dt = (6, 6, 6), 1.0 / 6, 8, 2e-3
    x = _safe_positions(rng, P, 6, lo=1.1, hi=4.9)
    mass = rng.uniform(0.5, 1.5, P)
    coeff = 0.05 * rng.standard_normal((3, R, P)) / (dx ** scenes.mode_degrees(R))[None, :, None]
    coeff[:, 1:4] = rng.normal(0.0, 40.0, (3, 3, P))          # dt C ~ 0.08: the map matters
    gm, gp = oracle.p2g(x, mass, coeff, n, dx, map_affine=True, dt=dt)
    bm, bp = bruteforce.p2g_mapped(x, mass, coeff, n, dx, _modes(R), dt)
    _, gp0 = oracle.p2g(x, mass, coeff, n, dx)
    for a in range(3):
        assert np.allclose(gm[a], bm[a], rtol=0, atol=1e-13)
        assert np.abs(gp[a] - bp[a]).max() <= 1e-11 * np.abs(bp[a]).max()
        assert np.abs(gp[a] - gp0[a]).max() > 1e-3 * np.abs(gp0[a]).max()


def test_affine_map_with_four_modes_is_a_transform_of_the_linear_coefficients():
    """With the 4-mode set, sum_r c_r s_r(M z) = c_0 + (M^T c_lin) . z: the
    mapped P2G equals the constant-map P2G of the transformed coefficients."""
    rng = np.random.default_rng(77)
    n, dx, P, dt = (8, 8, 8), 1.0 / 8, 40, 2e-3
    x = _safe_positions(rng, P, 8)
    mass = rng.uniform(0.5, 1.5, P)
    coeff = np.zeros((3, 4, P))
    coeff[:, 0] = rng.normal(0.0, 0.3, (3, P))
    coeff[:, 1:] = rng.normal(0.0, 40.0, (3, 3, P))
    ct = coeff.copy()
    for p in range(P):
        M = np.linalg.inv(np.eye(3) + dt * coeff[:, 1:, p])
        ct[:, 1:, p] = coeff[:, 1:, p] @ M                  # row a: sum_b c_{a,1+b} M_bg
    _, gp = oracle.p2g(x, mass, coeff, n, dx, map_affine=True, dt=dt)
    _, gt = oracle.p2g(x, mass, ct, n, dx)
    for a in range(3):
        assert np.abs(gp[a] - gt[a]).max() <= 1e-12 * np.abs(gt[a]).max()


def test_host_threads_give_the_serial_result():
    """The optional host threads (the all-core CPU baseline and the adjoint
    gate at full size): G2P and the P2G adjoint split independent particles,
    so their outputs are bit-identical; P2G and the G2P adjoint's grid part
    sum private grids in thread order, so they agree to FP64 rounding."""
    sc = scenes.parity_scene(n=16, R=27, seed=21, random_mode_init=True)
    f = sc.fluid
    assert oracle.get_threads() == 1
    gm1, gp1 = oracle.p2g(f.x, f.mass, f.coeff, sc.n, sc.dx)
    gv = oracle.grid_update(sc.n, sc.dt, (0.0, -9.81, 0.0), gm1, gp1)
    c1, x1 = oracle.g2p(f.x, gv, 27, sc.n, sc.dx, sc.dt)
    rng = np.random.default_rng(22)
    lc = rng.standard_normal(c1.shape)
    lxo = rng.standard_normal(x1.shape)
    lv1, lx1 = oracle.g2p_adjoint(f.x, gv, 27, sc.n, sc.dx, sc.dt, lc, lxo)
    lm = [rng.standard_normal(g.shape) for g in gm1]
    lp = [rng.standard_normal(g.shape) for g in gm1]
    la1, lxa1 = oracle.p2g_adjoint(f.x, f.mass, f.coeff, sc.n, sc.dx, lm, lp)
    try:
        oracle.set_threads(4)
        gm4, gp4 = oracle.p2g(f.x, f.mass, f.coeff, sc.n, sc.dx)
        c4, x4 = oracle.g2p(f.x, gv, 27, sc.n, sc.dx, sc.dt)
        lv4, lx4 = oracle.g2p_adjoint(f.x, gv, 27, sc.n, sc.dx, sc.dt, lc, lxo)
        la4, lxa4 = oracle.p2g_adjoint(f.x, f.mass, f.coeff, sc.n, sc.dx, lm, lp)
    finally:
        oracle.set_threads(1)
    for a in range(3):
        assert np.allclose(gm4[a], gm1[a], rtol=1e-13, atol=1e-13 * np.abs(gm1[a]).max())
        assert np.allclose(gp4[a], gp1[a], rtol=1e-13, atol=1e-13 * np.abs(gp1[a]).max())
        assert np.allclose(lv4[a], lv1[a], rtol=1e-13, atol=1e-13 * np.abs(lv1[a]).max())
    assert np.array_equal(c4, c1) and np.array_equal(x4, x1)
    assert np.array_equal(lx4, lx1) and np.array_equal(la4, la1) and np.array_equal(lxa4, lxa1)

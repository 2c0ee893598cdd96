"""Pins of the oracle's B-spline stencil and mode basis (host only).

Everything here is checked against the mathematics, not against the oracle's
own formulas: closed-form moments of the quadratic B-spline (Section 3.1),
the orthogonality the paper relies on for its decoupled fit (Section 3.3,
Eq 14) and an independent full weighted least-squares solve.
"""
import itertools

import numpy as np
import pytest

import oracle
from oracle import bruteforce


DX = 1.0 / 32


def _tq(face, xb, dx=DX):
    """t (offset from the middle node, in cells) of position xb, in FP64."""
    X = xb / dx - (0.0 if face else 0.5)
    base = np.floor(X - 0.5)
    return X - (base + 1), int(base)


@pytest.mark.parametrize("face", [True, False])
def test_weights_and_moments_closed_forms(face):
    rng = np.random.default_rng(1)
    for xb in rng.uniform(3 * DX, 20 * DX, size=200):
        base, w, z, mu2, kappa, guard = oracle.stencil_1d(xb, DX, face)
        t, b = _tq(face, xb)
        assert base == b
        # partition of unity and zero first moment of the quadratic B-spline
        assert abs(w.sum() - 1.0) < 1e-14
        assert abs(np.dot(w, z)) < 1e-14 * DX
        # second moment dx^2/4 (the constant in Eq 14) and third moment
        assert abs(mu2 - DX ** 2 / 4) < 1e-14 * DX ** 2
        assert abs(kappa - DX * t * (1 - 4 * t * t)) < 1e-13 * DX
        # node offsets z_k = (k - 1 - t) dx, nodes base..base+2
        assert np.allclose(z, (np.arange(3) - 1 - t) * DX, rtol=0, atol=1e-15)


def test_weights_special_values():
    # t = 0: particle on the middle node -> (1/8, 3/4, 1/8)
    _, w, _, _, _, _ = oracle.stencil_1d(10.5 * DX, DX, False)   # center grid: X = 10, t = 0
    assert np.allclose(w, [1 / 8, 3 / 4, 1 / 8], atol=1e-15)
    # t = 1/4 -> (1/32, 11/16, 9/32)
    _, w, _, _, _, _ = oracle.stencil_1d(10.25 * DX, DX, True)   # face grid: X = 10.25
    assert np.allclose(w, [1 / 32, 11 / 16, 9 / 32], atol=1e-15)
    # t = -1/4 -> mirror image
    _, w, _, _, _, _ = oracle.stencil_1d(9.75 * DX, DX, True)
    assert np.allclose(w, [9 / 32, 11 / 16, 1 / 32], atol=1e-15)


def test_guard_decision_is_fp32():
    # face grid, X = x/dx; the guard is q = (1-2t)(1+2t) < 2^-10 evaluated in FP32
    for xb in np.linspace(5.49 * DX, 5.5 * DX, 401):
        _, _, _, _, _, guard = oracle.stencil_1d(xb, DX, True)
        v = np.float32(np.float32(xb) * np.float32(1.0 / DX))
        base = np.floor(np.float32(v - np.float32(0.5)))
        t = np.float32(v - np.float32(base + np.float32(1.0)))
        q = np.float32(np.float32(1.0 - 2.0 * t) * np.float32(1.0 + 2.0 * t))
        assert guard == int(q < np.float32(2.0 ** -10))


def test_mode_order():
    modes = [oracle.mode_abc(r) for r in range(27)]
    assert sorted(modes) == sorted(itertools.product(range(3), repeat=3))
    assert modes[0] == (0, 0, 0)
    assert modes[1:4] == [(1, 0, 0), (0, 1, 0), (0, 0, 1)]
    # the documented order of the bilinear and trilinear modes
    assert modes[4:8] == [(1, 1, 0), (1, 0, 1), (0, 1, 1), (1, 1, 1)]
    # modes 0..7 are the 2^d multilinear ones (Section 3.3: 1 <= r <= 2^d)
    assert all(max(m) <= 1 for m in modes[:8])
    assert all(max(m) == 2 for m in modes[8:])
    # remaining triples in lexicographic order of (c, b, a)
    rest = [(m[2], m[1], m[0]) for m in modes[8:]]
    assert rest == sorted(rest)


def _particle(rng, dx=DX):
    return rng.uniform(4 * dx, 12 * dx, size=3)


@pytest.mark.parametrize("alpha", [0, 1, 2])
def test_gram_matrix_is_diagonal_with_closed_form(alpha):
    """Section 3.3: the modes are mass-orthogonal under the B-spline weights
    (multilinear ones naturally, quadratic ones after Eq 14), and
    d_r = d_a d_b d_c with d_0 = 1, d_1 = dx^2/4, d_2 = dx^4 q^2 (3 - 4t^2)/16."""
    rng = np.random.default_rng(2 + alpha)
    for _ in range(40):
        pos = _particle(rng)
        node, w, s, d, guard = oracle.particle_modes(pos, alpha, 27, DX)
        G = (s * w[:, None]).T @ s
        scale = np.sqrt(np.outer(np.diag(G), np.diag(G)))
        off = G - np.diag(np.diag(G))
        assert np.max(np.abs(off) / scale) < 1e-12
        assert np.allclose(np.diag(G), d, rtol=1e-13, atol=0)
        d1 = []
        for b in range(3):
            t, _ = _tq(b == alpha, pos[b])
            q = 1 - 4 * t * t
            d1.append([1.0, DX ** 2 / 4, DX ** 4 * q * q * (3 - 4 * t * t) / 16])
        for r in range(27):
            a, b, c = oracle.mode_abc(r)
            expect = d1[0][a] * d1[1][b] * d1[2][c]
            assert abs(d[r] - expect) <= 1e-12 * expect


@pytest.mark.parametrize("R", [1, 4, 8, 27])
def test_decoupled_fit_equals_full_least_squares(R):
    """The paper's decoupled fit c_r = <s_r, v>_w / <s_r, s_r>_w is the full
    weighted least-squares solution argmin sum_i w_i (v_i - sum_r c_r s_r)^2."""
    rng = np.random.default_rng(7)
    n = (16, 16, 16)
    for alpha in range(3):
        gv = [rng.standard_normal(oracle.face_shape(a, n)) for a in range(3)]
        for _ in range(5):
            pos = _particle(rng, 1 / 16)
            node, w, s, d, guard = oracle.particle_modes(pos, alpha, R, 1 / 16)
            assert not guard.any()
            v = np.array([gv[alpha][k, j, i] for (i, j, k) in node])
            sw = np.sqrt(w)
            c_ls, *_ = np.linalg.lstsq(s * sw[:, None], v * sw, rcond=None)
            c_or, _ = oracle.g2p(pos.reshape(3, 1), gv, R, n, 1 / 16, 0.0)
            assert np.allclose(c_or[alpha, :, 0], c_ls, rtol=1e-9, atol=1e-9 * np.abs(c_ls).max())


def test_quadratic_fit_is_second_difference():
    """Independent closed form: in 1-D the three-node weighted fit interpolates,
    so the coefficient of g (= z^2 + lower order) is the second difference
    (v0 - 2 v1 + v2) / (2 dx^2), whatever t is."""
    rng = np.random.default_rng(11)
    n = (12, 12, 12)
    dx = 1 / 12
    for _ in range(20):
        pos = rng.uniform(4 * dx, 8 * dx, size=3)
        # a field varying only along x on grid 1 (center offsets along x)
        prof = rng.standard_normal(12)
        gv = [np.zeros(oracle.face_shape(a, n)) for a in range(3)]
        gv[1][:, :, :] = prof[None, None, :]
        c, _ = oracle.g2p(pos.reshape(3, 1), gv, 27, n, dx, 0.0)
        base, _, _, _, _, guard = oracle.stencil_1d(pos[0], dx, False)
        if guard:
            continue
        r200 = [oracle.mode_abc(r) for r in range(27)].index((2, 0, 0))
        sd = (prof[base] - 2 * prof[base + 1] + prof[base + 2]) / (2 * dx * dx)
        assert abs(c[1, r200, 0] - sd) < 1e-9 * max(1.0, abs(sd))


def _guarded_position(rng, alpha, b, n, dx, delta=5e-5):
    """A position whose axis b lies in the degenerate band of face grid alpha
    (q = 1 - 4t^2 < 2^-10, t = -1/2 + delta in cells) and whose other axes sit
    well away from both bands.  Along the face axis (b == alpha, offset 0) the
    band is at the cell centre; along a centre axis (offset 1/2) at the cell
    boundary."""
    pos = np.empty(3)
    for e in range(3):
        m = rng.integers(4, n - 4)
        if e == b:
            pos[e] = (m + (0.5 if b == alpha else 1.0) + delta) * dx
        else:
            pos[e] = (m + rng.uniform(0.15, 0.35)) * dx
    return pos


@pytest.mark.parametrize("alpha", [0, 1, 2])
@pytest.mark.parametrize("b", [0, 1, 2])
def test_guard_zeroes_quadratic_modes_and_keeps_the_restricted_fit(alpha, b):
    """Reading of the degenerate quadratic mode (q = 1 - 4t^2 < 2^-10 on axis b,
    where d_2 -> 0, Section 3.3's fit being undefined in the limit): every mode
    with a quadratic factor on the guarded axis gets coefficient 0, and every
    other mode keeps the weighted least-squares fit restricted to the
    unguarded modes (an independent all-pairs evaluator and NumPy's lstsq).
    Controls: without the guard the quadratic fit is not 0, and the guard
    fires on axis b of grid alpha only."""
    n, dx = 16, 1 / 16
    ng = (n, n, n)
    rng = np.random.default_rng(100 + 3 * alpha + b)
    modes = [oracle.mode_abc(r) for r in range(27)]
    gv = [rng.standard_normal(oracle.face_shape(a, ng)) for a in range(3)]
    for _ in range(4):
        pos = _guarded_position(rng, alpha, b, n, dx)
        _, _, _, _, guard = oracle.particle_modes(pos, alpha, 27, dx)
        assert list(guard) == [int(e == b) for e in range(3)]
        c_or, _ = oracle.g2p(pos.reshape(3, 1), gv, 27, ng, dx, 0.0)
        c = c_or[alpha, :, 0]
        quad = [r for r, abc in enumerate(modes) if abc[b] == 2]
        free = [r for r, abc in enumerate(modes) if abc[b] != 2]
        assert len(quad) == 9 and np.all(c[quad] == 0.0)
        # the restricted least-squares fit over all nodes (weights > 0)
        w, s = bruteforce._particle_grid(pos, alpha, ng, dx, [modes[r] for r in free])
        m = w > 0
        sw = np.sqrt(w[m])
        A = np.stack([s[q][m] * sw for q in range(len(free))], axis=1)
        c_ls, *_ = np.linalg.lstsq(A, gv[alpha][m] * sw, rcond=None)
        assert np.allclose(c[free], c_ls, rtol=1e-9, atol=1e-9 * np.abs(c_ls).max())
        # control: the ungated decoupled fit of the guarded modes is not 0
        wq, sq = bruteforce._particle_grid(pos, alpha, ng, dx, [modes[r] for r in quad])
        num = np.tensordot(sq, wq * gv[alpha], axes=([1, 2, 3], [0, 1, 2]))
        den = np.tensordot(sq * sq, wq, axes=([1, 2, 3], [0, 1, 2]))
        scale = np.abs(gv[alpha]).max() / dx ** 2
        assert np.abs(num / den).max() > 1e-3 * scale


@pytest.mark.parametrize("alpha", [0, 1, 2])
@pytest.mark.parametrize("b", [0, 1, 2])
def test_guarded_modes_pass_no_gradient(alpha, b):
    """The G2P adjoint transposes the guard: the guarded coefficients are the
    constant 0 whatever the grid and the position, so a loss on them alone
    has zero gradient with respect to the grid velocities and the position
    (both places where the adjoint skips guarded modes are exercised).  The
    control seeds an unguarded mode and must see a non-zero gradient."""
    n, dx = 16, 1 / 16
    ng = (n, n, n)
    rng = np.random.default_rng(200 + 3 * alpha + b)
    modes = [oracle.mode_abc(r) for r in range(27)]
    gv = [rng.standard_normal(oracle.face_shape(a, ng)) for a in range(3)]
    pos = _guarded_position(rng, alpha, b, n, dx).reshape(3, 1)
    quad = [r for r, abc in enumerate(modes) if abc[b] == 2]
    lc = np.zeros((3, 27, 1))
    lc[alpha, quad, 0] = rng.standard_normal(len(quad))
    lv, lx = oracle.g2p_adjoint(pos, gv, 27, ng, dx, 0.0, lc, np.zeros((3, 1)))
    assert all(np.all(v == 0.0) for v in lv)
    assert np.all(lx == 0.0)
    free = [r for r, abc in enumerate(modes) if abc[b] != 2 and sum(abc) > 0]
    lc2 = np.zeros((3, 27, 1))
    lc2[alpha, free[0], 0] = 1.0
    lv2, lx2 = oracle.g2p_adjoint(pos, gv, 27, ng, dx, 0.0, lc2, np.zeros((3, 1)))
    assert np.abs(lv2[alpha]).max() > 0 and np.abs(lx2).max() > 0

"""All-pairs NumPy evaluator of the PolyPIC transfers -- TEST INFRASTRUCTURE ONLY.

Independent of the C oracle's stencil logic: for every particle and EVERY face
of a (tiny) grid it evaluates the quadratic B-spline N directly from the
distance (Section 3.1, w_ipa = N(x_p - x_ia)), builds the 1-D orthogonal basis
from moments summed over ALL nodes of the axis (Eq 11 with the Eq 14
substitution g = z^2 - (mu3/mu2) z - mu2), and forms

  P2G  m_ia = sum_p m_p w_ipa,  mv_ia = sum_p m_p w_ipa sum_r c_pra s_r(z)   (Eqs 1-5, 13)
  G2P  c_pra = sum_i w s_r v~_ia / sum_i w s_r^2                             (Section 3.3)

No base index, no 3x3x3 stencil, no guard: callers keep every particle away
from the degenerate band 1 - 4t^2 < 2^-10.  Mode order is passed in as a list
of (a, b, c) degree triples so that this module holds no mode table.

p2g_mapped evaluates the modes at Eq 12's mapped offsets xi = M z with
M = (I + dt C_p)^-1 from numpy's matrix inverse (C_ab = the coefficient of the
linear mode along b for component a), the per-axis basis constants from the
unmapped weights.
"""
from __future__ import annotations

import numpy as np


def bspline2(r):
    a = np.abs(r)
    return np.where(a < 0.5, 0.75 - a * a, np.where(a < 1.5, 0.5 * (1.5 - a) ** 2, 0.0))


def _axis(xb, dx, offset, nnodes):
    """Weights, offsets and basis coefficients of one particle along one axis,
    over all nodes 0..nnodes-1 of that axis."""
    nodes = np.arange(nnodes, dtype=np.float64)
    X = xb / dx - offset
    w = bspline2(X - nodes)
    z = (nodes - X) * dx
    mu2 = np.sum(w * z ** 2)
    mu3 = np.sum(w * z ** 3)
    kappa = mu3 / mu2
    f = np.stack([np.ones_like(z), z, z * z - kappa * z - mu2])
    return w, f


def _axis_moments(xb, dx, offset, nnodes):
    """Weights, node offsets z and the constants kappa, mu2 of one axis."""
    nodes = np.arange(nnodes, dtype=np.float64)
    X = xb / dx - offset
    w = bspline2(X - nodes)
    z = (nodes - X) * dx
    mu2 = np.sum(w * z ** 2)
    return w, z, np.sum(w * z ** 3) / mu2, mu2


def p2g_mapped(x, mass, coeff, n, dx, modes, dt):
    """P2G with the modes of particle p evaluated at xi = M_p z for every node."""
    x = np.asarray(x, dtype=np.float64)
    coeff = np.asarray(coeff, dtype=np.float64)
    P = x.shape[1]
    lin = {(1, 0, 0): 0, (0, 1, 0): 1, (0, 0, 1): 2}
    gm, gp = [], []
    for alpha in range(3):
        dims = [int(n[b]) + (1 if b == alpha else 0) for b in range(3)]
        m_acc = np.zeros((dims[2], dims[1], dims[0]))
        p_acc = np.zeros_like(m_acc)
        for p in range(P):
            C = np.zeros((3, 3))
            for r, abc in enumerate(modes):
                if abc in lin:
                    C[:, lin[abc]] = coeff[:, r, p]
            A = np.eye(3) + dt * C
            M = np.eye(3) if abs(np.linalg.det(A)) < 1e-6 else np.linalg.inv(A)
            ax = [_axis_moments(x[b, p], dx, 0.0 if b == alpha else 0.5, dims[b]) for b in range(3)]
            Z = np.stack(np.meshgrid(ax[2][1], ax[1][1], ax[0][1], indexing="ij")[::-1])  # (x, y, z)
            xi = np.einsum("bc,ckji->bkji", M, Z)
            w = np.einsum("k,j,i->kji", ax[2][0], ax[1][0], ax[0][0])
            f = [np.stack([np.ones_like(xi[b]), xi[b], xi[b] ** 2 - ax[b][2] * xi[b] - ax[b][3]])
                 for b in range(3)]
            S = sum(coeff[alpha, r, p] * f[0][a] * f[1][b] * f[2][c]
                    for r, (a, b, c) in enumerate(modes))
            m_acc += mass[p] * w
            p_acc += mass[p] * w * S
        gm.append(m_acc)
        gp.append(p_acc)
    return gm, gp


def _particle_grid(pos, alpha, n, dx, modes):
    """w (d_z, d_y, d_x) and s (R, d_z, d_y, d_x) of one particle on grid alpha."""
    dims = [int(n[b]) + (1 if b == alpha else 0) for b in range(3)]
    ax = [_axis(pos[b], dx, 0.0 if b == alpha else 0.5, dims[b]) for b in range(3)]
    w = np.einsum("k,j,i->kji", ax[2][0], ax[1][0], ax[0][0])
    s = np.stack([np.einsum("k,j,i->kji", ax[2][1][c], ax[1][1][b], ax[0][1][a])
                  for (a, b, c) in modes])
    return w, s


def p2g(x, mass, coeff, n, dx, modes):
    x = np.asarray(x, dtype=np.float64)
    coeff = np.asarray(coeff, dtype=np.float64)
    P = x.shape[1]
    gm, gp = [], []
    for alpha in range(3):
        m_acc = None
        p_acc = None
        for p in range(P):
            w, s = _particle_grid(x[:, p], alpha, n, dx, modes)
            S = np.tensordot(coeff[alpha, :, p], s, axes=(0, 0))
            m_acc = mass[p] * w if m_acc is None else m_acc + mass[p] * w
            p_acc = mass[p] * w * S if p_acc is None else p_acc + mass[p] * w * S
        gm.append(m_acc)
        gp.append(p_acc)
    return gm, gp


def g2p_fit(x, gv, n, dx, modes):
    """Coefficients only (no advection): (3, R, P)."""
    x = np.asarray(x, dtype=np.float64)
    P = x.shape[1]
    R = len(modes)
    out = np.zeros((3, R, P))
    for alpha in range(3):
        for p in range(P):
            w, s = _particle_grid(x[:, p], alpha, n, dx, modes)
            num = np.tensordot(s, w * gv[alpha], axes=([1, 2, 3], [0, 1, 2]))
            den = np.tensordot(s * s, w, axes=([1, 2, 3], [0, 1, 2]))
            out[alpha, :, p] = num / den
    return out

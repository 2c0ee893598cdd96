"""Parity at the full size of the benchmarked workload, in its launch
configuration: one polypic_step (sort, P2G with the fused grid update, G2P)
on the 128^3 dam break (3,813,248 particles, 27 modes, FP32), through the C
ABI exactly as bench.py calls it, with seeded random modes so that every mode
carries momentum.

  * the sort at full size: every cell's particle list against the oracle's
    stable sort, and the library's documented slot layout, bit for bit;
  * grid mass and momentum at ~2,400 sampled face nodes (tile seams, walls,
    free surfaces, interior), element by element: the oracle's P2G over the
    particles within reach of those nodes (found with NumPy's own sort) gives
    their exact values;
  * coefficients and positions of 200 sampled particles, every mode element
    by element: the oracle's P2G over the particles within three cells of
    them, its grid update, and its G2P;
  * at every node, mass and constant-mode momentum conservation (sums over
    the grid against sums over the particles), and bit-identical reruns;
  * the BF16 form at full size: the same conservation properties against the
    decoded coefficients.
"""
import numpy as np
import pytest
import torch

import oracle
import slot_layout
from paper_2308_01060_gb300 import polypic as pp
from paper_2308_01060_gb300 import scenes
from gpu_util import codes, max_rel, np_, rel, u32, upload

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def dam_break():
    sc = scenes.dam_break_scene(n=128, R=27)
    f = sc.fluid
    rng = np.random.default_rng(2024)
    c = scenes.random_modes(27, f.n, sc.dx, rng, sigma=0.05)
    c[:, 0] = rng.normal(0.0, 0.5, (3, f.n))
    f = scenes.ParticleSet(x=f.x, mass=f.mass, coeff=c.astype(np.float32), num_modes=27)
    return sc, f


class _CellIndex:
    """Particles by cell (NumPy's stable argsort of the cell index): the
    particles of any box of cells."""

    def __init__(self, x, n):
        self.n = n
        cell = np.minimum((x.astype(np.float64) * n[0]).astype(np.int64), n[0] - 1)
        self.key = (cell[2] * n[1] + cell[1]) * n[0] + cell[0]
        self.order = np.argsort(self.key, kind="stable")
        self.sorted = self.key[self.order]

    def box(self, lo, hi):
        """Indices of the particles in cells lo <= (i, j, k) <= hi (clipped)."""
        lo = np.maximum(lo, 0)
        hi = np.minimum(hi, np.array(self.n) - 1)
        out = []
        for k in range(lo[2], hi[2] + 1):
            for j in range(lo[1], hi[1] + 1):
                a = (k * self.n[1] + j) * self.n[0] + lo[0]
                b = (k * self.n[1] + j) * self.n[0] + hi[0]
                s = np.searchsorted(self.sorted, a, "left")
                e = np.searchsorted(self.sorted, b, "right")
                out.append(self.order[s:e])
        return np.concatenate(out) if out else np.zeros(0, np.int64)


def _run_step(ctx, f, dt):
    fi = upload(ctx, f)
    fo = ctx.new_particles(fi.count)
    g = ctx.new_grid()
    ws = ctx.workspace(fi.count)
    pp.polypic_step(ctx, fi, fo, g, pp.UpdateSettings(dt=dt), ws)
    torch.cuda.synchronize()
    return fi, fo, g


def _sample_nodes(rng, n):
    """About 2,400 face nodes per step, spread where a local mistake would
    hide from a norm over all 6.3M faces: tile seams of the 8x8x4 key tiles
    (the P2G tile merge), the walls and the layers next to them, the block's
    free surfaces (x = 64, z = 64 cells, the top), and the interior."""
    nodes = []
    for a in range(3):
        dims = [n[b] + (a == b) for b in range(3)]

        def pick(kind):
            ijk = [int(rng.integers(0, dims[b])) for b in range(3)]
            if kind == "seam":
                for b in range(3):
                    T = 8 if b < 2 else 4
                    if rng.uniform() < 0.7:
                        ijk[b] = int(np.clip(T * rng.integers(0, dims[b] // T + 1)
                                             + rng.integers(-1, 2), 0, dims[b] - 1))
                ijk = [min(v, 70) if b != 1 else v for b, v in enumerate(ijk)]
            elif kind == "wall":
                b = int(rng.integers(0, 3))
                ijk[b] = int(rng.choice([0, 1, 2, dims[b] - 3, dims[b] - 2, dims[b] - 1]))
                ijk = [min(v, 70) if (e != 1 and e != b) else v for e, v in enumerate(ijk)]
            elif kind == "surface":
                b = int(rng.choice([0, 1, 2]))
                edge = {0: 64, 1: 126, 2: 64}[b]
                ijk = [int(rng.integers(1, 66)) if e != 1 else int(rng.integers(1, 127))
                       for e in range(3)]
                ijk[b] = int(edge + rng.integers(-2, 3))
            else:
                ijk = [int(rng.integers(2, 64)) if b != 1 else int(rng.integers(2, 126))
                       for b in range(3)]
            return (a, [min(v, dims[e] - 1) for e, v in enumerate(ijk)])

        for kind, count in (("seam", 300), ("wall", 200), ("surface", 150), ("interior", 150)):
            nodes += [pick(kind) for _ in range(count)]
    return nodes


def test_full_size_step_sort_grid_and_particles(dam_break):
    sc, f = dam_break
    ctx = pp.Context(sc.n, sc.dx, 27)
    fi, fo, g = _run_step(ctx, f, sc.dt)
    assert pp.polypic_check_device_status(ctx) == 0

    # sort at full size: the oracle's stable per-cell lists, then the
    # library's documented slot layout, bit for bit
    assert slot_layout.per_cell_lists_match(u32(fi.perm), f.x, sc.n, sc.dx)
    perm, cs, _ = slot_layout.library_order(f.x, sc.n, sc.dx)
    assert np.array_equal(u32(fi.perm), perm)
    assert np.array_equal(u32(fi.cell_start), cs)

    idx = _CellIndex(f.x, sc.n)
    rng = np.random.default_rng(7)
    nodes = _sample_nodes(rng, sc.n)
    assert len(nodes) >= 2000
    sel = np.unique(np.concatenate([idx.box(np.array(ijk) - 2, np.array(ijk) + 2)
                                    for _, ijk in nodes]))
    gm, gp = oracle.p2g(f.x[:, sel], f.mass[sel], f.coeff[:, :, sel], sc.n, sc.dx)
    got_m = np.array([np_(g.mass[a])[k, j, i] for a, (i, j, k) in nodes])
    got_p = np.array([np_(g.mom[a])[k, j, i] for a, (i, j, k) in nodes])
    exp_m = np.array([gm[a][k, j, i] for a, (i, j, k) in nodes])
    exp_p = np.array([gp[a][k, j, i] for a, (i, j, k) in nodes])
    assert np.count_nonzero(exp_m) > 1000
    # element by element: no sampled node may be off by more than the tolerance
    # of the largest value, and the set as a whole within it norm-wise
    assert max_rel(got_m, exp_m) < TOL and rel(got_m, exp_m) < TOL
    assert max_rel(got_p, exp_p) < TOL and rel(got_p, exp_p) < TOL
    # nodes that hold no particle's weight are exactly zero on the GPU too
    assert np.all(got_m[exp_m == 0] == 0) and np.all(got_p[exp_m == 0] == 0)

    # sampled particles through the whole step
    ps = rng.choice(f.n, 200, replace=False)
    cells = np.minimum((f.x[:, ps].astype(np.float64) * sc.n[0]).astype(np.int64), sc.n[0] - 1)
    sel = np.unique(np.concatenate([idx.box(cells[:, q] - 3, cells[:, q] + 3)
                                    for q in range(ps.size)]))
    gm, gp = oracle.p2g(f.x[:, sel], f.mass[sel], f.coeff[:, :, sel], sc.n, sc.dx)
    gv = oracle.grid_update(sc.n, sc.dt, (0.0, -9.81, 0.0), gm, gp)
    c_or, x_or = oracle.g2p(f.x[:, ps], gv, 27, sc.n, sc.dx, sc.dt)
    inv = np.empty(f.n, np.int64)
    inv[perm] = np.arange(f.n)
    slots = inv[ps]
    c_gpu = np_(fo.coeff)[:, :, slots].astype(np.float64)
    scale = (sc.dx ** scenes.mode_degrees(27))[None, :, None]
    assert rel(c_gpu[:, 0], c_or[:, 0]) < TOL
    assert max_rel(c_gpu[:, 0], c_or[:, 0]) < TOL
    # higher modes in velocity units (c dx^L), each mode against its own scale
    for r in range(27):
        assert max_rel(c_gpu[:, r] * scale[0, r], c_or[:, r] * scale[0, r]) < 3 * TOL, r
    assert np.max(np.abs(np_(fo.x)[:, slots] - x_or)) < 2e-7
    assert np.array_equal(np_(fo.mass)[slots], f.mass[ps])


def test_full_size_conservation_and_determinism(dam_break):
    """Partition of unity and the orthogonality of the modes to the constant:
    sum_i m_ia = sum_p m_p and sum_i mv_ia = sum_p m_p c_p0a on every face
    grid, at full size; a second run is bit-identical."""
    sc, f = dam_break
    ctx = pp.Context(sc.n, sc.dx, 27)
    fi, fo, g = _run_step(ctx, f, sc.dt)
    m_tot = float(np.sum(f.mass.astype(np.float64)))
    for a in range(3):
        assert abs(np_(g.mass[a]).astype(np.float64).sum() / m_tot - 1.0) < 1e-5
        p_tot = float(np.sum(f.mass.astype(np.float64) * f.coeff[a, 0].astype(np.float64)))
        p_abs = float(np.sum(f.mass.astype(np.float64) * np.abs(f.coeff[a, 0])))
        assert abs(np_(g.mom[a]).astype(np.float64).sum() - p_tot) < 1e-5 * p_abs
    fi2, fo2, g2 = _run_step(ctx, f, sc.dt)
    for a in range(3):
        assert torch.equal(g.mass[a], g2.mass[a]) and torch.equal(g.mom[a], g2.mom[a])
        assert torch.equal(g.vel[a], g2.vel[a])
    assert torch.equal(fo.coeff, fo2.coeff) and torch.equal(fo.x, fo2.x)
    assert pp.polypic_check_device_status(ctx) == 0


def test_full_size_bf16_conservation(dam_break):
    """BF16 codes at full size (G2P encodes, the next P2G decodes): the grid
    conserves the mass and the constant-mode momentum of the decoded state."""
    sc, f = dam_break
    ctx = pp.Context(sc.n, sc.dx, 27, coeff_format="bf16")
    a = upload(ctx, scenes.ParticleSet(x=f.x, mass=f.mass, coeff=None, num_modes=27))
    b = ctx.new_particles(a.count)
    g = ctx.new_grid()
    ws = ctx.workspace(a.count)
    prm = pp.UpdateSettings(dt=sc.dt)
    for _ in range(3):                                   # gravity gives the state velocity
        pp.polypic_step(ctx, a, b, g, prm, ws)
        a, b = b, a
    pp.polypic_sort(ctx, a, ws)
    pp.polypic_p2g(ctx, a, g, ws)
    torch.cuda.synchronize()
    mass = np_(a.mass).astype(np.float64)
    c0 = np_(codes(a, 27)[:, 0]).astype(np.float64) * np_(a.scale).astype(np.float64)[None]
    for k in range(3):
        assert abs(np_(g.mass[k]).astype(np.float64).sum() / mass.sum() - 1.0) < 1e-5
        p_tot = float(np.sum(mass * c0[k]))
        p_abs = float(np.sum(mass * np.abs(c0[k])))
        assert abs(np_(g.mom[k]).astype(np.float64).sum() - p_tot) <= 1e-5 * p_abs + 1e-12
    assert pp.polypic_check_device_status(ctx) == 0

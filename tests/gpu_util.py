"""Helpers shared by the GPU tests: uploading seeded inputs, comparing with the
oracle.  Inputs always come from paper_2308_01060_gb300.scenes or from seeded
NumPy draws here; the oracle never receives a value computed on the GPU."""
import numpy as np
import torch

from paper_2308_01060_gb300 import polypic as pp


def np_(t):
    return t.detach().cpu().numpy()


def u32(t):
    return np_(t).view(np.uint32)


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def max_rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    m = np.abs(b).max()
    return float(np.abs(a - b).max() / (m if m > 0 else 1.0))


def codes(ps, R):
    """The 16-bit codes of a phase as a (3, R, P) float32 tensor in mode order
    (the library stores modes 2k and 2k + 1 as the halves of one word)."""
    c = ps.coeff
    H = c.shape[1]
    return c.permute(0, 1, 3, 2).reshape(3, 2 * H, c.shape[2])[:, :R].float()


def decoded(ps, R, dx):
    """Physical coefficients (3, R, P) float64 of a 16-bit phase:
    code * s_p / dx^L_r."""
    from paper_2308_01060_gb300 import scenes
    dxl = dx ** scenes.mode_degrees(R).astype(np.float64)
    return (np_(codes(ps, R)).astype(np.float64) * np_(ps.scale).astype(np.float64)[None, None, :]
            / dxl[None, :, None])


def upload(ctx, ps_host, device="cuda"):
    """scenes.ParticleSet -> pp.ParticleState (FP32 coefficients or zeros)."""
    coeff = ps_host.coeff
    return pp.upload_particles(ctx, ps_host.x, ps_host.mass, coeff, ps_host.mass_abs, device=device)


def sorted_particles(ctx, ps_host, ws=None):
    ps = upload(ctx, ps_host)
    if ws is None:
        ws = ctx.workspace(ps.count)
    pp.polypic_sort(ctx, ps, ws)
    return ps, ws


def grid_from_host(ctx, mass=None, mom=None, vel=None):
    g = ctx.new_grid()
    for a in range(3):
        if mass is not None:
            g.mass[a].copy_(torch.as_tensor(mass[a], dtype=torch.float32))
        if mom is not None:
            g.mom[a].copy_(torch.as_tensor(mom[a], dtype=torch.float32))
        if vel is not None:
            g.vel[a].copy_(torch.as_tensor(vel[a], dtype=torch.float32))
    return g


def random_grid_velocity(n, dx, seed, amp=1.0):
    """A seeded smooth-plus-noise velocity field on the three face grids
    (host float32 arrays): low Fourier modes plus 20% white noise."""
    rng = np.random.default_rng(seed)
    out = []
    for a in range(3):
        d = [int(n[b]) + (1 if b == a else 0) for b in range(3)]
        k, j, i = np.meshgrid(np.arange(d[2]), np.arange(d[1]), np.arange(d[0]), indexing="ij")
        f = np.zeros((d[2], d[1], d[0]))
        for _ in range(4):
            kv = rng.integers(1, 4, size=3)
            ph = rng.uniform(0, 2 * np.pi, size=3)
            f += rng.standard_normal() * (np.sin(2 * np.pi * kv[0] * i * dx + ph[0])
                                          * np.sin(2 * np.pi * kv[1] * j * dx + ph[1])
                                          * np.sin(2 * np.pi * kv[2] * k * dx + ph[2]))
        f += 0.2 * rng.standard_normal(f.shape)
        out.append((amp * f).astype(np.float32))
    return out


def assert_close(a, b, tol, what=""):
    """Element by element and as a whole: max|a - b| / max|b| and
    ||a - b|| / ||b|| both below tol (a wrong value at a few faces, a tile
    seam or a wall layer cannot hide in the norm)."""
    r, m = rel(a, b), max_rel(a, b)
    assert r < tol and m < tol, f"{what}: norm-wise {r:.3e}, element-wise {m:.3e} (tol {tol:g})"

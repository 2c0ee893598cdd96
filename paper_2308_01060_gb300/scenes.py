"""Seeded synthetic scenes shaped like the paper's workloads.

This module only draws inputs: particle positions, masses, initial velocities
and initial mode coefficients.  It holds none of the transfer arithmetic, so
both the CUDA library's tests and the FP64 oracle can be fed from it.

The paper's own scenes (dam break, fluid splashing on cloth and on yarn,
Section 4 and Table 2) are libWetCloth scene files that are not available, so
these stand-ins reproduce their structure: blocks and spheres of fluid seeded
at 8 particles per cell, and a triangulated sheet of fabric particles.

Conventions:
  * box [0, n dx]^3 with dx = 1/n for the cubic grids used here;
  * particles are seeded uniformly at random inside each selected cell, and
    only cells 2..n-3 on every axis are seeded (a 2-cell margin), so every
    particle's 3x3x3 stencil lies inside the face grids;
  * fluid density rho = 1000 kg/m^3, particle mass rho dx^3 / ppc;
  * coefficients are laid out (3, R, P): component, mode, particle, in the
    canonical mode order (r = 0 constant, r = 1..3 linear in x, y, z, ...).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

RHO_WATER = 1000.0
GRAVITY = (0.0, -9.81, 0.0)


def mode_degrees(R: int) -> np.ndarray:
    """Total polynomial degree of each of the first R modes (input scaling only).

    Follows the documented order: the 8 multilinear modes first
    ((000), (100), (010), (001), (110), (101), (011), (111)), then the triples
    containing a 2 in lexicographic order of (c, b, a)."""
    first = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, 0, 1), (0, 1, 1),
             (1, 1, 1)]
    rest = [(a, b, c) for c in range(3) for b in range(3) for a in range(3)
            if 2 in (a, b, c)]
    return np.array([sum(t) for t in (first + rest)[:R]], dtype=np.int64)


@dataclass
class ParticleSet:
    """One phase of particles.  All arrays are host NumPy arrays."""
    x: np.ndarray                      # (3, P) float32 positions
    mass: np.ndarray                   # (P,) float32
    coeff: Optional[np.ndarray]        # (3, R, P) float32, or None for all-zero
    mass_abs: Optional[np.ndarray] = None  # (P,) float32 absorbed fluid mass (solids)
    num_modes: int = 27

    @property
    def n(self) -> int:
        return int(self.x.shape[1])


@dataclass
class Scene:
    name: str
    n: tuple
    dx: float
    dt: float
    steps: int
    fluid: ParticleSet
    solid: Optional[ParticleSet] = None
    gravity: tuple = GRAVITY
    meta: dict = field(default_factory=dict)


# ------------------------------------------------------------------ seeding

def _interior(n):
    return [(2, int(n[b]) - 2) for b in range(3)]


def seed_cells(cells: np.ndarray, ppc: int, dx: float, rng) -> np.ndarray:
    """ppc uniform-random points in each cell of `cells` (K, 3); (3, K*ppc) float32."""
    K = cells.shape[0]
    u = rng.random((K, ppc, 3))
    pos = (cells[:, None, :].astype(np.float64) + u) * dx
    return np.ascontiguousarray(pos.reshape(K * ppc, 3).T.astype(np.float32))


def box_cells(n, lo, hi) -> np.ndarray:
    """All cells of the box [lo, hi) (per axis), clipped to the seeded margin;
    x fastest."""
    rng_ax = []
    for b, (mlo, mhi) in enumerate(_interior(n)):
        rng_ax.append(np.arange(max(lo[b], mlo), min(hi[b], mhi)))
    kk, jj, ii = np.meshgrid(rng_ax[2], rng_ax[1], rng_ax[0], indexing="ij")
    return np.stack([ii.ravel(), jj.ravel(), kk.ravel()], axis=1)


def vortex_velocity(x: np.ndarray, omega: float = 2.0, center=(0.5, 0.5)):
    """Solid-body rotation about the vertical axis through (center[0], ., center[1]):
    v = (omega (z - cz), 0, -omega (x - cx)), and its gradient dv_a/dx_b."""
    v = np.zeros_like(x, dtype=np.float64)
    v[0] = omega * (x[2] - center[1])
    v[2] = -omega * (x[0] - center[0])
    grad = np.zeros((3, 3), dtype=np.float64)
    grad[0, 2] = omega
    grad[2, 0] = -omega
    return v, grad


def coefficients_from_field(v: np.ndarray, grad: Optional[np.ndarray], R: int) -> np.ndarray:
    """c_0 = v_p, linear modes = the field's gradient (a Taylor expansion in the
    mode basis); higher modes 0.  grad is (3, 3) or (3, 3, P) or None."""
    P = v.shape[1]
    c = np.zeros((3, R, P), dtype=np.float64)
    c[:, 0, :] = v
    if grad is not None and R >= 4:
        g = grad if grad.ndim == 3 else np.broadcast_to(grad[:, :, None], (3, 3, P))
        for a in range(3):
            for b in range(3):
                c[a, 1 + b, :] = g[a, b]
    return c


def random_modes(R: int, P: int, dx: float, rng, sigma: float = 0.1) -> np.ndarray:
    """c_r ~ N(0, sigma^2) / dx^deg(r) for r >= 1 (every mode exercised)."""
    deg = mode_degrees(R)
    c = rng.standard_normal((3, R, P)) * sigma
    c = c / (dx ** deg)[None, :, None]
    c[:, 0, :] = 0.0
    return c


# ------------------------------------------------------------------ scenes

def parity_scene(n: int = 32, R: int = 27, seed: int = 0, random_mode_init: bool = False,
                 dt: float = 1e-3, sigma_v: float = 0.5) -> Scene:
    """Plain PolyPIC, fluid only: the lower half-box at 8 particles per cell,
    velocities ~ N(0, sigma_v^2) plus a solid-body vortex of 2 rad/s; one step."""
    dx = 1.0 / n
    rng = np.random.default_rng(seed)
    cells = box_cells((n, n, n), (0, 0, 0), (n, n // 2, n))
    x = seed_cells(cells, 8, dx, rng)
    P = x.shape[1]
    mass = np.full(P, RHO_WATER * dx ** 3 / 8, dtype=np.float32)
    v_vortex, grad = vortex_velocity(x.astype(np.float64))
    v = v_vortex + rng.standard_normal((3, P)) * sigma_v
    c = coefficients_from_field(v, grad, R)
    if random_mode_init and R > 1:
        rm = random_modes(R, P, dx, rng)
        c[:, 1:, :] += rm[:, 1:, :]
    fluid = ParticleSet(x=x, mass=mass, coeff=c.astype(np.float32), num_modes=R)
    return Scene(name=f"polypic_fluid_{n}^3_halfbox", n=(n, n, n), dx=dx, dt=dt, steps=1,
                 fluid=fluid, meta={"seed": seed, "ppc": 8})


def dam_break_scene(n: int = 128, R: int = 27, seed: int = 0, dt: float = 5e-4,
                    steps: int = 200) -> Scene:
    """Fluid dam break: an (n/2) x n x (n/2)-cell block in the x-low, z-low corner,
    8 particles per cell, zero initial velocity (all coefficients 0)."""
    dx = 1.0 / n
    rng = np.random.default_rng(seed)
    cells = box_cells((n, n, n), (0, 0, 0), (n // 2, n, n // 2))
    x = seed_cells(cells, 8, dx, rng)
    P = x.shape[1]
    mass = np.full(P, RHO_WATER * dx ** 3 / 8, dtype=np.float32)
    fluid = ParticleSet(x=x, mass=mass, coeff=None, num_modes=R)
    return Scene(name=f"dam_break_{n}^3", n=(n, n, n), dx=dx, dt=dt, steps=steps, fluid=fluid,
                 meta={"seed": seed, "ppc": 8, "block_cells": (n // 2, n, n // 2)})


def sheet_particles(verts_per_side: int, side: float, height: float, center_xz=(0.5, 0.5),
                    areal_density: float = 0.1):
    """A horizontal triangulated square sheet (two triangles per quad).

    Vertex particles sit on the vertices, element particles at the triangle
    centroids.  Each triangle's mass (areal_density * area) goes half to its
    element particle and one sixth to each of its three vertices.  Returns
    (x (3, P) float32, mass (P,) float32, num_vertices)."""
    m = verts_per_side
    h = side / (m - 1)
    gx = center_xz[0] - side / 2 + h * np.arange(m)
    gz = center_xz[1] - side / 2 + h * np.arange(m)
    zz, xx = np.meshgrid(gz, gx, indexing="ij")
    vx = np.stack([xx.ravel(), np.full(m * m, height), zz.ravel()])
    vmass = np.zeros(m * m)
    idx = np.arange(m * m).reshape(m, m)
    a = idx[:-1, :-1].ravel()
    b = idx[:-1, 1:].ravel()
    c = idx[1:, :-1].ravel()
    d = idx[1:, 1:].ravel()
    tris = np.concatenate([np.stack([a, b, d], 1), np.stack([a, d, c], 1)])
    tri_mass = areal_density * 0.5 * h * h
    for k in range(3):
        np.add.at(vmass, tris[:, k], tri_mass / 6.0)
    cent = vx[:, tris].mean(axis=2)
    x = np.concatenate([vx, cent], axis=1).astype(np.float32)
    mass = np.concatenate([vmass, np.full(tris.shape[0], tri_mass / 2.0)]).astype(np.float32)
    return np.ascontiguousarray(x), mass, m * m


def splash_scene(n: int = 128, R_fluid: int = 27, R_solid: int = 27, seed: int = 0,
                 sheet_verts: int = 256, dt: float = 2.5e-4, steps: int = 400) -> Scene:
    """Liquid-fabric coupling: a fluid sphere (radius 0.15, centre (0.5, 0.55, 0.5),
    8 particles per cell, velocity (0, -2, 0)) above a horizontal sheet of side
    0.8 at height 0.35 made of vertex and element particles."""
    dx = 1.0 / n
    rng = np.random.default_rng(seed)
    c0 = np.array([0.5, 0.55, 0.5])
    rad = 0.15
    lo = np.floor((c0 - rad) / dx).astype(int)
    hi = np.ceil((c0 + rad) / dx).astype(int) + 1
    cells = box_cells((n, n, n), lo, hi)
    x = seed_cells(cells, 8, dx, rng)
    inside = np.sum((x.astype(np.float64) - c0[:, None]) ** 2, axis=0) <= rad * rad
    x = np.ascontiguousarray(x[:, inside])
    P = x.shape[1]
    mass = np.full(P, RHO_WATER * dx ** 3 / 8, dtype=np.float32)
    v = np.zeros((3, P))
    v[1] = -2.0
    fc = coefficients_from_field(v, None, R_fluid).astype(np.float32)
    fluid = ParticleSet(x=x, mass=mass, coeff=fc, num_modes=R_fluid)
    sx, smass, nv = sheet_particles(sheet_verts, 0.8, 0.35)
    solid = ParticleSet(x=sx, mass=smass, coeff=None, num_modes=R_solid,
                        mass_abs=np.zeros(sx.shape[1], dtype=np.float32))
    return Scene(name=f"splash_sheet_{n}^3", n=(n, n, n), dx=dx, dt=dt, steps=steps,
                 fluid=fluid, solid=solid,
                 meta={"seed": seed, "sheet_vertices": nv,
                       "pinned": "none (the fabric stand-in has no constraints)"})


def random_velocity_scene(n: int = 64, R: int = 27, seed: int = 0, sigma_v: float = 0.3,
                          dt: float = 1e-3, steps: int = 32, modes: bool = True) -> Scene:
    """Half-box at 8 particles per cell with random velocities ~ N(0, sigma_v^2)
    and random higher modes (the differentiable-transfer workload)."""
    dx = 1.0 / n
    rng = np.random.default_rng(seed)
    cells = box_cells((n, n, n), (0, 0, 0), (n, n // 2, n))
    x = seed_cells(cells, 8, dx, rng)
    P = x.shape[1]
    mass = np.full(P, RHO_WATER * dx ** 3 / 8, dtype=np.float32)
    c = np.zeros((3, R, P))
    c[:, 0, :] = rng.standard_normal((3, P)) * sigma_v
    if modes and R > 1:
        rm = random_modes(R, P, dx, rng)
        c[:, 1:, :] = rm[:, 1:, :]
    fluid = ParticleSet(x=x, mass=mass, coeff=c.astype(np.float32), num_modes=R)
    return Scene(name=f"random_velocity_{n}^3", n=(n, n, n), dx=dx, dt=dt, steps=steps,
                 fluid=fluid, meta={"seed": seed, "ppc": 8})


def taylor_green(xf: np.ndarray, alpha: int) -> np.ndarray:
    """Component alpha of the Taylor-Green target field
    u = (sin 2pi x cos 2pi y cos 2pi z, -cos 2pi x sin 2pi y cos 2pi z, 0)."""
    tp = 2.0 * np.pi
    x, y, z = xf
    if alpha == 0:
        return np.sin(tp * x) * np.cos(tp * y) * np.cos(tp * z)
    if alpha == 1:
        return -np.cos(tp * x) * np.sin(tp * y) * np.cos(tp * z)
    return np.zeros_like(x)


def face_positions(alpha: int, n, dx: float):
    """Physical positions of the faces of grid alpha, as (x, y, z) arrays of
    shape (d_z, d_y, d_x)."""
    d = [int(n[b]) + (1 if b == alpha else 0) for b in range(3)]
    off = [0.0 if b == alpha else 0.5 for b in range(3)]
    k, j, i = np.meshgrid(np.arange(d[2]), np.arange(d[1]), np.arange(d[0]), indexing="ij")
    return ((i + off[0]) * dx, (j + off[1]) * dx, (k + off[2]) * dx)


def vortical_modes(seed: int = 0, count: int = 4, amp: float = 0.5):
    """`count` solenoidal Fourier modes u(x) = a sin(2 pi k.x + phi) with integer
    wave vectors k (components 1..3), a random unit direction orthogonal to k
    scaled so that the sum has amplitude ~amp: each mode is divergence free
    because a . k = 0.  Returns a list of (k, a, phi)."""
    rng = np.random.default_rng(seed)
    modes = []
    for _ in range(count):
        k = rng.integers(1, 4, size=3).astype(np.float64)
        r = rng.standard_normal(3)
        a = r - k * (r @ k) / (k @ k)
        a *= amp / (np.linalg.norm(a) * np.sqrt(count))
        modes.append((k, a, float(rng.uniform(0, 2 * np.pi))))
    return modes


def large_scene(n: int = 256, seed: int = 0, sheet_verts: int = 1024, dt: float = 2.5e-4,
                steps: int = 100, amp: float = 0.5) -> Scene:
    """Large fluid + fabric: the lower half-box (y < 1/2) at 8 particles per
    cell inside the 2-cell margin (about 64M particles on 256^3), whose
    initial velocity is the vortical field of `vortical_modes` (the caller
    samples it on the grid and fits the particles' modes from it), plus a
    horizontal sheet of sheet_verts^2 vertices, side 0.8, at height 0.75
    (above the fluid; the height is a stated choice)."""
    dx = 1.0 / n
    rng = np.random.default_rng(seed)
    cells = box_cells((n, n, n), (0, 0, 0), (n, n // 2, n))
    x = seed_cells(cells, 8, dx, rng)
    P = x.shape[1]
    mass = np.full(P, RHO_WATER * dx ** 3 / 8, dtype=np.float32)
    fluid = ParticleSet(x=x, mass=mass, coeff=None, num_modes=27)
    sx, smass, nv = sheet_particles(sheet_verts, 0.8, 0.75)
    solid = ParticleSet(x=sx, mass=smass, coeff=None, num_modes=27,
                        mass_abs=np.zeros(sx.shape[1], dtype=np.float32))
    return Scene(name=f"large_fluid_fabric_{n}^3", n=(n, n, n), dx=dx, dt=dt, steps=steps,
                 fluid=fluid, solid=solid,
                 meta={"seed": seed, "ppc": 8, "sheet_vertices": nv,
                       "field": vortical_modes(seed, 4, amp)})

"""Thin ctypes binding of libpolypic (include/polypic.h).

Argument marshalling only: every step of the transfers runs in the CUDA
library.  PyTorch supplies device memory and streams.  The functions carry the
C entry points' names (``polypic_p2g`` etc.) and take the small state objects
defined here, whose tensors live on the GPU.

Importing this module does not load the library; the first call does, and it
raises ``PolyPICError`` if ``libpolypic.so`` has not been built (there is no
CPU fallback).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpolypic.so")

POLYPIC_OK = 0
STATUS_NAMES = {
    0: "OK", 1: "INVALID_ARG", 2: "UNSUPPORTED", 3: "OUT_OF_DOMAIN", 4: "NONFINITE",
    5: "NOT_CONVERGED", 6: "TIMEOUT", 7: "CUDA", 8: "WORKSPACE",
}
COEFF_FORMATS = {"f32": 0, "bf16": 1, "f16": 2}
ADJ_ACCUMULATE = 1


class PolyPICError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        self.name = STATUS_NAMES.get(status, str(status))
        super().__init__(f"{where}: POLYPIC_ERR_{self.name}")


# ------------------------------------------------------------------ C structs

_vp = ctypes.c_void_p


class Config(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32 * 3), ("dx", ctypes.c_double), ("num_modes", ctypes.c_int32),
                ("coeff_format", ctypes.c_int32), ("map", ctypes.c_int32),
                ("apic_variant", ctypes.c_int32)]


class Particles(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int64), ("x", _vp * 3), ("mass", _vp), ("mass_abs", _vp),
                ("coeff", _vp), ("coeff_scale", _vp), ("key", _vp), ("perm", _vp),
                ("cell_start", _vp), ("id", _vp)]


class FabricParams(ctypes.Structure):
    _fields_ = [("verts_per_side", ctypes.c_int32), ("rest_length", ctypes.c_float),
                ("k_stretch", ctypes.c_float), ("k_shear", ctypes.c_float),
                ("k_bend", ctypes.c_float), ("damping", ctypes.c_float),
                ("absorb_rate", ctypes.c_float), ("absorb_capacity", ctypes.c_float),
                ("absorb_max_fraction", ctypes.c_float)]


class Grid(ctypes.Structure):
    _fields_ = [("mass", _vp * 3), ("mom", _vp * 3), ("vel", _vp * 3)]


class UpdateParams(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_float), ("gravity", ctypes.c_float * 3), ("drag_k", ctypes.c_float),
                ("rho", ctypes.c_float), ("project", ctypes.c_int32),
                ("pcg_maxiter", ctypes.c_int32), ("pcg_rtol", ctypes.c_double)]


_lib = None

EXPORTS = [
    "polypic_create", "polypic_destroy", "polypic_num_keys", "polypic_cell_key",
    "polypic_grid_dims", "polypic_workspace_bytes", "polypic_sort", "polypic_p2g",
    "polypic_p2g_mapped", "polypic_p2g_noalloc",
    "polypic_grid_update", "polypic_g2p", "polypic_step", "polypic_g2p_adjoint",
    "polypic_grid_update_adjoint", "polypic_p2g_adjoint", "polypic_check_device_status",
    "polypic_status_string", "polypic_fabric_forces", "polypic_absorb", "polypic_step_coupled",
    "polypic_g2p2g",
]


def load_library(path: str = LIB_PATH):
    """Load libpolypic.so and declare its signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise PolyPICError(7, f"{path} is missing (build it with paper_2308_01060_gb300.build)")
    L = ctypes.CDLL(path)
    P = ctypes.POINTER
    st = ctypes.c_int
    sigs = {
        "polypic_create": (st, [P(Config), P(_vp)]),
        "polypic_destroy": (None, [_vp]),
        "polypic_num_keys": (ctypes.c_int64, [_vp]),
        "polypic_cell_key": (ctypes.c_uint32, [_vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
        "polypic_grid_dims": (st, [_vp, ctypes.c_int32, P(ctypes.c_int32)]),
        "polypic_workspace_bytes": (ctypes.c_size_t, [_vp, ctypes.c_int64, ctypes.c_int64]),
        "polypic_sort": (st, [_vp, P(Particles), _vp, ctypes.c_size_t, _vp]),
        "polypic_p2g": (st, [_vp, P(Particles), P(Grid), _vp, ctypes.c_size_t, _vp]),
        "polypic_p2g_mapped": (st, [_vp, P(Particles), P(Grid), ctypes.c_float, _vp,
                                    ctypes.c_size_t, _vp]),
        "polypic_p2g_noalloc": (st, [_vp, P(Particles), P(Grid), _vp]),
        "polypic_grid_update": (st, [_vp, P(Grid), P(Grid), P(Particles), P(UpdateParams), _vp,
                                     ctypes.c_size_t, _vp]),
        "polypic_g2p": (st, [_vp, P(Grid), P(Particles), P(Particles), ctypes.c_float, _vp,
                             ctypes.c_size_t, _vp]),
        "polypic_step": (st, [_vp, P(Particles), P(Particles), P(Particles), P(Particles),
                              P(Grid), P(Grid), P(UpdateParams), _vp, ctypes.c_size_t, _vp]),
        "polypic_g2p_adjoint": (st, [_vp, P(Grid), P(Particles), ctypes.c_float, P(Particles),
                                     P(Grid), P(Particles), ctypes.c_int32, _vp, ctypes.c_size_t,
                                     _vp]),
        "polypic_grid_update_adjoint": (st, [_vp, P(Grid), P(Grid), P(Particles), P(UpdateParams),
                                             P(Grid), P(Grid), P(Grid), P(Grid), _vp,
                                             ctypes.c_size_t, _vp]),
        "polypic_p2g_adjoint": (st, [_vp, P(Particles), P(Grid), P(Particles), ctypes.c_int32, _vp,
                                     ctypes.c_size_t, _vp]),
        "polypic_check_device_status": (st, [_vp, _vp]),
        "polypic_g2p2g": (st, [_vp, P(Grid), P(Particles), P(Particles), P(Particles), P(Grid),
                               ctypes.c_float, _vp, ctypes.c_size_t, _vp]),
        "polypic_fabric_forces": (st, [_vp, P(Particles), P(FabricParams), ctypes.c_float, _vp,
                                       ctypes.c_size_t, _vp]),
        "polypic_absorb": (st, [_vp, P(Particles), P(Particles), P(FabricParams), ctypes.c_float,
                                _vp]),
        "polypic_step_coupled": (st, [_vp, P(Particles), P(Particles), P(Particles),
                                      P(Particles), P(Grid), P(Grid), P(UpdateParams),
                                      P(FabricParams), _vp, ctypes.c_size_t, _vp]),
        "polypic_status_string": (ctypes.c_char_p, [st]),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(status: int, where: str):
    if status != POLYPIC_OK:
        raise PolyPICError(status, where)


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    return _vp(t.data_ptr())


def _stream(stream) -> _vp:
    if stream is None:
        stream = torch.cuda.current_stream()
    return _vp(stream.cuda_stream)


# ------------------------------------------------------------------ state objects

@dataclass
class ParticleState:
    """One phase of particles on the GPU.  x: (3, P) float32; coeff: (3, R, P)
    float32, or for the 16-bit formats bfloat16 / float16 codes shaped
    (3, (R + 1) // 2, P, 2) (mode 2k of particle p at [a, k, p, 0], mode 2k + 1
    at [a, k, p, 1]: the library's word layout) with scale (P,);
    key, perm: (P,) int32 holding uint32; cell_start: (K + 1,) int32."""
    x: torch.Tensor
    mass: torch.Tensor
    coeff: torch.Tensor
    key: torch.Tensor
    perm: torch.Tensor
    cell_start: torch.Tensor
    mass_abs: Optional[torch.Tensor] = None
    scale: Optional[torch.Tensor] = None
    id: Optional[torch.Tensor] = None

    @property
    def count(self) -> int:
        return int(self.x.shape[1])

    def c_struct(self) -> Particles:
        s = Particles()
        s.count = self.count
        for a in range(3):
            s.x[a] = self.x[a].data_ptr()
        s.mass = self.mass.data_ptr()
        s.mass_abs = None if self.mass_abs is None else self.mass_abs.data_ptr()
        s.coeff = self.coeff.data_ptr()
        s.coeff_scale = None if self.scale is None else self.scale.data_ptr()
        s.key = self.key.data_ptr()
        s.perm = self.perm.data_ptr()
        s.cell_start = self.cell_start.data_ptr()
        s.id = None if self.id is None else self.id.data_ptr()
        return s


@dataclass
class GridState:
    mass: List[torch.Tensor] = field(default_factory=list)
    mom: List[torch.Tensor] = field(default_factory=list)
    vel: List[torch.Tensor] = field(default_factory=list)

    def c_struct(self) -> Grid:
        g = Grid()
        for a in range(3):
            g.mass[a] = self.mass[a].data_ptr() if self.mass else None
            g.mom[a] = self.mom[a].data_ptr() if self.mom else None
            g.vel[a] = self.vel[a].data_ptr() if self.vel else None
        return g


@dataclass
class UpdateSettings:
    dt: float
    gravity: tuple = (0.0, -9.81, 0.0)
    drag_k: float = 0.0
    rho: float = 1000.0
    project: bool = False
    pcg_maxiter: int = 500
    pcg_rtol: float = 1e-6

    def c_struct(self) -> UpdateParams:
        u = UpdateParams()
        u.dt = self.dt
        for a in range(3):
            u.gravity[a] = self.gravity[a]
        u.drag_k = self.drag_k
        u.rho = self.rho
        u.project = int(self.project)
        u.pcg_maxiter = self.pcg_maxiter
        u.pcg_rtol = self.pcg_rtol
        return u


class Context:
    """A polypic_ctx: grid size, cell width, mode count and coefficient format."""

    def __init__(self, n, dx: float, num_modes: int = 27, coeff_format: str = "f32",
                 map_affine: bool = False, apic_grad_w: bool = False):
        L = load_library()
        cfg = Config()
        for a in range(3):
            cfg.n[a] = int(n[a])
        cfg.dx = float(dx)
        cfg.num_modes = int(num_modes)
        cfg.coeff_format = COEFF_FORMATS[coeff_format]
        cfg.map = int(bool(map_affine))
        cfg.apic_variant = int(bool(apic_grad_w))
        h = _vp()
        _check(L.polypic_create(ctypes.byref(cfg), ctypes.byref(h)), "polypic_create")
        self._h = h
        self.n = tuple(int(v) for v in n)
        self.dx = float(dx)
        self.num_modes = int(num_modes)
        self.coeff_format = coeff_format
        self.variant = bool(map_affine or apic_grad_w)
        self.num_keys = int(L.polypic_num_keys(h))

    @property
    def handle(self):
        return self._h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.polypic_destroy(h)
            self._h = None

    def grid_dims(self, axis: int):
        d = (ctypes.c_int32 * 3)()
        _check(load_library().polypic_grid_dims(self._h, axis, d), "polypic_grid_dims")
        return (d[0], d[1], d[2])

    def cell_key(self, i, j, k) -> int:
        return int(load_library().polypic_cell_key(self._h, i, j, k))

    def workspace_bytes(self, n_fluid: int, n_solid: int = 0) -> int:
        return int(load_library().polypic_workspace_bytes(self._h, n_fluid, n_solid))

    def workspace(self, n_fluid: int, n_solid: int = 0, device="cuda") -> torch.Tensor:
        nbytes = self.workspace_bytes(n_fluid, n_solid)
        return torch.empty(nbytes + 256, dtype=torch.uint8, device=device)

    # -------------------------------------------------------------- allocation helpers
    def coeff_shape(self, count: int):
        """Shape of a phase's coefficient tensor (see ParticleState)."""
        R = self.num_modes
        return (3, R, count) if self.coeff_format == "f32" else (3, (R + 1) // 2, count, 2)

    def coeff_dtype(self):
        return {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[self.coeff_format]

    def new_particles(self, count: int, solid: bool = False, device="cuda",
                      ids: bool = False) -> ParticleState:
        R = self.num_modes
        return ParticleState(
            x=torch.empty((3, count), dtype=torch.float32, device=device),
            mass=torch.empty(count, dtype=torch.float32, device=device),
            coeff=torch.zeros(self.coeff_shape(count), dtype=self.coeff_dtype(), device=device),
            key=torch.empty(count, dtype=torch.int32, device=device),
            perm=torch.empty(count, dtype=torch.int32, device=device),
            cell_start=torch.empty(self.num_keys + 1, dtype=torch.int32, device=device),
            mass_abs=torch.zeros(count, dtype=torch.float32, device=device) if solid else None,
            scale=(torch.zeros(count, dtype=torch.float32, device=device)
                   if self.coeff_format != "f32" else None),
            id=torch.zeros(count, dtype=torch.int32, device=device) if ids else None,
        )

    def new_grid(self, device="cuda", vel=True) -> GridState:
        shapes = [tuple(reversed(self.grid_dims(a))) for a in range(3)]
        z = lambda: [torch.zeros(s, dtype=torch.float32, device=device) for s in shapes]
        return GridState(mass=z(), mom=z(), vel=z() if vel else [])


def _ws(ws: torch.Tensor):
    """A 256-byte-aligned view of a workspace tensor: (pointer, bytes)."""
    base = ws.data_ptr()
    off = (-base) % 256
    return _vp(base + off), ws.numel() - off


# ------------------------------------------------------------------ entry points

def polypic_sort(ctx: Context, p: ParticleState, ws: torch.Tensor, stream=None):
    cs = p.c_struct()
    wp, wb = _ws(ws)
    _check(load_library().polypic_sort(ctx.handle, ctypes.byref(cs), wp, wb, _stream(stream)),
           "polypic_sort")


def polypic_p2g(ctx: Context, p: ParticleState, g: GridState, ws: torch.Tensor, stream=None):
    cs = p.c_struct()
    cg = g.c_struct()
    wp, wb = _ws(ws)
    _check(load_library().polypic_p2g(ctx.handle, ctypes.byref(cs), ctypes.byref(cg), wp, wb,
                                      _stream(stream)), "polypic_p2g")


def polypic_p2g_mapped(ctx: Context, p: ParticleState, g: GridState, dt: float,
                       ws: torch.Tensor, stream=None):
    """P2G over a step of dt (Eq 12's affine map on contexts made with
    map_affine=True; the same as polypic_p2g otherwise)."""
    cs = p.c_struct()
    cg = g.c_struct()
    wp, wb = _ws(ws)
    _check(load_library().polypic_p2g_mapped(ctx.handle, ctypes.byref(cs), ctypes.byref(cg),
                                             float(dt), wp, wb, _stream(stream)),
           "polypic_p2g_mapped")


def polypic_p2g_noalloc(ctx: Context, p: ParticleState, g: GridState, stream=None):
    """P2G using the library's built-in scratch instead of a workspace, for
    callers that must not allocate device memory while running (grids of at
    most 2048 key tiles).  Calls that overlap on the GPU race on that scratch."""
    cs = p.c_struct()
    cg = g.c_struct()
    _check(load_library().polypic_p2g_noalloc(ctx.handle, ctypes.byref(cs), ctypes.byref(cg),
                                              _stream(stream)), "polypic_p2g_noalloc")


def polypic_grid_update(ctx: Context, fluid: GridState, params: UpdateSettings,
                        solid: Optional[GridState] = None,
                        fluid_particles: Optional[ParticleState] = None,
                        ws: Optional[torch.Tensor] = None, stream=None):
    cf = fluid.c_struct()
    csol = solid.c_struct() if solid is not None else None
    cp = fluid_particles.c_struct() if fluid_particles is not None else None
    up = params.c_struct()
    wp, wb = _ws(ws) if ws is not None else (None, 0)
    _check(load_library().polypic_grid_update(
        ctx.handle, ctypes.byref(cf), ctypes.byref(csol) if csol is not None else None,
        ctypes.byref(cp) if cp is not None else None, ctypes.byref(up), wp, wb, _stream(stream)),
        "polypic_grid_update")


def polypic_g2p(ctx: Context, g: GridState, p_in: ParticleState, p_out: ParticleState, dt: float,
                ws: Optional[torch.Tensor] = None, stream=None):
    cg = g.c_struct()
    ci = p_in.c_struct()
    co = p_out.c_struct()
    wp, wb = _ws(ws) if ws is not None else (None, 0)
    _check(load_library().polypic_g2p(ctx.handle, ctypes.byref(cg), ctypes.byref(ci),
                                      ctypes.byref(co), float(dt), wp, wb, _stream(stream)),
           "polypic_g2p")


def polypic_step(ctx: Context, fluid_in: ParticleState, fluid_out: ParticleState, gf: GridState,
                 params: UpdateSettings, ws: torch.Tensor, solid_in: Optional[ParticleState] = None,
                 solid_out: Optional[ParticleState] = None, gs: Optional[GridState] = None,
                 stream=None):
    fi, fo = fluid_in.c_struct(), fluid_out.c_struct()
    si = solid_in.c_struct() if solid_in is not None else None
    so = solid_out.c_struct() if solid_out is not None else None
    cgf = gf.c_struct()
    cgs = gs.c_struct() if gs is not None else None
    up = params.c_struct()
    wp, wb = _ws(ws)
    ref = lambda s: ctypes.byref(s) if s is not None else None
    _check(load_library().polypic_step(ctx.handle, ref(fi), ref(fo), ref(si), ref(so), ref(cgf),
                                       ref(cgs), ref(up), wp, wb, _stream(stream)), "polypic_step")


def polypic_g2p2g(ctx: Context, g: GridState, p_in: ParticleState, p_out: ParticleState,
                  spill: ParticleState, g_next: GridState, dt: float, ws: torch.Tensor,
                  stream=None):
    cg, ci, co, cs, cn = (g.c_struct(), p_in.c_struct(), p_out.c_struct(), spill.c_struct(),
                          g_next.c_struct())
    wp, wb = _ws(ws)
    _check(load_library().polypic_g2p2g(ctx.handle, ctypes.byref(cg), ctypes.byref(ci),
                                        ctypes.byref(co), ctypes.byref(cs), ctypes.byref(cn),
                                        float(dt), wp, wb, _stream(stream)), "polypic_g2p2g")


@dataclass
class FabricSettings:
    """The fabric and absorption stand-ins (see polypic_fabric_params)."""
    verts_per_side: int
    rest_length: float
    k_stretch: float = 0.0
    k_shear: float = 0.0
    k_bend: float = 0.0
    damping: float = 0.0
    absorb_rate: float = 0.0
    absorb_capacity: float = 1.0
    absorb_max_fraction: float = 0.5

    def c_struct(self) -> FabricParams:
        f = FabricParams()
        for k in ("verts_per_side", "rest_length", "k_stretch", "k_shear", "k_bend", "damping",
                  "absorb_rate", "absorb_capacity", "absorb_max_fraction"):
            setattr(f, k, getattr(self, k))
        return f


def polypic_fabric_forces(ctx: Context, solid: ParticleState, fabric: FabricSettings, dt: float,
                          ws: torch.Tensor, stream=None):
    cs, cf = solid.c_struct(), fabric.c_struct()
    wp, wb = _ws(ws)
    _check(load_library().polypic_fabric_forces(ctx.handle, ctypes.byref(cs), ctypes.byref(cf),
                                                float(dt), wp, wb, _stream(stream)),
           "polypic_fabric_forces")


def polypic_absorb(ctx: Context, fluid: ParticleState, solid: ParticleState,
                   fabric: FabricSettings, dt: float, stream=None):
    cfl, cs, cf = fluid.c_struct(), solid.c_struct(), fabric.c_struct()
    _check(load_library().polypic_absorb(ctx.handle, ctypes.byref(cfl), ctypes.byref(cs),
                                         ctypes.byref(cf), float(dt), _stream(stream)),
           "polypic_absorb")


def polypic_step_coupled(ctx: Context, fluid_in: ParticleState, fluid_out: ParticleState,
                         solid_in: ParticleState, solid_out: ParticleState, gf: GridState,
                         gs: GridState, params: UpdateSettings, fabric: FabricSettings,
                         ws: torch.Tensor, stream=None):
    fi, fo, si, so = (fluid_in.c_struct(), fluid_out.c_struct(), solid_in.c_struct(),
                      solid_out.c_struct())
    cgf, cgs, up, cf = gf.c_struct(), gs.c_struct(), params.c_struct(), fabric.c_struct()
    wp, wb = _ws(ws)
    _check(load_library().polypic_step_coupled(
        ctx.handle, ctypes.byref(fi), ctypes.byref(fo), ctypes.byref(si), ctypes.byref(so),
        ctypes.byref(cgf), ctypes.byref(cgs), ctypes.byref(up), ctypes.byref(cf), wp, wb,
        _stream(stream)), "polypic_step_coupled")


def polypic_g2p_adjoint(ctx: Context, g: GridState, p_in: ParticleState, dt: float,
                        bar_out: ParticleState, bar_grid: GridState, bar_in: ParticleState,
                        ws: torch.Tensor, accumulate: bool = False, stream=None):
    cg, ci, bo, bg, bi = (g.c_struct(), p_in.c_struct(), bar_out.c_struct(), bar_grid.c_struct(),
                          bar_in.c_struct())
    wp, wb = _ws(ws)
    _check(load_library().polypic_g2p_adjoint(
        ctx.handle, ctypes.byref(cg), ctypes.byref(ci), float(dt), ctypes.byref(bo),
        ctypes.byref(bg), ctypes.byref(bi), ADJ_ACCUMULATE if accumulate else 0, wp, wb,
        _stream(stream)), "polypic_g2p_adjoint")


def polypic_grid_update_adjoint(ctx: Context, g: GridState, params: UpdateSettings,
                                bar_out: GridState, bar_in: GridState,
                                solid: Optional[GridState] = None,
                                bar_solid_out: Optional[GridState] = None,
                                bar_solid_in: Optional[GridState] = None,
                                fluid_particles: Optional[ParticleState] = None,
                                ws: Optional[torch.Tensor] = None, stream=None):
    ref = lambda x: ctypes.byref(x) if x is not None else None
    cs = lambda x: x.c_struct() if x is not None else None
    cg, bo, bi = g.c_struct(), bar_out.c_struct(), bar_in.c_struct()
    up = params.c_struct()
    wp, wb = _ws(ws) if ws is not None else (None, 0)
    _check(load_library().polypic_grid_update_adjoint(
        ctx.handle, ctypes.byref(cg), ref(cs(solid)), ref(cs(fluid_particles)), ctypes.byref(up),
        ctypes.byref(bo), ref(cs(bar_solid_out)), ctypes.byref(bi), ref(cs(bar_solid_in)), wp, wb,
        _stream(stream)), "polypic_grid_update_adjoint")


def polypic_p2g_adjoint(ctx: Context, p_in: ParticleState, bar_grid: GridState,
                        bar_in: ParticleState, ws: torch.Tensor, accumulate: bool = False,
                        stream=None):
    ci, bg, bi = p_in.c_struct(), bar_grid.c_struct(), bar_in.c_struct()
    wp, wb = _ws(ws)
    _check(load_library().polypic_p2g_adjoint(
        ctx.handle, ctypes.byref(ci), ctypes.byref(bg), ctypes.byref(bi),
        ADJ_ACCUMULATE if accumulate else 0, wp, wb, _stream(stream)), "polypic_p2g_adjoint")


def polypic_check_device_status(ctx: Context, stream=None) -> int:
    """Synchronise the stream; return the latched device status (0 = OK) and clear it."""
    return int(load_library().polypic_check_device_status(ctx.handle, _stream(stream)))


# ------------------------------------------------------------------ conveniences

def upload_particles(ctx: Context, x, mass, coeff=None, mass_abs=None, device="cuda",
                     ids=None) -> ParticleState:
    """Copy host arrays (NumPy or torch) into a new ParticleState (FP32
    coefficients are copied as given; 16-bit contexts start from zero codes
    and get theirs from G2P; ids: the labels polypic_step_coupled carries)."""
    P = int(x.shape[1])
    ps = ctx.new_particles(P, solid=mass_abs is not None, device=device, ids=ids is not None)
    if ids is not None:
        ps.id.copy_(torch.as_tensor(np.asarray(ids).astype(np.int64).astype(np.int32)))
    ps.x.copy_(torch.as_tensor(x, dtype=torch.float32))
    ps.mass.copy_(torch.as_tensor(mass, dtype=torch.float32))
    if mass_abs is not None:
        ps.mass_abs.copy_(torch.as_tensor(mass_abs, dtype=torch.float32))
    if coeff is not None:
        if ctx.coeff_format != "f32":
            raise ValueError("upload_particles: 16-bit contexts take their codes from G2P")
        ps.coeff.copy_(torch.as_tensor(coeff, dtype=torch.float32))
    return ps

"""FP64 CPU oracle for the PolyPIC transfers -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never imports, links or calls it, and it imports nothing
from the product path.

``polypic_oracle.c`` holds the literal FP64 transfers (Eqs 1-20 of the paper);
this module compiles it with gcc and wraps it with ctypes, taking and returning
NumPy arrays.  ``bruteforce`` holds an all-pairs NumPy evaluator for tiny grids.

Grid arrays are NumPy arrays of shape (d_z, d_y, d_x) with x fastest, where
face grid ``a`` has d = (n_x + [a == 0], n_y + [a == 1], n_z + [a == 2]).
Coefficients are arrays of shape (3, R, P): component, mode, particle.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "polypic_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

OR_OK = 0
OR_ERR_ARG = -1
OR_ERR_DOMAIN = -2
OR_ERR_NOT_CONVERGED = -3


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile polypic_oracle.c into oracle/liboracle.so (plain C99, no FMA)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_D = ctypes.POINTER(ctypes.c_double)
_F = ctypes.POINTER(ctypes.c_float)
_U32 = ctypes.POINTER(ctypes.c_uint32)
_U8 = ctypes.POINTER(ctypes.c_uint8)
_PA = ctypes.c_void_p   # a C array of three double pointers (see _ptr3)
_I = ctypes.POINTER(ctypes.c_int)
_i64 = ctypes.c_int64
_int = ctypes.c_int
_dbl = ctypes.c_double


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    sig = {
        "or_mode_abc": (None, [_int, _I]),
        "or_set_threads": (None, [_int]),
        "or_get_threads": (_int, []),
        "or_keys": (None, [_i64, _F, _F, _F, _int, _int, _int, _dbl, _U32]),
        "or_stable_sort": (None, [_i64, _U32, ctypes.c_uint32, _U32, _U32]),
        "or_stencil_1d": (_int, [_dbl, _dbl, _int, _I, _D, _D, _D, _D, _I]),
        "or_particle_modes": (_int, [_dbl, _dbl, _dbl, _int, _int, _dbl, _I, _D, _D, _D, _I]),
        "or_p2g": (_int, [_i64, _D, _D, _D, _D, _D, _D, _int, _int, _int, _int, _dbl, _int,
                          _dbl, _D, _D, _D, _D, _D, _D]),
        "or_grid_update": (None, [_int, _int, _int, _dbl, _dbl, _dbl, _dbl, _dbl]
                           + [_D] * 18),
        "or_g2p": (_int, [_i64, _D, _D, _D, _D, _D, _D, _int, _int, _int, _int, _dbl, _dbl,
                          _int, _D, _D, _D, _D]),
        "or_p2g_adjoint": (_int, [_i64, _D, _D, _D, _D, _D, _D, _int, _int, _int, _int, _dbl]
                           + [_D] * 10),
        "or_grid_update_adjoint": (_int, [_int, _int, _int, _dbl, _dbl, _dbl, _dbl, _dbl, _PA,
                                          _PA, _PA, _PA, _U8, _dbl, _int, _PA, _PA, _PA, _PA,
                                          _PA, _PA]),
        "or_g2p_adjoint": (_int, [_i64, _D, _D, _D, _D, _D, _D, _int, _int, _int, _int, _dbl,
                                  _dbl] + [_D] * 10),
        "or_fabric_forces": (None, [_i64, _D, _D, _D, _D, _D, _D, _int, _U32, _int, _dbl, _dbl,
                                    _dbl, _dbl, _dbl, _dbl]),
        "or_absorb": (None, [_i64, _F, _F, _F, _D, _i64, _F, _F, _F, _D, _D, _int, _int, _int,
                             _dbl, _dbl, _dbl, _dbl, _dbl]),
        "or_pcg_project": (_int, [_int, _int, _int, _dbl, _dbl, _dbl, _U8, _D, _D, _D, _D,
                                  _dbl, _int]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


# ---------------------------------------------------------------- helpers

def _p(a, ctype):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def face_dims(alpha: int, n) -> tuple:
    """(d_x, d_y, d_z) of face grid alpha on an n = (n_x, n_y, n_z) cell grid."""
    return tuple(int(n[b]) + (1 if b == alpha else 0) for b in range(3))


def face_shape(alpha: int, n) -> tuple:
    d = face_dims(alpha, n)
    return (d[2], d[1], d[0])


def _check(rc, what):
    if rc == OR_ERR_DOMAIN:
        raise OracleError(f"{what}: particle outside [dx, (n-1)dx)")
    if rc == OR_ERR_ARG:
        raise OracleError(f"{what}: invalid argument")
    if rc == OR_ERR_NOT_CONVERGED:
        raise OracleError(f"{what}: not converged")


# ---------------------------------------------------------------- modes / keys

def set_threads(n: int) -> None:
    """Host threads of P2G and G2P (1, the default, runs the plain serial
    loops; more split G2P by particle and give P2G private grids summed in
    thread order)."""
    _load().or_set_threads(int(n))


def get_threads() -> int:
    return int(_load().or_get_threads())


def mode_abc(r: int) -> tuple:
    out = (ctypes.c_int * 3)()
    _load().or_mode_abc(r, out)
    return (out[0], out[1], out[2])


def num_cells(n) -> int:
    return int(n[0]) * int(n[1]) * int(n[2])


def keys(x32, n, dx) -> np.ndarray:
    """Cell index (k n_y + j) n_x + i of each particle; x32 is a (3, P) float32
    array.  The cell is decided in FP32 (one rounding of x * (float)(1/dx))."""
    x32 = _f32(x32)
    P = x32.shape[1]
    out = np.empty(P, dtype=np.uint32)
    _load().or_keys(P, _p(x32[0], ctypes.c_float), _p(x32[1], ctypes.c_float),
                    _p(x32[2], ctypes.c_float), int(n[0]), int(n[1]), int(n[2]),
                    float(dx), _p(out, ctypes.c_uint32))
    return out


def stable_sort(key, nkeys: int):
    """(perm in (key, index) order, cell_start)."""
    key = np.ascontiguousarray(key, dtype=np.uint32)
    P = key.shape[0]
    perm = np.empty(P, dtype=np.uint32)
    cs = np.empty(nkeys + 1, dtype=np.uint32)
    _load().or_stable_sort(P, _p(key, ctypes.c_uint32), nkeys, _p(perm, ctypes.c_uint32),
                           _p(cs, ctypes.c_uint32))
    return perm, cs


def cell_sort(x32, n, dx):
    """Stable counting sort of the particles by cell index: (perm, cell_start,
    key).  perm[cell_start[c]:cell_start[c + 1]] lists the particles of cell c
    in increasing index order."""
    key = keys(x32, n, dx)
    perm, cs = stable_sort(key, num_cells(n))
    return perm, cs, key


# ---------------------------------------------------------------- basis

def stencil_1d(xb: float, dx: float, face: bool):
    base = ctypes.c_int()
    w = np.empty(3)
    z = np.empty(3)
    mu2 = ctypes.c_double()
    kappa = ctypes.c_double()
    guard = ctypes.c_int()
    _load().or_stencil_1d(float(xb), float(dx), int(bool(face)), ctypes.byref(base),
                          _p(w, ctypes.c_double), _p(z, ctypes.c_double), ctypes.byref(mu2),
                          ctypes.byref(kappa), ctypes.byref(guard))
    return base.value, w, z, mu2.value, kappa.value, guard.value


def particle_modes(pos, alpha: int, R: int, dx: float):
    node = np.empty((27, 3), dtype=np.int32)
    w = np.empty(27)
    s = np.empty((27, R))
    d = np.empty(R)
    guard = np.empty(3, dtype=np.int32)
    _load().or_particle_modes(float(pos[0]), float(pos[1]), float(pos[2]), alpha, R, float(dx),
                              _p(node, ctypes.c_int), _p(w, ctypes.c_double),
                              _p(s, ctypes.c_double), _p(d, ctypes.c_double),
                              _p(guard, ctypes.c_int))
    return node, w, s, d, guard


# ---------------------------------------------------------------- transfers

def p2g(x, mass, coeff, n, dx, mass_abs=None, map_affine=False, dt=0.0):
    """P2G (Eqs 1-5, 13, 15-18).  x: (3, P), mass: (P,), coeff: (3, R, P).
    Returns (gm, gp): lists of 3 face-grid arrays (mass, momentum)."""
    x = _f64(x)
    mass = _f64(mass)
    coeff = _f64(coeff)
    mabs = None if mass_abs is None else _f64(mass_abs)
    R = coeff.shape[1]
    P = x.shape[1]
    gm = [np.zeros(face_shape(a, n)) for a in range(3)]
    gp = [np.zeros(face_shape(a, n)) for a in range(3)]
    D = ctypes.c_double
    rc = _load().or_p2g(P, _p(x[0], D), _p(x[1], D), _p(x[2], D), _p(mass, D), _p(mabs, D),
                        _p(coeff, D), R, int(n[0]), int(n[1]), int(n[2]), float(dx),
                        int(bool(map_affine)), float(dt), *[_p(g, D) for g in gm],
                        *[_p(g, D) for g in gp])
    _check(rc, "p2g")
    return gm, gp


def grid_update(n, dt, gravity, fm, fp, sm=None, sp=None, drag_k=0.0):
    """Grid update: v = mv/m, + dt g, optional two-phase drag, wall faces zeroed.
    Returns fv (and sv when a solid grid is given)."""
    D = ctypes.c_double
    fm = [_f64(a) for a in fm]
    fp = [_f64(a) for a in fp]
    fv = [np.zeros_like(a) for a in fm]
    if sm is not None:
        sm = [_f64(a) for a in sm]
        sp = [_f64(a) for a in sp]
        sv = [np.zeros_like(a) for a in sm]
        sargs = [_p(a, D) for a in sm] + [_p(a, D) for a in sp] + [_p(a, D) for a in sv]
    else:
        sv = None
        sargs = [None] * 9
    _load().or_grid_update(int(n[0]), int(n[1]), int(n[2]), float(dt), float(gravity[0]),
                           float(gravity[1]), float(gravity[2]), float(drag_k),
                           *[_p(a, D) for a in fm], *[_p(a, D) for a in fp],
                           *[_p(a, D) for a in fv], *sargs)
    return (fv, sv) if sm is not None else fv


def g2p(x, gv, R, n, dx, dt, apic_grad=False):
    """G2P fit + advection.  Returns (coeff (3, R, P), x_new (3, P))."""
    D = ctypes.c_double
    x = _f64(x)
    gv = [_f64(a) for a in gv]
    P = x.shape[1]
    coeff = np.zeros((3, R, P))
    xo = np.zeros((3, P))
    rc = _load().or_g2p(P, _p(x[0], D), _p(x[1], D), _p(x[2], D), *[_p(a, D) for a in gv], R,
                        int(n[0]), int(n[1]), int(n[2]), float(dx), float(dt),
                        int(bool(apic_grad)), _p(coeff, D), _p(xo[0], D), _p(xo[1], D),
                        _p(xo[2], D))
    _check(rc, "g2p")
    return coeff, xo


def p2g_adjoint(x, mass, coeff, n, dx, lm, lp, mass_abs=None):
    """Adjoint of P2G at the given state: returns (lc (3, R, P), lx (3, P))."""
    D = ctypes.c_double
    x = _f64(x)
    mass = _f64(mass)
    coeff = _f64(coeff)
    mabs = None if mass_abs is None else _f64(mass_abs)
    lm = [_f64(a) for a in lm]
    lp = [_f64(a) for a in lp]
    R = coeff.shape[1]
    P = x.shape[1]
    lc = np.zeros((3, R, P))
    lx = np.zeros((3, P))
    rc = _load().or_p2g_adjoint(P, _p(x[0], D), _p(x[1], D), _p(x[2], D), _p(mass, D),
                                _p(mabs, D), _p(coeff, D), R, int(n[0]), int(n[1]), int(n[2]),
                                float(dx), *[_p(a, D) for a in lm], *[_p(a, D) for a in lp],
                                _p(lc, D), _p(lx[0], D), _p(lx[1], D), _p(lx[2], D))
    _check(rc, "p2g_adjoint")
    return lc, lx


def _ptr3(arrs):
    """Three FP64 arrays as a C array of three pointers (None stays NULL)."""
    if arrs is None:
        return None
    return (ctypes.c_void_p * 3)(*[a.ctypes.data for a in arrs])


def grid_update_adjoint(n, fm, fp, lv, dt=0.0, gravity=(0.0, -9.81, 0.0), sm=None, sp=None,
                        lsv=None, drag_k=0.0, fluid=None, rtol=1e-12, maxiter=5000):
    """Adjoint of grid_update (then pcg_project on the fluid velocity when the
    fluid-cell mask `fluid` (n_z, n_y, n_x) is given).  lv (and lsv with a
    solid grid sm, sp): dL/dv~.  Returns (lm, lp), or (lm, lp, lsm, lsp) with a
    solid grid."""
    fm = [_f64(a) for a in fm]
    fp = [_f64(a) for a in fp]
    lv = [_f64(a) for a in lv]
    lm = [np.zeros_like(a) for a in fm]
    lp = [np.zeros_like(a) for a in fm]
    solid = sm is not None
    if solid:
        sm = [_f64(a) for a in sm]
        sp = [_f64(a) for a in sp]
        lsv = [_f64(a) for a in lsv] if lsv is not None else [np.zeros_like(a) for a in sm]
        lsm = [np.zeros_like(a) for a in sm]
        lsp = [np.zeros_like(a) for a in sm]
    else:
        lsv = lsm = lsp = None
    fl = None if fluid is None else np.ascontiguousarray(fluid, dtype=np.uint8)
    rc = _load().or_grid_update_adjoint(
        int(n[0]), int(n[1]), int(n[2]), float(dt), float(gravity[0]), float(gravity[1]),
        float(gravity[2]), float(drag_k), _ptr3(fm), _ptr3(fp), _ptr3(sm), _ptr3(sp),
        _p(fl, ctypes.c_uint8), float(rtol), int(maxiter), _ptr3(lv), _ptr3(lsv), _ptr3(lm),
        _ptr3(lp), _ptr3(lsm), _ptr3(lsp))
    _check(rc, "grid_update_adjoint")
    return (lm, lp, lsm, lsp) if solid else (lm, lp)


def g2p_adjoint(x, gv, R, n, dx, dt, lc_out, lx_out):
    """Adjoint of G2P + advection: returns (lv (3 grids), lx (3, P))."""
    D = ctypes.c_double
    x = _f64(x)
    gv = [_f64(a) for a in gv]
    lc_out = _f64(lc_out)
    lx_out = _f64(lx_out)
    P = x.shape[1]
    lv = [np.zeros_like(a) for a in gv]
    lx = np.zeros((3, P))
    rc = _load().or_g2p_adjoint(P, _p(x[0], D), _p(x[1], D), _p(x[2], D),
                                *[_p(a, D) for a in gv], R, int(n[0]), int(n[1]), int(n[2]),
                                float(dx), float(dt), _p(lc_out, D), _p(lx_out[0], D),
                                _p(lx_out[1], D), _p(lx_out[2], D), *[_p(a, D) for a in lv],
                                _p(lx[0], D), _p(lx[1], D), _p(lx[2], D))
    _check(rc, "g2p_adjoint")
    return lv, lx


def pcg_project(n, dx, dt, rho, fluid, v, rtol=1e-6, maxiter=1000):
    """Jacobi-PCG projection.  fluid: (n_z, n_y, n_x) bool.  Returns
    (v_projected (3 grids), pressure (n_z, n_y, n_x), iterations)."""
    D = ctypes.c_double
    v = [_f64(a).copy() for a in v]
    fl = np.ascontiguousarray(fluid, dtype=np.uint8)
    pr = np.zeros((int(n[2]), int(n[1]), int(n[0])))
    it = _load().or_pcg_project(int(n[0]), int(n[1]), int(n[2]), float(dx), float(dt),
                                float(rho), _p(fl, ctypes.c_uint8), *[_p(a, D) for a in v],
                                _p(pr, D), float(rtol), int(maxiter))
    _check(it, "pcg_project")
    return v, pr, it


def step(x, mass, coeff, n, dx, dt, gravity=(0.0, -9.81, 0.0), mass_abs=None):
    """One single-phase transfer step without projection: P2G, grid update, G2P.
    Returns (coeff_new, x_new, (gm, gp, gv))."""
    R = np.asarray(coeff).shape[1]
    gm, gp = p2g(x, mass, coeff, n, dx, mass_abs=mass_abs)
    gv = grid_update(n, dt, gravity, gm, gp)
    c_new, x_new = g2p(x, gv, R, n, dx, dt)
    return c_new, x_new, (gm, gp, gv)


def fabric_forces(x, mass, coeff, vertex_id, m, h, k_stretch, k_shear, k_bend, damping, dt,
                  mass_abs=None):
    """Mass-spring stand-in on the sheet's vertex lattice: returns the
    coefficients with mode 0 (the velocity) of every vertex advanced by
    dt f / (m + m_abs).  vertex_id: lattice id per particle (>= m^2: no
    springs)."""
    D = ctypes.c_double
    x = _f64(x)
    mass = _f64(mass)
    mabs = None if mass_abs is None else _f64(mass_abs)
    c = _f64(coeff).copy()
    ids = np.ascontiguousarray(vertex_id, dtype=np.uint32)
    P = x.shape[1]
    _load().or_fabric_forces(P, _p(x[0], D), _p(x[1], D), _p(x[2], D), _p(mass, D),
                             _p(mabs, D), _p(c, D), int(c.shape[1]), _p(ids, ctypes.c_uint32),
                             int(m), float(h), float(k_stretch), float(k_shear), float(k_bend),
                             float(damping), float(dt))
    return c


def absorb(xf32, fmass, xs32, smass, mass_abs, n, dx, dt, rate, capacity, max_fraction):
    """Absorption stand-in per cell: returns (fluid masses, solid m_abs)."""
    D = ctypes.c_double
    xf32 = _f32(xf32)
    xs32 = _f32(xs32)
    fm = _f64(fmass).copy()
    ma = _f64(mass_abs).copy()
    sm = _f64(smass)
    F = ctypes.c_float
    _load().or_absorb(xf32.shape[1], _p(xf32[0], F), _p(xf32[1], F), _p(xf32[2], F), _p(fm, D),
                      xs32.shape[1], _p(xs32[0], F), _p(xs32[1], F), _p(xs32[2], F), _p(sm, D),
                      _p(ma, D), int(n[0]), int(n[1]), int(n[2]), float(dx), float(dt),
                      float(rate), float(capacity), float(max_fraction))
    return fm, ma

"""Mutation check of the oracle's pins.

Each entry below plants one plausible mistake in a copy of the oracle package
-- in polypic_oracle.c, its ctypes wrappers or the all-pairs evaluator: a
dropped term, a flipped sign, a wrong index or operand, a transposed matrix,
a missing guard, wall or clamp -- compiles the copy, and runs the host pins
(tests/test_oracle_*.py and tests/test_slot_layout.py) against it in a child
process.  Every mutant must make the pins fail:
a mistake anywhere in the oracle's arithmetic that the pins let through would
leave the GPU parity tests comparing against an unverified reference.  A
control run of the unmodified copy must pass, so that a broken harness cannot
count as a caught mutant.

The mutants cover the cell key and the stable sort, the quadratic B-spline and
its derivative, the staggered stencil and its moments (Eq 14's
orthogonalisation), the mode order and mode values (Eq 11), P2G (Eqs 1-5, 13,
15-18), Eq 12's affine map, the grid update (gravity, drag, walls, empty
faces), the G2P fit with its guard and the advection clamp (Section 3.3),
Eq 10's gradient form, the three adjoints with their position terms, the
pressure projection, and the fabric and absorption stand-ins.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "polypic_oracle.c")
PINS = ["tests/test_oracle_basis.py", "tests/test_oracle_transfers.py",
        "tests/test_oracle_update_adjoint.py", "tests/test_oracle_fabric.py",
        "tests/test_slot_layout.py"]

# (name, text in polypic_oracle.c, replacement, which occurrence (0-based))
MUTANTS = [
    # cell key and sort
    ("key transposed", "key[p] = (uint32_t)(((int64_t)k * ny + j) * nx + i);",
     "key[p] = (uint32_t)(((int64_t)i * ny + j) * nz + k);", 0),
    ("sort not stable", "for (int64_t p = 0; p < np; ++p) perm[fill[key[p]]++] = (uint32_t)p;",
     "for (int64_t p = np - 1; p >= 0; --p) perm[fill[key[p]]++] = (uint32_t)p;", 0),
    ("upper clamp off by one", "if (f > (float)(n - 1)) return n - 1;",
     "if (f > (float)(n - 1)) return n - 2;", 0),
    ("no upper clamp", "if (f > (float)(n - 1)) return n - 1;\n", "", 0),
    ("cell decided in FP64", "float v = x * inv_dx;\n    float f = floorf(v);",
     "float f = (float)floor((double)x / (1.0 / (double)inv_dx));", 0),
    ("cell starts miss the last cell", "for (uint32_t k = 0; k < nkeys; ++k) cell_start[k + 1] += cell_start[k];",
     "for (uint32_t k = 0; k + 1 < nkeys; ++k) cell_start[k + 1] += cell_start[k];", 0),
    # kernel N and dN/dr
    ("outer weight halved", "{ double b = 1.5 - a; return 0.5 * b * b; }",
     "{ double b = 1.5 - a; return 0.25 * b * b; }", 0),
    ("inner derivative sign", "if (a < 0.5) return -2.0 * r;", "if (a < 0.5) return 2.0 * r;", 0),
    ("outer derivative sign", "if (a < 1.5) return -sgn * (1.5 - a);",
     "if (a < 1.5) return sgn * (1.5 - a);", 0),
    # stencil, moments, basis
    ("stagger swapped", "double X = xb / dx - (face ? 0.0 : 0.5);",
     "double X = xb / dx - (face ? 0.5 : 0.0);", 0),
    ("offset sign", "s->z[k] = (node - X) * dx;", "s->z[k] = (X - node) * dx;", 0),
    ("kappa sign", "s->kappa = mu[3] / mu[2];", "s->kappa = -mu[3] / mu[2];", 0),
    ("moment derivative sign",
     "dmu[n] += s->dw[k] * zpow[n] - (n > 0 ? (double)n * s->w[k] * zpow[n - 1] : 0.0);",
     "dmu[n] += s->dw[k] * zpow[n] + (n > 0 ? (double)n * s->w[k] * zpow[n - 1] : 0.0);", 0),
    ("guard band narrowed", "s->guard = q32 < 0x1p-10f ? 1 : 0;",
     "s->guard = q32 < 0x1p-12f ? 1 : 0;", 0),
    ("quadratic basis constant", "return z * z - s->kappa * z - s->mu2;",
     "return z * z - s->kappa * z + s->mu2;", 0),
    ("basis derivative drops dkappa",
     "return 2.0 * z * dz - s->dkappa * z - s->kappa * dz - s->dmu2;",
     "return 2.0 * z * dz - s->kappa * dz - s->dmu2;", 0),
    ("upper edge accepted", "vx >= 1.0f && vx < (float)(nx - 1)",
     "vx >= 1.0f && vx <= (float)(nx - 1)", 0),
    ("lower edge refused", "vx >= 1.0f && vx < (float)(nx - 1)",
     "vx > 1.0f && vx < (float)(nx - 1)", 0),
    # (flipping the sign of the mu3 dmu2 term of dkappa would be equivalent:
    # mu2 = dx^2 / 4 at every t, so dmu2 = 0)
    ("kappa derivative dropped",
     "s->dkappa = (dmu[3] * mu[2] - mu[3] * dmu[2]) / (mu[2] * mu[2]);",
     "s->dkappa = (0.0 * dmu[3] * mu[2] - mu[3] * dmu[2]) / (mu[2] * mu[2]);", 0),
    ("basis derivative halves z^2", "return 2.0 * z * dz - s->dkappa",
     "return z * dz - s->dkappa", 0),
    ("valid region widened", "return vx >= 1.0f && vx < (float)(nx - 1) &&",
     "return vx >= 0.5f && vx < (float)(nx - 1) &&", 0),
    # mode order and values
    ("multilinear modes reordered", "{1, 1, 0}, {1, 0, 1}, {0, 1, 1}, {1, 1, 1}};",
     "{1, 0, 1}, {1, 1, 0}, {0, 1, 1}, {1, 1, 1}};", 0),
    ("quadratic modes in (a, b, c) order",
     "for (int c = 0; c < 3; ++c)\n        for (int b = 0; b < 3; ++b)\n"
     "            for (int a = 0; a < 3; ++a)",
     "for (int a = 0; a < 3; ++a)\n        for (int b = 0; b < 3; ++b)\n"
     "            for (int c = 0; c < 3; ++c)", 0),
    ("mode value wrong degree", "basis_f(&st[1], g_modes[r][1], zz[1]) *",
     "basis_f(&st[1], g_modes[r][2], zz[1]) *", 0),
    # Eq 12 affine map
    ("affine C transposed", "coeff[((int64_t)a * R + 1 + b) * np + p] : 0.0;",
     "coeff[((int64_t)b * R + 1 + a) * np + p] : 0.0;", 0),
    ("affine map transposed", "zm[i] = M[i][0] * zz[0] + M[i][1] * zz[1] + M[i][2] * zz[2];",
     "zm[i] = M[0][i] * zz[0] + M[1][i] * zz[1] + M[2][i] * zz[2];", 0),
    ("affine minus dt", "A[a][b] = (a == b ? 1.0 : 0.0) + dt * c;",
     "A[a][b] = (a == b ? 1.0 : 0.0) - dt * c;", 0),
    # P2G
    ("P2G drops m_abs", "double mt = mass[p] + (mass_abs ? mass_abs[p] : 0.0);\n    double M[3][3];",
     "double mt = mass[p];\n    double M[3][3];", 0),
    ("P2G coefficient layout", "S += coeff[((int64_t)a * R + r) * np + p] * mode_value(st, r, zz);",
     "S += coeff[((int64_t)r * 3 + a) * np + p] * mode_value(st, r, zz);", 0),
    ("P2G mass unweighted", "gm[a][idx] += mt * w;", "gm[a][idx] += w;", 0),
    ("P2G momentum unweighted", "gp[a][idx] += mt * w * S;", "gp[a][idx] += w * S;", 0),
    ("P2G threads sum the wrong grid", "for (size_t i = 0; i < cnt[a]; ++i) gp[a][i] += base[cnt[a] + i];",
     "for (size_t i = 0; i < cnt[a]; ++i) gp[a][i] += base[i];", 0),
    # grid update
    ("gravity sign", "vf += dt * g[a];", "vf -= dt * g[a];", 0),
    ("drag weights swapped", "vf = mean + ms / (mf + ms) * u;", "vf = mean + mf / (mf + ms) * u;", 0),
    ("upper wall kept", "if (ia == 0 || ia == d[a] - 1) v[((size_t)k * d[1] + j) * d[0] + i] = 0.0;",
     "if (ia == 0) v[((size_t)k * d[1] + j) * d[0] + i] = 0.0;", 0),
    ("solid walls kept", "if (solid) wall_zero(a, d, sv[a]);", "", 0),
    ("empty face not zero", "double vf = fm[a][i] > 0.0 ? fp[a][i] / fm[a][i] : 0.0;",
     "double vf = fm[a][i] > 0.0 ? fp[a][i] / fm[a][i] : 1.0;", 0),
    # G2P fit, guard, advection, Eq 10
    ("fit denominator unsquared", "den[r] += w * s * s;\n                        }\n"
     "                        if (apic_grad)",
     "den[r] += w * s;\n                        }\n                        if (apic_grad)", 0),
    ("fit guard removed", "double c = guarded ? 0.0 : num[r] / den[r];",
     "double c = num[r] / den[r];", 0),
    ("fit guard on the wrong axis", "(g_modes[r][1] == 2 && st[1].guard) ||",
     "(g_modes[r][1] == 2 && st[0].guard) ||", 0),
    ("clamp margin", "double lo = 1.5 * dx, hi = ((double)n3[a] - 1.5) * dx;\n"
     "            double xn = pos[a] + dt * vp[a];",
     "double lo = 1.0 * dx, hi = ((double)n3[a] - 1.5) * dx;\n"
     "            double xn = pos[a] + dt * vp[a];", 0),
    ("advection sign", "double xn = pos[a] + dt * vp[a];", "double xn = pos[a] - dt * vp[a];", 0),
    ("clamp upper margin", "double lo = 1.5 * dx, hi = ((double)n3[a] - 1.5) * dx;\n"
     "            double xn = pos[a] + dt * vp[a];",
     "double lo = 1.5 * dx, hi = ((double)n3[a] - 1.0) * dx;\n"
     "            double xn = pos[a] + dt * vp[a];", 0),
    ("grad w in shifted mode slots", "if (apic_grad && r >= 1) c = gradw[r - 1];",
     "if (apic_grad && r >= 1) c = gradw[r % 3];", 0),
    ("grad w on the wrong axis", "gradw[1] += st[0].w[kx] * st[1].dw[ky] * st[2].w[kz] * v;",
     "gradw[1] += st[0].dw[kx] * st[1].w[ky] * st[2].w[kz] * v;", 0),
    # P2G adjoint
    ("P2G adjoint drops the mass", "acc_c[r] += mt * w * s * LP;", "acc_c[r] += w * s * LP;", 0),
    ("P2G adjoint drops the mass term", "lpos[b][p] += mt * (dwb * (S * LP + LM) + w * dS * LP);",
     "lpos[b][p] += mt * (dwb * (S * LP) + w * dS * LP);", 0),
    ("P2G adjoint offset derivative sign", "ds *= (e == b) ? basis_df(&st[e], deg, zz[e], -1.0)",
     "ds *= (e == b) ? basis_df(&st[e], deg, zz[e], 1.0)", 0),
    ("P2G adjoint weight derivative on the wrong axis",
     "dwb *= (e == b) ? st[e].dw[k3[e]] : st[e].w[k3[e]];",
     "dwb *= (e != b) ? st[e].dw[k3[e]] : st[e].w[k3[e]];", 0),
    # G2P adjoint
    ("G2P adjoint weight derivative on the wrong axis",
     "dwb *= (e == b) ? st[e].dw[k3[e]] : st[e].w[k3[e]];",
     "dwb *= (e != b) ? st[e].dw[k3[e]] : st[e].w[k3[e]];", 1),
    ("G2P adjoint ignores the clamp", "if (xn >= lo && xn <= hi) {", "if (1) {", 0),
    # (halving the 2 w s ds term of dden would be an equivalent mutant: summed
    # over the stencil it vanishes, since d f_a / d x_p lies in the span of
    # the lower-degree factors, to which f_a is orthogonal)
    ("G2P adjoint denominator drops dw", "dden[r][b] += dwb * s * s + 2.0 * w * s * ds;",
     "dden[r][b] += 2.0 * w * s * ds;", 0),
    ("G2P adjoint numerator drops ds", "dnum[r][b] += (dwb * s + w * ds) * v;",
     "dnum[r][b] += (dwb * s) * v;", 0),
    ("G2P adjoint advection without dt", "mu[0] += dt * lpo[a][p];", "mu[0] += lpo[a][p];", 0),
    ("G2P adjoint quotient rule sign", "lpos[b][p] += mu[r] * (dnum[r][b] - c * dden[r][b]) / den[r];",
     "lpos[b][p] += mu[r] * (dnum[r][b] + c * dden[r][b]) / den[r];", 0),
    ("G2P adjoint position guard removed", "if (guarded || mu[r] == 0.0) continue;",
     "if (mu[r] == 0.0) continue;", 0),
    ("G2P adjoint grid guard removed", "if (guarded) continue;\n                        acc +=",
     "acc +=", 0),
    ("G2P adjoint wrong denominator", "acc += mu[r] * w * mode_value(st, r, zz) / den[r];",
     "acc += mu[r] * w * mode_value(st, r, zz) / den[0];", 0),
    # pressure projection
    ("projection rhs sign", "b[c] = -(rho * dx * dx / dt) * div;", "b[c] = (rho * dx * dx / dt) * div;", 0),
    ("projection gradient sign", "dt / (rho * dx) * (pressure[ch] - pressure[cl]);",
     "dt / (rho * dx) * (pressure[cl] - pressure[ch]);", 0),
    ("projection skips fluid-air faces", "if (!fluid[cl] && !fluid[ch]) continue;",
     "if (!fluid[cl] || !fluid[ch]) continue;", 0),
    ("Laplacian with Dirichlet walls", "diag[c] = (double)((i > 0) + (i < nx - 1) + (j > 0)",
     "diag[c] = 6.0 + 0.0 * (double)((i > 0) + (i < nx - 1) + (j > 0)", 0),
    ("Laplacian misses a neighbour", "if (k < nz - 1 && fluid[CIDX(i, j, k + 1)]) s -= src[CIDX(i, j, k + 1)];",
     "", 0),
    # grid update adjoint
    ("update adjoint projection sign", "lf[a][((size_t)k * d[1] + j) * d[0] + i] += ql - qh;",
     "lf[a][((size_t)k * d[1] + j) * d[0] + i] += qh - ql;", 0),
    ("update adjoint divergence sign", "if (ijk[a] > 0) acc += lf", "if (ijk[a] > 0) acc -= lf", 0),
    ("update adjoint wall faces in G^T", "if (ijk[a] + 1 < n3[a]) acc -= lf", "acc -= lf", 0),
    ("update adjoint walls kept", "double lvf = wall ? 0.0 : lf[a][idx];", "double lvf = lf[a][idx];", 0),
    ("update adjoint drag weights", "double lf_new = lvf * (wb + wa / Dd) + lvs * (wb - wb / Dd);",
     "double lf_new = lvf * (wa + wb / Dd) + lvs * (wb - wb / Dd);", 0),
    ("update adjoint drops du/dm", "dmf = lvf * (mean_f + wa_f * u + wa * u_f)",
     "dmf = lvf * (mean_f + wa_f * u)", 0),
    ("update adjoint mean derivative sign", "mean_s = (vs - mean) / M;", "mean_s = (mean - vs) / M;", 0),
    ("update adjoint solid row", "double ls_new = lvf * (wa - wa / Dd) + lvs * (wa + wb / Dd);",
     "double ls_new = lvf * (wa - wa / Dd) + lvs * (wa + wa / Dd);", 0),
    ("update adjoint division sign", "lfm[a][idx] = dmf - lvf * fp[a][idx] / (mf * mf);",
     "lfm[a][idx] = dmf + lvf * fp[a][idx] / (mf * mf);", 0),
    ("update adjoint keeps the solid walls", "double lvs = (solid && !wall) ? lsv[a][idx] : 0.0;",
     "double lvs = solid ? lsv[a][idx] : 0.0;", 0),
    ("update adjoint through empty faces", "lfp[a][idx] = 0.0;", "lfp[a][idx] = lvf;", 0),
    ("update adjoint without gravity", "double vf = fp[a][idx] / mf + dt * g[a];",
     "double vf = fp[a][idx] / mf;", 0),
    ("update adjoint drops the drag mass term", "lsm[a][idx] = dms - lvs * sp[a][idx] / (ms * ms);",
     "lsm[a][idx] = -lvs * sp[a][idx] / (ms * ms);", 0),
    # fabric and absorption stand-ins
    ("shear rest length", "double L0 = s < 4 ? h : s < 8 ? h * sqrt(2.0) : 2.0 * h;",
     "double L0 = s < 4 ? h : s < 8 ? h : 2.0 * h;", 0),
    ("damper sign", "f[a] += (kk * (L - L0) + damping * rv) * d[a] / L;",
     "f[a] += (kk * (L - L0) - damping * rv) * d[a] / L;", 0),
    ("spring direction", "d[a] = pos[a][q] - pos[a][p];", "d[a] = pos[a][p] - pos[a][q];", 0),
    ("no bending springs", "for (int s = 0; s < 12; ++s) {", "for (int s = 0; s < 8; ++s) {", 0),
    ("fabric ignores m_abs",
     "double mt = mass[p] + (mass_abs ? mass_abs[p] : 0.0);\n        for (int a = 0; a < 3; ++a) dv",
     "double mt = mass[p];\n        for (int a = 0; a < 3; ++a) dv", 0),
    ("springs on element particles", "if (id[p] >= (uint32_t)nv) continue;", "", 0),
    ("bending stiffness", "double kk = s < 4 ? k_stretch : s < 8 ? k_shear : k_bend;",
     "double kk = s < 4 ? k_stretch : s < 8 ? k_shear : k_shear;", 0),
    ("absorption taken equally", "if (D > 0.0) fmass[q] -= fmass[q] * D / Mf[c];",
     "if (D > 0.0) fmass[q] -= D / 2.0;", 0),
    ("absorption without capacity", "d[p] = room > 0.0 ? (want < room ? want : room) : 0.0;",
     "d[p] = want;", 0),
    ("absorption without the fluid limit",
     "double D = Dd[c] < max_fraction * Mf[c] ? Dd[c] : max_fraction * Mf[c];\n"
     "        if (D > 0.0) mass_abs",
     "double D = Dd[c];\n        if (D > 0.0) mass_abs", 0),
]

# The same for the oracle's Python layer (the ctypes wrappers, the step they
# compose, and the all-pairs NumPy evaluator the stencil oracle is pinned to):
# (name, file in oracle/, text, replacement, which occurrence)
PY_MUTANTS = [
    ("grid arrays x slowest", "__init__.py", "    return (d[2], d[1], d[0])",
     "    return (d[0], d[1], d[2])", 0),
    ("keys with the axes swapped", "__init__.py",
     "_p(x32[2], ctypes.c_float), int(n[0]), int(n[1]), int(n[2]),",
     "_p(x32[2], ctypes.c_float), int(n[1]), int(n[0]), int(n[2]),", 0),
    ("gravity components swapped", "__init__.py",
     "float(gravity[1]), float(gravity[2]), float(drag_k),",
     "float(gravity[2]), float(gravity[1]), float(drag_k),", 0),
    ("step fits the momentum", "__init__.py", "    c_new, x_new = g2p(x, gv, R, n, dx, dt)",
     "    c_new, x_new = g2p(x, gp, R, n, dx, dt)", 0),
    ("affine map with -dt", "__init__.py",
     "int(bool(map_affine)), float(dt), *[_p(g, D) for g in gm],",
     "int(bool(map_affine)), float(-dt), *[_p(g, D) for g in gm],", 0),
    ("absorption limits swapped", "__init__.py",
     "float(rate), float(capacity), float(max_fraction))",
     "float(rate), float(max_fraction), float(capacity))", 0),
    ("spring families swapped", "__init__.py",
     "float(k_stretch), float(k_shear), float(k_bend),",
     "float(k_stretch), float(k_bend), float(k_shear),", 0),
    ("all-pairs inner weight", "bruteforce.py", "np.where(a < 0.5, 0.75 - a * a,",
     "np.where(a < 0.5, 0.75 - 0.5 * a * a,", 0),
    ("all-pairs kappa inverted", "bruteforce.py", "    kappa = mu3 / mu2\n",
     "    kappa = mu2 / mu3\n", 0),
    ("all-pairs map transposed", "bruteforce.py", 'xi = np.einsum("bc,ckji->bkji", M, Z)',
     'xi = np.einsum("cb,ckji->bkji", M, Z)', 0),
    ("all-pairs C transposed", "bruteforce.py", "C[:, lin[abc]] = coeff[:, r, p]",
     "C[lin[abc], :] = coeff[:, r, p]", 0),
    ("all-pairs fit denominator", "bruteforce.py",
     "den = np.tensordot(s * s, w, axes=([1, 2, 3], [0, 1, 2]))",
     "den = np.tensordot(s, w, axes=([1, 2, 3], [0, 1, 2]))", 0),
    ("all-pairs mode degrees swapped", "bruteforce.py",
     'np.einsum("k,j,i->kji", ax[2][1][c], ax[1][1][b], ax[0][1][a])',
     'np.einsum("k,j,i->kji", ax[2][1][a], ax[1][1][b], ax[0][1][c])', 0),
]

ORACLE = os.path.join(ROOT, "oracle")


def _mutate(text, old, new, occurrence):
    at = -1
    for _ in range(occurrence + 1):
        at = text.find(old, at + 1)
        assert at >= 0, f"text not found in the oracle (occurrence {occurrence}): {old!r}"
    return text[:at] + new + text[at + len(old):]


def _jobs():
    """name -> (file in oracle/, mutated text), the control first."""
    with open(SRC) as f:
        jobs = {"control": ("polypic_oracle.c", f.read())}
    for name, old, new, occ in MUTANTS:
        jobs[name] = ("polypic_oracle.c", _mutate(jobs["control"][1], old, new, occ))
    for name, fname, old, new, occ in PY_MUTANTS:
        with open(os.path.join(ORACLE, fname)) as f:
            jobs[name] = (fname, _mutate(f.read(), old, new, occ))
    return jobs


def _run(workdir, fname, text):
    """A copy of oracle/ in workdir with `fname` replaced by `text`, compiled
    there; the pins run against it (first on the path) in a child process.
    Returns (exit code, last lines of the output)."""
    pkg = os.path.join(workdir, "oracle")
    shutil.copytree(ORACLE, pkg, ignore=shutil.ignore_patterns("*.so", "*.tmp*", "__pycache__"))
    with open(os.path.join(pkg, fname), "w") as f:
        f.write(text)
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "--noconftest",
           "-W", "ignore::pytest.PytestUnknownMarkWarning", *[os.path.join(ROOT, t) for t in PINS]]
    env = dict(os.environ, OMP_NUM_THREADS="1", PYTHONDONTWRITEBYTECODE="1",
               PYTHONPATH=os.pathsep.join([workdir, ROOT]))
    try:
        r = subprocess.run(cmd, cwd=workdir, capture_output=True, text=True, timeout=900, env=env)
    except subprocess.TimeoutExpired:
        return None, "timed out"
    tail = "\n".join((r.stdout + r.stderr).strip().splitlines()[-3:])
    return r.returncode, tail


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    base = str(tmp_path_factory.mktemp("oracle_mutants"))
    jobs = _jobs()
    names = list(jobs)
    workers = max(1, min(len(names), os.cpu_count() or 1))
    with ThreadPoolExecutor(max_workers=workers) as ex:
        futs = {n: ex.submit(_run, os.path.join(base, f"m{i:02d}"), *jobs[n])
                for i, n in enumerate(names)}
        res = {n: futs[n].result() for n in names}
    shutil.rmtree(base, ignore_errors=True)
    return res


def test_mutants_are_distinct_and_found():
    names = [m[0] for m in MUTANTS] + [m[0] for m in PY_MUTANTS]
    assert len(set(names)) == len(names) and "control" not in names
    jobs = _jobs()
    for name in names:
        fname, text = jobs[name]
        with open(os.path.join(ORACLE, fname)) as f:
            assert text != f.read(), name


def test_unmodified_copy_passes_the_pins(outcomes):
    rc, tail = outcomes["control"]
    assert rc == 0, tail


@pytest.mark.parametrize("name", [m[0] for m in MUTANTS] + [m[0] for m in PY_MUTANTS])
def test_pins_catch_the_mutant(outcomes, name):
    rc, tail = outcomes[name]
    assert rc not in (0, None), f"{name}: the pins did not catch it ({tail})"

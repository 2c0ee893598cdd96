/*
 * polypic_oracle.c -- plain, slow FP64 CPU oracle for the PolyPIC transfers.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls
 * this file: only tests/, the smoke check and the CPU-baseline leg of the
 * benchmark use it.  It shares no code, header, table or constant with the CUDA
 * library; the two are written independently from the paper's equations.
 *
 * Paper: "Using The Polynomial Particle-in-Cell Method for Liquid-Fabric
 * Interaction" (arXiv 2308.01060).
 *
 *   Section 3.1, Eqs 1-5   PIC particle-to-grid (P2G) of mass and momentum
 *   Section 3.1, Eqs 6-8   PIC grid-to-particle (G2P), read per component
 *   Section 3.2, Eqs 9-10  APIC transfer and its grad-w velocity derivative
 *   Section 3.3, Eq 11     monomial modes s(z) = prod z_b^{i_b}
 *   Section 3.3, Eq 12     affine map xi (optional here, flag `map`)
 *   Section 3.3, Eq 13     PolyPIC P2G with N_r modes
 *   Section 3.3, Eq 14     orthogonalised quadratic factor g_b
 *   Section 3.4, Eqs 15-20 fluid and solid (absorbed-mass) transfers
 *
 * Everything is written the obvious way: loops over particles, grids and the
 * 3x3x3 stencil nodes, every mode value s_r evaluated directly at every node,
 * every least-squares denominator d_r summed directly as sum_i w_i s_r(z_i)^2.
 * There is no sum factorisation, no blocking and no closed-form shortcut.
 *
 * Discrete decisions (a particle's cell, the lowest stencil node and the
 * near-degenerate quadratic guard) are taken in FP32 from the FP32 position,
 * exactly as the library documents them, so that both sides take the same
 * decision; all arithmetic after the decision is FP64.
 *
 * Readings taken where the paper is silent or garbled (the library takes the
 * same ones):
 *   - N(x) is the quadratic B-spline (Eq 14's dx^2/4 is its second moment).
 *   - Eq 14's printed symbols are read as g(z) = z^2 - (mu3/mu2) z - mu2, the
 *     Gram-Schmidt orthogonalisation of z^2 against {1, z} under the 1-D
 *     B-spline weights (mu_n = sum_k w_k z_k^n), z = x_i - x_p.
 *   - Modes are evaluated with the particle's current position (constant map)
 *     unless `map` = 1, which applies Eq 12's affine map to the offsets.
 *   - If q = 1 - 4t^2 < 2^-10 on an axis (t = particle offset from the middle
 *     stencil node, in cells), the G2P fit sets the coefficient of every mode
 *     with a quadratic factor on that axis to 0.
 *   - Eqs 6-8 are read per component: v_pa = sum_i w_ipa v~_ia.
 *   - Eq 20's denominator is the node total sum_p (m_s,p + m_abs,p) w_ipa.
 *   - Advection is forward Euler with v_p = c_p0, clamped to
 *     [1.5 dx, (n - 1.5) dx] per axis instead of deleting particles.
 *
 * Build: plain C99, -O2 -ffp-contract=off (no fused multiply-add, so the FP32
 * decisions round exactly as documented), -fopenmp for the optional host
 * threads of P2G and G2P (or_set_threads; one thread by default).  Callers
 * pass flat arrays.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_ERR_ARG (-1)
#define OR_ERR_DOMAIN (-2)
#define OR_ERR_NOT_CONVERGED (-3)

/* ------------------------------------------------------------------------ */
/* Quadratic B-spline kernel N(r) and dN/dr (Section 3.1, w_ipa = N(x_p - x_ia)) */

static double bspline2(double r)
{
    double a = fabs(r);
    if (a < 0.5) return 0.75 - a * a;
    if (a < 1.5) { double b = 1.5 - a; return 0.5 * b * b; }
    return 0.0;
}

static double bspline2_deriv(double r)
{
    double a = fabs(r), sgn = r < 0.0 ? -1.0 : 1.0;
    if (a < 0.5) return -2.0 * r;
    if (a < 1.5) return -sgn * (1.5 - a);
    return 0.0;
}

/* ------------------------------------------------------------------------ */
/* Canonical mode order (Eq 11 with the Eq 14 substitution): r <-> (a,b,c),
 * the per-axis degrees along x, y, z.  r = 0: (000); r = 1..3: (100), (010),
 * (001); r = 4..7: (110), (101), (011), (111); r = 8..26: the remaining
 * triples with a 2 in them, in lexicographic order of (c, b, a).  Section 3.3
 * counts the 2^d multilinear modes first, so N_r = 1, 4, 8, 27 are prefixes. */

static int g_modes[27][3];
static int g_modes_ready = 0;

static void build_modes(void)
{
    if (g_modes_ready) return;
    static const int first8[8][3] = {
        {0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1},
        {1, 1, 0}, {1, 0, 1}, {0, 1, 1}, {1, 1, 1}};
    int r = 0;
    for (; r < 8; ++r) {
        g_modes[r][0] = first8[r][0];
        g_modes[r][1] = first8[r][1];
        g_modes[r][2] = first8[r][2];
    }
    for (int c = 0; c < 3; ++c)
        for (int b = 0; b < 3; ++b)
            for (int a = 0; a < 3; ++a)
                if (a == 2 || b == 2 || c == 2) {
                    g_modes[r][0] = a; g_modes[r][1] = b; g_modes[r][2] = c;
                    ++r;
                }
    g_modes_ready = 1;
}

void or_mode_abc(int r, int *abc)
{
    build_modes();
    abc[0] = g_modes[r][0]; abc[1] = g_modes[r][1]; abc[2] = g_modes[r][2];
}

/* ------------------------------------------------------------------------ */
/* Cell index and stable sort (an implementation device; the paper has none).
 *
 * cell (i,j,k): i = clamp(floor(fl(x * inv_dx)), 0, n_x - 1) with the product
 * rounded once in FP32 and inv_dx = (float)(1.0 / dx); the key of a particle
 * is the plain cell index (k * n_y + j) * n_x + i, x fastest.              */

static float inv_dx_f32(double dx) { return (float)(1.0 / dx); }

static int cell_of(float x, float inv_dx, int n)
{
    float v = x * inv_dx;
    float f = floorf(v);
    if (!(f >= 0.0f)) return 0;               /* also catches NaN */
    if (f > (float)(n - 1)) return n - 1;
    return (int)f;
}

void or_keys(int64_t np, const float *x, const float *y, const float *z,
             int nx, int ny, int nz, double dx, uint32_t *key)
{
    float inv = inv_dx_f32(dx);
    for (int64_t p = 0; p < np; ++p) {
        int i = cell_of(x[p], inv, nx), j = cell_of(y[p], inv, ny), k = cell_of(z[p], inv, nz);
        key[p] = (uint32_t)(((int64_t)k * ny + j) * nx + i);
    }
}

/* Stable counting sort: perm[j] = index of the j-th particle in (key, index)
 * order; cell_start[k] = number of particles with key < k (so the first
 * sorted slot with key >= k), cell_start[nkeys] = np. */
void or_stable_sort(int64_t np, const uint32_t *key, uint32_t nkeys,
                    uint32_t *perm, uint32_t *cell_start)
{
    memset(cell_start, 0, sizeof(uint32_t) * ((size_t)nkeys + 1));
    for (int64_t p = 0; p < np; ++p) cell_start[key[p] + 1] += 1;
    for (uint32_t k = 0; k < nkeys; ++k) cell_start[k + 1] += cell_start[k];
    uint32_t *fill = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)nkeys + 1));
    memcpy(fill, cell_start, sizeof(uint32_t) * ((size_t)nkeys + 1));
    for (int64_t p = 0; p < np; ++p) perm[fill[key[p]]++] = (uint32_t)p;
    free(fill);
}

/* ------------------------------------------------------------------------ */
/* One-axis stencil of a particle on one face grid.
 *
 * Face grid a holds velocity component a at ((i + o_x) dx, (j + o_y) dx,
 * (k + o_z) dx) with o_b = 0 if b == a and 1/2 otherwise (the MAC grid of
 * Section 3).  Along one axis the particle touches nodes base..base+2 where
 * base = floor(X - 1/2), X = x/dx - o (FP32 decision).  Weights are
 * N(X - node), offsets z = x_node - x_p.  The 1-D basis (Eq 11 with Eq 14):
 * f0 = 1, f1 = z, f2 = z^2 - kappa z - mu2 with mu_n = sum_k w_k z_k^n and
 * kappa = mu3/mu2 (Gram-Schmidt of z^2 against {1, z}; sum w = 1 and
 * sum w z = 0 for this kernel, which the tests pin).                        */

typedef struct {
    int base;
    double w[3], dw[3];   /* weights and dw/dx_p */
    double z[3];          /* node - particle (physical) */
    double mu2, kappa;    /* g(z) = z^2 - kappa z - mu2 */
    double dmu2, dkappa;  /* derivatives w.r.t. x_p */
    int guard;            /* 1: quadratic factor on this axis is suppressed in G2P */
} axis_stencil;

static void axis_stencil_eval(double xb, double dx, int face, axis_stencil *s)
{
    /* FP32 decisions, one rounding per operation */
    float xf = (float)xb;
    float v = xf * inv_dx_f32(dx);
    float X32 = face ? v : v - 0.5f;
    float fb = floorf(X32 - 0.5f);
    float t32 = X32 - (fb + 1.0f);
    float one_m = 1.0f - 2.0f * t32;
    float one_p = 1.0f + 2.0f * t32;
    float q32 = one_m * one_p;
    s->base = (int)fb;
    s->guard = q32 < 0x1p-10f ? 1 : 0;

    /* FP64 arithmetic */
    double X = xb / dx - (face ? 0.0 : 0.5);
    double mu[5] = {0, 0, 0, 0, 0}, dmu[4] = {0, 0, 0, 0};
    for (int k = 0; k < 3; ++k) {
        double node = (double)(s->base + k);
        s->w[k] = bspline2(X - node);
        s->dw[k] = bspline2_deriv(X - node) / dx;
        s->z[k] = (node - X) * dx;
    }
    for (int k = 0; k < 3; ++k) {
        double zpow[4] = {1.0, s->z[k], s->z[k] * s->z[k], s->z[k] * s->z[k] * s->z[k]};
        for (int n = 0; n < 4; ++n) {
            mu[n] += s->w[k] * zpow[n];
            /* d/dx_p of w z^n = dw z^n - n w z^(n-1), since dz/dx_p = -1 */
            dmu[n] += s->dw[k] * zpow[n] - (n > 0 ? (double)n * s->w[k] * zpow[n - 1] : 0.0);
        }
    }
    s->mu2 = mu[2];
    s->kappa = mu[3] / mu[2];
    s->dmu2 = dmu[2];
    s->dkappa = (dmu[3] * mu[2] - mu[3] * dmu[2]) / (mu[2] * mu[2]);
}

/* f_a(z) and d f_a / d x_p for the particle's axis basis; z is the (possibly
 * mapped) offset, dz its derivative w.r.t. x_p along this axis. */
static double basis_f(const axis_stencil *s, int a, double z)
{
    if (a == 0) return 1.0;
    if (a == 1) return z;
    return z * z - s->kappa * z - s->mu2;
}

static double basis_df(const axis_stencil *s, int a, double z, double dz)
{
    if (a == 0) return 0.0;
    if (a == 1) return dz;
    return 2.0 * z * dz - s->dkappa * z - s->kappa * dz - s->dmu2;
}

/* Exposed for the pins: one axis of one particle. */
int or_stencil_1d(double xb, double dx, int face, int *base, double *w, double *z,
                  double *mu2, double *kappa, int *guard)
{
    axis_stencil s;
    axis_stencil_eval(xb, dx, face, &s);
    *base = s.base;
    for (int k = 0; k < 3; ++k) { w[k] = s.w[k]; z[k] = s.z[k]; }
    *mu2 = s.mu2; *kappa = s.kappa; *guard = s.guard;
    return OR_OK;
}

/* ------------------------------------------------------------------------ */

static int in_domain(double x, double y, double zc, int nx, int ny, int nz, double dx)
{
    float inv = inv_dx_f32(dx);
    float vx = (float)x * inv, vy = (float)y * inv, vz = (float)zc * inv;
    return vx >= 1.0f && vx < (float)(nx - 1) &&
           vy >= 1.0f && vy < (float)(ny - 1) &&
           vz >= 1.0f && vz < (float)(nz - 1);
}

static void face_dims(int alpha, int nx, int ny, int nz, int d[3])
{
    d[0] = nx + (alpha == 0);
    d[1] = ny + (alpha == 1);
    d[2] = nz + (alpha == 2);
}

/* Particle p on face grid alpha: its three axis stencils. */
static void particle_stencils(double px, double py, double pz, int alpha, double dx,
                              axis_stencil st[3])
{
    axis_stencil_eval(px, dx, alpha == 0, &st[0]);
    axis_stencil_eval(py, dx, alpha == 1, &st[1]);
    axis_stencil_eval(pz, dx, alpha == 2, &st[2]);
}

/* Mode value s_r at offset z (3 components), Eq 11 with g from Eq 14. */
static double mode_value(const axis_stencil st[3], int r, const double zz[3])
{
    return basis_f(&st[0], g_modes[r][0], zz[0]) *
           basis_f(&st[1], g_modes[r][1], zz[1]) *
           basis_f(&st[2], g_modes[r][2], zz[2]);
}

/* Affine map of Eq 12 applied to the node offset: z' = (I + dt C)^-1 z, with
 * C_ab = coefficient of mode z_b for component a (the linear modes r = 1..3).
 * Falls back to the identity when |det(I + dt C)| < 1e-6.                  */
static void affine_matrix(const double *coeff, int R, int64_t np, int64_t p, double dt, double M[3][3])
{
    double A[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double c = (R >= 4) ? coeff[((int64_t)a * R + 1 + b) * np + p] : 0.0;
            A[a][b] = (a == b ? 1.0 : 0.0) + dt * c;
        }
    double det = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1])
               - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0])
               + A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
    if (fabs(det) < 1e-6) {
        for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) M[a][b] = (a == b);
        return;
    }
    M[0][0] = (A[1][1] * A[2][2] - A[1][2] * A[2][1]) / det;
    M[0][1] = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) / det;
    M[0][2] = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) / det;
    M[1][0] = (A[1][2] * A[2][0] - A[1][0] * A[2][2]) / det;
    M[1][1] = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) / det;
    M[1][2] = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) / det;
    M[2][0] = (A[1][0] * A[2][1] - A[1][1] * A[2][0]) / det;
    M[2][1] = (A[0][1] * A[2][0] - A[0][0] * A[2][1]) / det;
    M[2][2] = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) / det;
}

/* Exposed for the pins: nodes, weights, mode values and the least-squares
 * denominators d_r = sum_i w_i s_r(z_i)^2 of one particle on grid alpha.
 * node: [27][3], w: [27], s: [27][R], d: [R], guard: [3].                   */
int or_particle_modes(double px, double py, double pz, int alpha, int R,
                      double dx, int *node, double *w, double *s, double *d, int *guard)
{
    build_modes();
    axis_stencil st[3];
    particle_stencils(px, py, pz, alpha, dx, st);
    for (int r = 0; r < R; ++r) d[r] = 0.0;
    int n = 0;
    for (int kz = 0; kz < 3; ++kz)
        for (int ky = 0; ky < 3; ++ky)
            for (int kx = 0; kx < 3; ++kx, ++n) {
                double zz[3] = {st[0].z[kx], st[1].z[ky], st[2].z[kz]};
                node[3 * n + 0] = st[0].base + kx;
                node[3 * n + 1] = st[1].base + ky;
                node[3 * n + 2] = st[2].base + kz;
                w[n] = st[0].w[kx] * st[1].w[ky] * st[2].w[kz];
                for (int r = 0; r < R; ++r) {
                    s[n * R + r] = mode_value(st, r, zz);
                    d[r] += w[n] * s[n * R + r] * s[n * R + r];
                }
            }
    for (int b = 0; b < 3; ++b) guard[b] = st[b].guard;
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Host threads for P2G and G2P (1 = the plain serial loops).  With more
 * threads, G2P splits the particles between them (each particle's fit is
 * independent) and P2G gives every thread private grids that are summed in
 * thread order afterwards, so the result does not depend on timing.       */
static int g_threads = 1;

void or_set_threads(int n) { g_threads = n > 0 ? n : 1; }
int or_get_threads(void) { return g_threads; }

/* ------------------------------------------------------------------------ */
/* P2G: Eqs 1, 4 (mass), Eq 13 (PolyPIC momentum), Eqs 15-18 (phase masses).
 *   m_ia  += mt_p w_ipa
 *   mv_ia += mt_p w_ipa sum_{r<R} c_pra s_r(z_ipa)
 * mt_p = mass[p] (+ mass_abs[p] for solids, Eq 18).  Grids are zeroed first.
 * coeff: [3][R][np].  Grid a has dims face_dims(a), x fastest.
 * Returns OR_ERR_DOMAIN if a particle lies outside [dx, (n-1) dx).          */
/* The deposit of particle p into the grids gm, gp (the body of or_p2g). */
static void p2g_particle(int64_t np, int64_t p, const double *x, const double *y,
                         const double *z, const double *mass, const double *mass_abs,
                         const double *coeff, int R, int nx, int ny, int nz, double dx,
                         int map, double dt, double *const gm[3], double *const gp[3])
{
    double mt = mass[p] + (mass_abs ? mass_abs[p] : 0.0);
    double M[3][3];
    if (map == 1) affine_matrix(coeff, R, np, p, dt, M);
    for (int a = 0; a < 3; ++a) {
        int d[3]; face_dims(a, nx, ny, nz, d);
        axis_stencil st[3];
        particle_stencils(x[p], y[p], z[p], a, dx, st);
        for (int kz = 0; kz < 3; ++kz)
            for (int ky = 0; ky < 3; ++ky)
                for (int kx = 0; kx < 3; ++kx) {
                    double w = st[0].w[kx] * st[1].w[ky] * st[2].w[kz];
                    double zz[3] = {st[0].z[kx], st[1].z[ky], st[2].z[kz]};
                    if (map == 1) {
                        double zm[3];
                        for (int i = 0; i < 3; ++i)
                            zm[i] = M[i][0] * zz[0] + M[i][1] * zz[1] + M[i][2] * zz[2];
                        zz[0] = zm[0]; zz[1] = zm[1]; zz[2] = zm[2];
                    }
                    double S = 0.0;
                    for (int r = 0; r < R; ++r)
                        S += coeff[((int64_t)a * R + r) * np + p] * mode_value(st, r, zz);
                    int ix = st[0].base + kx, iy = st[1].base + ky, iz = st[2].base + kz;
                    size_t idx = ((size_t)iz * d[1] + iy) * d[0] + ix;
                    gm[a][idx] += mt * w;
                    gp[a][idx] += mt * w * S;
                }
    }
}

int or_p2g(int64_t np, const double *x, const double *y, const double *z,
           const double *mass, const double *mass_abs, const double *coeff, int R,
           int nx, int ny, int nz, double dx, int map, double dt,
           double *gm0, double *gm1, double *gm2, double *gp0, double *gp1, double *gp2)
{
    build_modes();
    if (R != 1 && R != 4 && R != 8 && R != 27) return OR_ERR_ARG;
    double *gm[3] = {gm0, gm1, gm2}, *gp[3] = {gp0, gp1, gp2};
    for (int a = 0; a < 3; ++a) {
        int d[3]; face_dims(a, nx, ny, nz, d);
        size_t cnt = (size_t)d[0] * d[1] * d[2];
        memset(gm[a], 0, cnt * sizeof(double));
        memset(gp[a], 0, cnt * sizeof(double));
    }
    for (int64_t p = 0; p < np; ++p)
        if (!in_domain(x[p], y[p], z[p], nx, ny, nz, dx)) return OR_ERR_DOMAIN;

    if (g_threads <= 1) {
        for (int64_t p = 0; p < np; ++p)
            p2g_particle(np, p, x, y, z, mass, mass_abs, coeff, R, nx, ny, nz, dx, map, dt, gm, gp);
        return OR_OK;
    }
    /* private grids per thread, summed in thread order */
    int T = g_threads;
    size_t cnt[3], tot = 0;
    for (int a = 0; a < 3; ++a) {
        int d[3]; face_dims(a, nx, ny, nz, d);
        cnt[a] = (size_t)d[0] * d[1] * d[2];
        tot += 2 * cnt[a];
    }
    double *priv = (double *)calloc((size_t)T * tot, sizeof(double));
    if (!priv) return OR_ERR_ARG;
#pragma omp parallel num_threads(T)
    {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        double *base = priv + (size_t)t * tot;
        double *pm[3], *pv[3];
        for (int a = 0; a < 3; ++a) {
            pm[a] = base;
            pv[a] = base + cnt[a];
            base += 2 * cnt[a];
        }
#pragma omp for schedule(static)
        for (int64_t p = 0; p < np; ++p)
            p2g_particle(np, p, x, y, z, mass, mass_abs, coeff, R, nx, ny, nz, dx, map, dt, pm, pv);
    }
    for (int t = 0; t < T; ++t) {
        double *base = priv + (size_t)t * tot;
        for (int a = 0; a < 3; ++a) {
            for (size_t i = 0; i < cnt[a]; ++i) gm[a][i] += base[i];
            for (size_t i = 0; i < cnt[a]; ++i) gp[a][i] += base[cnt[a] + i];
            base += 2 * cnt[a];
        }
    }
    free(priv);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Grid update (the paper delegates it to the host simulator; the stated
 * minimal form):  v = mv/m where m > 0, else 0 (Eq 5); v~ = v + dt g_a;
 * with a solid grid, implicit two-phase drag on faces where both masses are
 * positive: u' = u / (1 + dt K (1/m_f + 1/m_s)) for u = v_f - v_s, keeping
 * the mass-weighted mean; then v~_a = 0 on the wall faces i_a in {0, n_a}.   */
static void wall_zero(int a, const int d[3], double *v)
{
    for (int k = 0; k < d[2]; ++k)
        for (int j = 0; j < d[1]; ++j)
            for (int i = 0; i < d[0]; ++i) {
                int ia = (a == 0) ? i : (a == 1) ? j : k;
                if (ia == 0 || ia == d[a] - 1) v[((size_t)k * d[1] + j) * d[0] + i] = 0.0;
            }
}

void or_grid_update(int nx, int ny, int nz, double dt, double gx, double gy, double gz,
                    double drag_k,
                    const double *fm0, const double *fm1, const double *fm2,
                    const double *fp0, const double *fp1, const double *fp2,
                    double *fv0, double *fv1, double *fv2,
                    const double *sm0, const double *sm1, const double *sm2,
                    const double *sp0, const double *sp1, const double *sp2,
                    double *sv0, double *sv1, double *sv2)
{
    const double *fm[3] = {fm0, fm1, fm2}, *fp[3] = {fp0, fp1, fp2};
    const double *sm[3] = {sm0, sm1, sm2}, *sp[3] = {sp0, sp1, sp2};
    double *fv[3] = {fv0, fv1, fv2}, *sv[3] = {sv0, sv1, sv2};
    double g[3] = {gx, gy, gz};
    int solid = sm0 != NULL;
    for (int a = 0; a < 3; ++a) {
        int d[3]; face_dims(a, nx, ny, nz, d);
        size_t cnt = (size_t)d[0] * d[1] * d[2];
        for (size_t i = 0; i < cnt; ++i) {
            double vf = fm[a][i] > 0.0 ? fp[a][i] / fm[a][i] : 0.0;
            vf += dt * g[a];
            if (solid) {
                double vs = sm[a][i] > 0.0 ? sp[a][i] / sm[a][i] : 0.0;
                vs += dt * g[a];
                if (fm[a][i] > 0.0 && sm[a][i] > 0.0 && drag_k > 0.0) {
                    double mf = fm[a][i], ms = sm[a][i];
                    double mean = (mf * vf + ms * vs) / (mf + ms);
                    double u = (vf - vs) / (1.0 + dt * drag_k * (1.0 / mf + 1.0 / ms));
                    vf = mean + ms / (mf + ms) * u;
                    vs = mean - mf / (mf + ms) * u;
                }
                sv[a][i] = vs;
            }
            fv[a][i] = vf;
        }
        wall_zero(a, d, fv[a]);
        if (solid) wall_zero(a, d, sv[a]);
    }
}

/* ------------------------------------------------------------------------ */
/* G2P: Eqs 6-8 per component plus the PolyPIC fit (Section 3.3, decoupled
 * least squares over an orthogonal basis):
 *   c_pra = sum_i w_ipa s_r(z_ipa) v~_ia / d_r,   d_r = sum_i w_ipa s_r^2,
 * with the guard; v_pa = c_p0a; x_p <- clamp(x_p + dt v_p, 1.5dx, (n-1.5)dx).
 * apic_grad = 1 (R = 4 only) replaces the linear modes by Eq 10:
 *   c_p(1+b)a = sum_i (d w_ipa / d x_pb) v~_ia.
 * coeff_out: [3][R][np]; positions written to xo, yo, zo (may alias nothing). */
int or_g2p(int64_t np, const double *x, const double *y, const double *z,
           const double *gv0, const double *gv1, const double *gv2, int R,
           int nx, int ny, int nz, double dx, double dt, int apic_grad,
           double *coeff_out, double *xo, double *yo, double *zo)
{
    build_modes();
    if (R != 1 && R != 4 && R != 8 && R != 27) return OR_ERR_ARG;
    if (apic_grad && R != 4) return OR_ERR_ARG;
    const double *gv[3] = {gv0, gv1, gv2};
    for (int64_t p = 0; p < np; ++p)
        if (!in_domain(x[p], y[p], z[p], nx, ny, nz, dx)) return OR_ERR_DOMAIN;
    int n3[3] = {nx, ny, nz};
#pragma omp parallel for num_threads(g_threads) schedule(static) if (g_threads > 1)
    for (int64_t p = 0; p < np; ++p) {
        double pos[3] = {x[p], y[p], z[p]};
        double vp[3];
        for (int a = 0; a < 3; ++a) {
            int d[3]; face_dims(a, nx, ny, nz, d);
            axis_stencil st[3];
            particle_stencils(x[p], y[p], z[p], a, dx, st);
            double num[27], den[27], gradw[3] = {0, 0, 0};
            for (int r = 0; r < R; ++r) { num[r] = 0.0; den[r] = 0.0; }
            for (int kz = 0; kz < 3; ++kz)
                for (int ky = 0; ky < 3; ++ky)
                    for (int kx = 0; kx < 3; ++kx) {
                        double w = st[0].w[kx] * st[1].w[ky] * st[2].w[kz];
                        double zz[3] = {st[0].z[kx], st[1].z[ky], st[2].z[kz]};
                        int ix = st[0].base + kx, iy = st[1].base + ky, iz = st[2].base + kz;
                        double v = gv[a][((size_t)iz * d[1] + iy) * d[0] + ix];
                        for (int r = 0; r < R; ++r) {
                            double s = mode_value(st, r, zz);
                            num[r] += w * s * v;
                            den[r] += w * s * s;
                        }
                        if (apic_grad) {
                            gradw[0] += st[0].dw[kx] * st[1].w[ky] * st[2].w[kz] * v;
                            gradw[1] += st[0].w[kx] * st[1].dw[ky] * st[2].w[kz] * v;
                            gradw[2] += st[0].w[kx] * st[1].w[ky] * st[2].dw[kz] * v;
                        }
                    }
            for (int r = 0; r < R; ++r) {
                int guarded = (g_modes[r][0] == 2 && st[0].guard) ||
                              (g_modes[r][1] == 2 && st[1].guard) ||
                              (g_modes[r][2] == 2 && st[2].guard);
                double c = guarded ? 0.0 : num[r] / den[r];
                if (apic_grad && r >= 1) c = gradw[r - 1];
                coeff_out[((int64_t)a * R + r) * np + p] = c;
            }
            vp[a] = coeff_out[((int64_t)a * R + 0) * np + p];
        }
        double out[3];
        for (int a = 0; a < 3; ++a) {
            double lo = 1.5 * dx, hi = ((double)n3[a] - 1.5) * dx;
            double xn = pos[a] + dt * vp[a];
            out[a] = xn < lo ? lo : (xn > hi ? hi : xn);
        }
        xo[p] = out[0]; yo[p] = out[1]; zo[p] = out[2];
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Adjoints (transposes of the steps above, constant map, FP64).
 *
 * P2G adjoint.  Given lm_a = dL/dm_ia and lp_a = dL/d(mv)_ia on the three
 * grids, writes lc = dL/dc_pra ([3][R][np]) and adds the position terms to
 * lx, ly, lz (which the caller zeroes or pre-loads):
 *   dL/dc_pra  = mt_p sum_i w s_r lp_ia
 *   dL/dx_pb  += mt_p sum_{a,i} [dw/dx_b (S lp + lm) + w sum_r c_r ds_r/dx_b lp]  */
int or_p2g_adjoint(int64_t np, const double *x, const double *y, const double *z,
                   const double *mass, const double *mass_abs, const double *coeff, int R,
                   int nx, int ny, int nz, double dx,
                   const double *lm0, const double *lm1, const double *lm2,
                   const double *lp0, const double *lp1, const double *lp2,
                   double *lc, double *lx, double *ly, double *lz)
{
    build_modes();
    if (R != 1 && R != 4 && R != 8 && R != 27) return OR_ERR_ARG;
    const double *lm[3] = {lm0, lm1, lm2}, *lp[3] = {lp0, lp1, lp2};
    double *lpos[3] = {lx, ly, lz};
    for (int64_t p = 0; p < np; ++p)
        if (!in_domain(x[p], y[p], z[p], nx, ny, nz, dx)) return OR_ERR_DOMAIN;
    /* each particle writes only its own entries of lc and lx, ly, lz */
#pragma omp parallel for num_threads(g_threads) schedule(static) if (g_threads > 1)
    for (int64_t p = 0; p < np; ++p) {
        double mt = mass[p] + (mass_abs ? mass_abs[p] : 0.0);
        for (int a = 0; a < 3; ++a) {
            int d[3]; face_dims(a, nx, ny, nz, d);
            axis_stencil st[3];
            particle_stencils(x[p], y[p], z[p], a, dx, st);
            double acc_c[27];
            for (int r = 0; r < R; ++r) acc_c[r] = 0.0;
            for (int kz = 0; kz < 3; ++kz)
                for (int ky = 0; ky < 3; ++ky)
                    for (int kx = 0; kx < 3; ++kx) {
                        int k3[3] = {kx, ky, kz};
                        double w = st[0].w[kx] * st[1].w[ky] * st[2].w[kz];
                        double zz[3] = {st[0].z[kx], st[1].z[ky], st[2].z[kz]};
                        int ix = st[0].base + kx, iy = st[1].base + ky, iz = st[2].base + kz;
                        size_t idx = ((size_t)iz * d[1] + iy) * d[0] + ix;
                        double LP = lp[a][idx], LM = lm[a][idx];
                        double S = 0.0;
                        for (int r = 0; r < R; ++r) {
                            double s = mode_value(st, r, zz);
                            S += coeff[((int64_t)a * R + r) * np + p] * s;
                            acc_c[r] += mt * w * s * LP;
                        }
                        for (int b = 0; b < 3; ++b) {
                            double dwb = 1.0;
                            for (int e = 0; e < 3; ++e)
                                dwb *= (e == b) ? st[e].dw[k3[e]] : st[e].w[k3[e]];
                            double dS = 0.0;
                            for (int r = 0; r < R; ++r) {
                                double ds = 1.0;
                                for (int e = 0; e < 3; ++e) {
                                    int deg = g_modes[r][e];
                                    ds *= (e == b) ? basis_df(&st[e], deg, zz[e], -1.0)
                                                   : basis_f(&st[e], deg, zz[e]);
                                }
                                dS += coeff[((int64_t)a * R + r) * np + p] * ds;
                            }
                            lpos[b][p] += mt * (dwb * (S * LP + LM) + w * dS * LP);
                        }
                    }
            for (int r = 0; r < R; ++r) lc[((int64_t)a * R + r) * np + p] = acc_c[r];
        }
    }
    return OR_OK;
}

/* G2P adjoint with the advection.  Given lc_out = dL/dc'_pra ([3][R][np]) and
 * lxo = dL/dx'_p, adds dL/dv~_ia to lv0..2 (the caller zeroes them) and adds
 * dL/dx_p to lx, ly, lz.  Clamped axes pass no gradient through the advection. */
/* The adjoint of particle p's fit and advection (the body of or_g2p_adjoint):
 * adds its grid-velocity adjoint to lv and writes its position adjoint. */
static void g2p_adjoint_particle(int64_t np, int64_t p, const double *x, const double *y,
                                 const double *z, const double *const gv[3], int R,
                                 const int n3[3], double dx, double dt, const double *lc_out,
                                 const double *const lpo[3], double *const lv[3],
                                 double *const lpos[3])
{
    int nx = n3[0], ny = n3[1], nz = n3[2];
    double pos[3] = {x[p], y[p], z[p]};
    for (int a = 0; a < 3; ++a) {
        int d[3]; face_dims(a, nx, ny, nz, d);
        axis_stencil st[3];
        particle_stencils(x[p], y[p], z[p], a, dx, st);
        /* forward quantities: num_r, den_r and their x-derivatives */
        double num[27], den[27], dnum[27][3], dden[27][3];
        for (int r = 0; r < R; ++r) {
            num[r] = den[r] = 0.0;
            for (int b = 0; b < 3; ++b) dnum[r][b] = dden[r][b] = 0.0;
        }
        for (int kz = 0; kz < 3; ++kz)
            for (int ky = 0; ky < 3; ++ky)
                for (int kx = 0; kx < 3; ++kx) {
                    int k3[3] = {kx, ky, kz};
                    double w = st[0].w[kx] * st[1].w[ky] * st[2].w[kz];
                    double zz[3] = {st[0].z[kx], st[1].z[ky], st[2].z[kz]};
                    int ix = st[0].base + kx, iy = st[1].base + ky, iz = st[2].base + kz;
                    double v = gv[a][((size_t)iz * d[1] + iy) * d[0] + ix];
                    for (int r = 0; r < R; ++r) {
                        double s = mode_value(st, r, zz);
                        num[r] += w * s * v;
                        den[r] += w * s * s;
                        for (int b = 0; b < 3; ++b) {
                            double dwb = 1.0, ds = 1.0;
                            for (int e = 0; e < 3; ++e) {
                                dwb *= (e == b) ? st[e].dw[k3[e]] : st[e].w[k3[e]];
                                int deg = g_modes[r][e];
                                ds *= (e == b) ? basis_df(&st[e], deg, zz[e], -1.0)
                                               : basis_f(&st[e], deg, zz[e]);
                            }
                            dnum[r][b] += (dwb * s + w * ds) * v;
                            dden[r][b] += dwb * s * s + 2.0 * w * s * ds;
                        }
                    }
                }
        /* adjoint seed on the output coefficients, plus advection */
        double mu[27];
        for (int r = 0; r < R; ++r) mu[r] = lc_out[((int64_t)a * R + r) * np + p];
        double c0 = num[0] / den[0];
        double lo = 1.5 * dx, hi = ((double)n3[a] - 1.5) * dx;
        double xn = pos[a] + dt * c0;
        if (xn >= lo && xn <= hi) {
            mu[0] += dt * lpo[a][p];
            lpos[a][p] += lpo[a][p];
        }
        for (int r = 0; r < R; ++r) {
            int guarded = (g_modes[r][0] == 2 && st[0].guard) ||
                          (g_modes[r][1] == 2 && st[1].guard) ||
                          (g_modes[r][2] == 2 && st[2].guard);
            if (guarded || mu[r] == 0.0) continue;
            double c = num[r] / den[r];
            for (int b = 0; b < 3; ++b)
                lpos[b][p] += mu[r] * (dnum[r][b] - c * dden[r][b]) / den[r];
        }
        for (int kz = 0; kz < 3; ++kz)
            for (int ky = 0; ky < 3; ++ky)
                for (int kx = 0; kx < 3; ++kx) {
                    double w = st[0].w[kx] * st[1].w[ky] * st[2].w[kz];
                    double zz[3] = {st[0].z[kx], st[1].z[ky], st[2].z[kz]};
                    int ix = st[0].base + kx, iy = st[1].base + ky, iz = st[2].base + kz;
                    double acc = 0.0;
                    for (int r = 0; r < R; ++r) {
                        int guarded = (g_modes[r][0] == 2 && st[0].guard) ||
                                      (g_modes[r][1] == 2 && st[1].guard) ||
                                      (g_modes[r][2] == 2 && st[2].guard);
                        if (guarded) continue;
                        acc += mu[r] * w * mode_value(st, r, zz) / den[r];
                    }
                    lv[a][((size_t)iz * d[1] + iy) * d[0] + ix] += acc;
                }
    }
}

int or_g2p_adjoint(int64_t np, const double *x, const double *y, const double *z,
                   const double *gv0, const double *gv1, const double *gv2, int R,
                   int nx, int ny, int nz, double dx, double dt,
                   const double *lc_out, const double *lxo, const double *lyo, const double *lzo,
                   double *lv0, double *lv1, double *lv2,
                   double *lx, double *ly, double *lz)
{
    build_modes();
    if (R != 1 && R != 4 && R != 8 && R != 27) return OR_ERR_ARG;
    const double *gv[3] = {gv0, gv1, gv2};
    double *lv[3] = {lv0, lv1, lv2};
    const double *lpo[3] = {lxo, lyo, lzo};
    double *lpos[3] = {lx, ly, lz};
    int n3[3] = {nx, ny, nz};
    for (int64_t p = 0; p < np; ++p)
        if (!in_domain(x[p], y[p], z[p], nx, ny, nz, dx)) return OR_ERR_DOMAIN;
    if (g_threads <= 1) {
        for (int64_t p = 0; p < np; ++p)
            g2p_adjoint_particle(np, p, x, y, z, gv, R, n3, dx, dt, lc_out, lpo, lv, lpos);
        return OR_OK;
    }
    /* private grid adjoints per thread, added to lv in thread order */
    int T = g_threads;
    size_t cnt[3], tot = 0;
    for (int a = 0; a < 3; ++a) {
        int d[3]; face_dims(a, nx, ny, nz, d);
        cnt[a] = (size_t)d[0] * d[1] * d[2];
        tot += cnt[a];
    }
    double *priv = (double *)calloc((size_t)T * tot, sizeof(double));
    if (!priv) return OR_ERR_ARG;
#pragma omp parallel num_threads(T)
    {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        double *base = priv + (size_t)t * tot;
        double *pl[3] = {base, base + cnt[0], base + cnt[0] + cnt[1]};
#pragma omp for schedule(static)
        for (int64_t p = 0; p < np; ++p)
            g2p_adjoint_particle(np, p, x, y, z, gv, R, n3, dx, dt, lc_out, lpo, pl, lpos);
    }
    for (int t = 0; t < T; ++t) {
        double *base = priv + (size_t)t * tot;
        for (int a = 0; a < 3; ++a) {
            for (size_t i = 0; i < cnt[a]; ++i) lv[a][i] += base[i];
            base += cnt[a];
        }
    }
    free(priv);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Pressure projection (delegated to the host simulator in the paper; the
 * stated minimal form): cell-centred pressure on fluid cells (fluid[c] != 0),
 * p = 0 in non-fluid cells, zero normal velocity at the walls.  For a fluid
 * cell c:  sum_{non-wall neighbours n} (p_c - p_n) = -(rho dx^2 / dt) div_c,
 * div_c = sum_a (v_a(c + e_a) - v_a(c)) / dx.  Solved by Jacobi-preconditioned
 * CG to ||r|| <= rtol ||b||; then v_a -= dt/(rho dx) (p_right - p_left) on
 * every non-wall face with a fluid cell on at least one side.  Returns the
 * iteration count, or OR_ERR_NOT_CONVERGED.                                */
#define CIDX(i, j, k) (((size_t)(k) * ny + (j)) * nx + (i))

/* diag[c] = number of non-wall neighbours of fluid cell c (0 elsewhere). */
static void laplacian_diag(int nx, int ny, int nz, const uint8_t *fluid, double *diag)
{
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t c = CIDX(i, j, k);
                diag[c] = 0.0;
                if (!fluid[c]) continue;
                diag[c] = (double)((i > 0) + (i < nx - 1) + (j > 0) + (j < ny - 1) + (k > 0) +
                                   (k < nz - 1));
            }
}

/* dst = A src on fluid cells: diag p_c minus the fluid neighbours' p. */
static void laplacian_apply(int nx, int ny, int nz, const uint8_t *fluid, const double *diag,
                            const double *src, double *dst)
{
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t c = CIDX(i, j, k);
                if (!fluid[c]) { dst[c] = 0.0; continue; }
                double s = diag[c] * src[c];
                if (i > 0 && fluid[CIDX(i - 1, j, k)]) s -= src[CIDX(i - 1, j, k)];
                if (i < nx - 1 && fluid[CIDX(i + 1, j, k)]) s -= src[CIDX(i + 1, j, k)];
                if (j > 0 && fluid[CIDX(i, j - 1, k)]) s -= src[CIDX(i, j - 1, k)];
                if (j < ny - 1 && fluid[CIDX(i, j + 1, k)]) s -= src[CIDX(i, j + 1, k)];
                if (k > 0 && fluid[CIDX(i, j, k - 1)]) s -= src[CIDX(i, j, k - 1)];
                if (k < nz - 1 && fluid[CIDX(i, j, k + 1)]) s -= src[CIDX(i, j, k + 1)];
                dst[c] = s;
            }
}

/* Jacobi-preconditioned CG for A x = b on the fluid cells, x from 0, to
 * ||r|| <= rtol ||b||.  Returns the iteration count (-1: not converged). */
static int jacobi_pcg(int nx, int ny, int nz, const uint8_t *fluid, const double *diag,
                      const double *b, double *x, double rtol, int maxiter)
{
    size_t nc = (size_t)nx * ny * nz;
    double *r = calloc(nc, sizeof(double)), *zv = calloc(nc, sizeof(double));
    double *pd = calloc(nc, sizeof(double)), *Ap = calloc(nc, sizeof(double));
    double bnorm = 0.0;
    for (size_t c = 0; c < nc; ++c) { x[c] = 0.0; r[c] = b[c]; bnorm += b[c] * b[c]; }
    bnorm = sqrt(bnorm);
    int it = 0, converged = bnorm == 0.0;
    double rz = 0.0;
    for (size_t c = 0; c < nc; ++c) {
        zv[c] = fluid[c] ? r[c] / diag[c] : 0.0;
        pd[c] = zv[c];
        rz += r[c] * zv[c];
    }
    while (!converged && it < maxiter) {
        laplacian_apply(nx, ny, nz, fluid, diag, pd, Ap);
        double pAp = 0.0;
        for (size_t c = 0; c < nc; ++c) pAp += pd[c] * Ap[c];
        double alpha = rz / pAp;
        double rn = 0.0;
        for (size_t c = 0; c < nc; ++c) {
            x[c] += alpha * pd[c];
            r[c] -= alpha * Ap[c];
            rn += r[c] * r[c];
        }
        ++it;
        if (sqrt(rn) <= rtol * bnorm) { converged = 1; break; }
        double rz_new = 0.0;
        for (size_t c = 0; c < nc; ++c) {
            zv[c] = fluid[c] ? r[c] / diag[c] : 0.0;
            rz_new += r[c] * zv[c];
        }
        double beta = rz_new / rz;
        rz = rz_new;
        for (size_t c = 0; c < nc; ++c) pd[c] = zv[c] + beta * pd[c];
    }
    free(r); free(zv); free(pd); free(Ap);
    return converged ? it : -1;
}

int or_pcg_project(int nx, int ny, int nz, double dx, double dt, double rho,
                   const uint8_t *fluid, double *v0, double *v1, double *v2,
                   double *pressure, double rtol, int maxiter)
{
    double *v[3] = {v0, v1, v2};
    int n3[3] = {nx, ny, nz};
    size_t nc = (size_t)nx * ny * nz;
    double *b = calloc(nc, sizeof(double)), *diag = calloc(nc, sizeof(double));
    laplacian_diag(nx, ny, nz, fluid, diag);
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t c = CIDX(i, j, k);
                if (!fluid[c]) continue;
                double div = 0.0;
                for (int a = 0; a < 3; ++a) {
                    int d[3]; face_dims(a, nx, ny, nz, d);
                    int lo[3] = {i, j, k}, hi[3] = {i, j, k};
                    hi[a] += 1;
                    double vl = v[a][((size_t)lo[2] * d[1] + lo[1]) * d[0] + lo[0]];
                    double vh = v[a][((size_t)hi[2] * d[1] + hi[1]) * d[0] + hi[0]];
                    div += (vh - vl) / dx;
                }
                b[c] = -(rho * dx * dx / dt) * div;
            }
    int it = jacobi_pcg(nx, ny, nz, fluid, diag, b, pressure, rtol, maxiter);
    /* velocity update on interior faces touching a fluid cell */
    for (int a = 0; a < 3; ++a) {
        int d[3]; face_dims(a, nx, ny, nz, d);
        for (int k = 0; k < d[2]; ++k)
            for (int j = 0; j < d[1]; ++j)
                for (int i = 0; i < d[0]; ++i) {
                    int f[3] = {i, j, k};
                    if (f[a] == 0 || f[a] == n3[a]) continue;
                    int lo[3] = {i, j, k};
                    lo[a] -= 1;
                    size_t cl = CIDX(lo[0], lo[1], lo[2]), ch = CIDX(i, j, k);
                    if (!fluid[cl] && !fluid[ch]) continue;
                    v[a][((size_t)k * d[1] + j) * d[0] + i] -=
                        dt / (rho * dx) * (pressure[ch] - pressure[cl]);
                }
    }
    free(b); free(diag);
    return it >= 0 ? it : OR_ERR_NOT_CONVERGED;
}

/* ------------------------------------------------------------------------ */
/* Adjoint of the whole grid update (or_grid_update, then or_pcg_project on
 * the fluid velocity when `fluid` is given), each step's transpose written
 * out, last step first.  Given lfv = dL/dv~_f (and lsv = dL/dv~_s with a
 * solid grid), writes lfm = dL/dm_f, lfp = dL/d(mv)_f (and lsm, lsp).
 *   projection  v' = v + dx G A^-1 D v, with (G p)_f = p_ch - p_cl on the
 *               interior faces touching fluid and (D v)_c = div_c above, so
 *               v^ = v^' + dx D^T A^-1 G^T v^': s = G^T v^' on the fluid
 *               cells, A q = s (Jacobi-PCG, rtol), v^_f += q_cl - q_ch (dx
 *               times D^T q, whose entries are +-1/dx; q = 0 off the fluid
 *               cells; every face, walls included);
 *   walls       v^ = 0 on the wall faces;
 *   drag        per face holding both masses (drag_k > 0): the transposed
 *               Jacobian of (v_f, v_s) -> (v_f', v_s') and its derivatives
 *               in m_f and m_s (through the mean, the weights m/(m_f+m_s) and
 *               the factor 1/(1 + dt K (1/m_f + 1/m_s)));
 *   gravity     identity;
 *   division    v = mv/m where m > 0: (mv)^ = v^/m, m^ += -v^ mv/m^2; faces
 *               with m = 0 pass nothing.
 * Returns OR_OK, or OR_ERR_NOT_CONVERGED if the adjoint solve did not.      */
int or_grid_update_adjoint(int nx, int ny, int nz, double dt, double gx, double gy, double gz,
                           double drag_k, const double *const *fm,
                           const double *const *fp, const double *const *sm,
                           const double *const *sp, const uint8_t *fluid, double rtol,
                           int maxiter, const double *const *lfv, const double *const *lsv,
                           double *const *lfm, double *const *lfp, double *const *lsm,
                           double *const *lsp)
{
    int n3[3] = {nx, ny, nz};
    double g[3] = {gx, gy, gz};
    int solid = sm != NULL;
    int rc = OR_OK;
    double *lf[3];
    for (int a = 0; a < 3; ++a) {
        int d[3]; face_dims(a, nx, ny, nz, d);
        size_t cnt = (size_t)d[0] * d[1] * d[2];
        lf[a] = malloc(cnt * sizeof(double));
        memcpy(lf[a], lfv[a], cnt * sizeof(double));
    }
    if (fluid) {
        size_t nc = (size_t)nx * ny * nz;
        double *s = calloc(nc, sizeof(double)), *q = calloc(nc, sizeof(double));
        double *diag = calloc(nc, sizeof(double));
        laplacian_diag(nx, ny, nz, fluid, diag);
        /* s = G^T v^': +v^' on a face whose upper cell is c, -v^' on one whose
         * lower cell is c, interior faces only */
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    size_t c = CIDX(i, j, k);
                    if (!fluid[c]) continue;
                    int ijk[3] = {i, j, k};
                    double acc = 0.0;
                    for (int a = 0; a < 3; ++a) {
                        int d[3]; face_dims(a, nx, ny, nz, d);
                        int lo[3] = {i, j, k}, hi[3] = {i, j, k};
                        hi[a] += 1;
                        if (ijk[a] > 0) acc += lf[a][((size_t)lo[2] * d[1] + lo[1]) * d[0] + lo[0]];
                        if (ijk[a] + 1 < n3[a]) acc -= lf[a][((size_t)hi[2] * d[1] + hi[1]) * d[0] + hi[0]];
                    }
                    s[c] = acc;
                }
        if (jacobi_pcg(nx, ny, nz, fluid, diag, s, q, rtol, maxiter) < 0) rc = OR_ERR_NOT_CONVERGED;
        /* v^ += dx D^T q: face f gets (q_cl - q_ch)/dx from the two cells it bounds */
        for (int a = 0; a < 3; ++a) {
            int d[3]; face_dims(a, nx, ny, nz, d);
            for (int k = 0; k < d[2]; ++k)
                for (int j = 0; j < d[1]; ++j)
                    for (int i = 0; i < d[0]; ++i) {
                        int f[3] = {i, j, k};
                        double ql = 0.0, qh = 0.0;
                        if (f[a] > 0) {
                            int lo[3] = {i, j, k};
                            lo[a] -= 1;
                            size_t cl = CIDX(lo[0], lo[1], lo[2]);
                            if (fluid[cl]) ql = q[cl];
                        }
                        if (f[a] < n3[a]) {
                            size_t ch = CIDX(i, j, k);
                            if (fluid[ch]) qh = q[ch];
                        }
                        lf[a][((size_t)k * d[1] + j) * d[0] + i] += ql - qh;
                    }
        }
        free(s); free(q); free(diag);
    }
    for (int a = 0; a < 3; ++a) {
        int d[3]; face_dims(a, nx, ny, nz, d);
        for (int k = 0; k < d[2]; ++k)
            for (int j = 0; j < d[1]; ++j)
                for (int i = 0; i < d[0]; ++i) {
                    size_t idx = ((size_t)k * d[1] + j) * d[0] + i;
                    int ia = (a == 0) ? i : (a == 1) ? j : k;
                    int wall = (ia == 0 || ia == d[a] - 1);
                    double lvf = wall ? 0.0 : lf[a][idx];
                    double lvs = (solid && !wall) ? lsv[a][idx] : 0.0;
                    double mf = fm[a][idx], ms = solid ? sm[a][idx] : 0.0;
                    double dmf = 0.0, dms = 0.0;   /* mass adjoints from the drag */
                    if (solid && drag_k > 0.0 && mf > 0.0 && ms > 0.0) {
                        double vf = fp[a][idx] / mf + dt * g[a];
                        double vs = sp[a][idx] / ms + dt * g[a];
                        double M = mf + ms, wa = ms / M, wb = mf / M;
                        double Dd = 1.0 + dt * drag_k * (1.0 / mf + 1.0 / ms);
                        double u = (vf - vs) / Dd, mean = wb * vf + wa * vs;
                        /* d(mean)/dm, d(wa)/dm, d(wb)/dm, du/dm */
                        double mean_f = (vf - mean) / M, mean_s = (vs - mean) / M;
                        double wa_f = -ms / (M * M), wa_s = mf / (M * M);
                        double wb_f = ms / (M * M), wb_s = -mf / (M * M);
                        double u_f = u * dt * drag_k / (Dd * mf * mf);
                        double u_s = u * dt * drag_k / (Dd * ms * ms);
                        dmf = lvf * (mean_f + wa_f * u + wa * u_f) + lvs * (mean_f - wb_f * u - wb * u_f);
                        dms = lvf * (mean_s + wa_s * u + wa * u_s) + lvs * (mean_s - wb_s * u - wb * u_s);
                        double lf_new = lvf * (wb + wa / Dd) + lvs * (wb - wb / Dd);
                        double ls_new = lvf * (wa - wa / Dd) + lvs * (wa + wb / Dd);
                        lvf = lf_new;
                        lvs = ls_new;
                    }
                    if (mf > 0.0) {
                        lfp[a][idx] = lvf / mf;
                        lfm[a][idx] = dmf - lvf * fp[a][idx] / (mf * mf);
                    } else {
                        lfp[a][idx] = 0.0;
                        lfm[a][idx] = 0.0;
                    }
                    if (solid) {
                        if (ms > 0.0) {
                            lsp[a][idx] = lvs / ms;
                            lsm[a][idx] = dms - lvs * sp[a][idx] / (ms * ms);
                        } else {
                            lsp[a][idx] = 0.0;
                            lsm[a][idx] = 0.0;
                        }
                    }
                }
        free(lf[a]);
    }
    return rc;
}
#undef CIDX
/* ------------------------------------------------------------------------ */
/* Fabric stand-in (the paper takes the cloth mechanics from Fei et al.,
 * Sections 3.4 and 4, and gives no force model): a mass-spring lattice on the
 * sheet's vertex particles.  Vertex (i, k) of an m x m lattice has id k m + i;
 * ids >= m^2 (element particles) carry no springs.  Springs join each vertex
 * to its lattice neighbours at offsets (+-1, 0), (0, +-1) [stretch, rest h],
 * (+-1, +-1) [shear, rest h sqrt 2] and (+-2, 0), (0, +-2) [bend, rest 2h].
 * The force of the spring to neighbour j on vertex i, with d = x_j - x_i,
 * L = |d|, e = d / L:   f = k (L - L0) e + c ((v_j - v_i) . e) e.
 * The velocity of vertex i (mode 0 of its coefficients) then takes one
 * explicit step  v_i += dt sum f / (m_i + m_abs,i); every velocity is read
 * before any is written.  x, v in particle order, id[p] the lattice id.    */
void or_fabric_forces(int64_t np, const double *x, const double *y, const double *z,
                      const double *mass, const double *mass_abs, double *coeff, int R,
                      const uint32_t *id, int m, double h, double k_stretch, double k_shear,
                      double k_bend, double damping, double dt)
{
    int64_t nv = (int64_t)m * m;
    int64_t *slot = malloc((size_t)nv * sizeof(int64_t));
    double *dv = calloc((size_t)np * 3, sizeof(double));
    for (int64_t v = 0; v < nv; ++v) slot[v] = -1;
    for (int64_t p = 0; p < np; ++p)
        if (id[p] < (uint32_t)nv) slot[id[p]] = p;
    const int off[12][2] = {{1, 0}, {-1, 0}, {0, 1}, {0, -1}, {1, 1}, {1, -1}, {-1, 1},
                            {-1, -1}, {2, 0}, {-2, 0}, {0, 2}, {0, -2}};
    const double *pos[3] = {x, y, z};
    for (int64_t p = 0; p < np; ++p) {
        if (id[p] >= (uint32_t)nv) continue;
        int i = (int)(id[p] % (uint32_t)m), k = (int)(id[p] / (uint32_t)m);
        double f[3] = {0.0, 0.0, 0.0};
        for (int s = 0; s < 12; ++s) {
            int i2 = i + off[s][0], k2 = k + off[s][1];
            if (i2 < 0 || i2 >= m || k2 < 0 || k2 >= m) continue;
            int64_t q = slot[(int64_t)k2 * m + i2];
            if (q < 0) continue;
            double kk = s < 4 ? k_stretch : s < 8 ? k_shear : k_bend;
            double L0 = s < 4 ? h : s < 8 ? h * sqrt(2.0) : 2.0 * h;
            double d[3], L = 0.0;
            for (int a = 0; a < 3; ++a) {
                d[a] = pos[a][q] - pos[a][p];
                L += d[a] * d[a];
            }
            L = sqrt(L);
            if (!(L > 0.0)) continue;
            double rv = 0.0;
            for (int a = 0; a < 3; ++a)
                rv += (coeff[((size_t)a * R) * np + q] - coeff[((size_t)a * R) * np + p]) * d[a] / L;
            for (int a = 0; a < 3; ++a) f[a] += (kk * (L - L0) + damping * rv) * d[a] / L;
        }
        double mt = mass[p] + (mass_abs ? mass_abs[p] : 0.0);
        for (int a = 0; a < 3; ++a) dv[(size_t)a * np + p] = dt * f[a] / mt;
    }
    for (int64_t p = 0; p < np; ++p)
        for (int a = 0; a < 3; ++a) coeff[((size_t)a * R) * np + p] += dv[(size_t)a * np + p];
    free(slot);
    free(dv);
}

/* Absorption stand-in (the paper takes m_abs as given, Eqs 18-20; its
 * dynamics are Fei et al.'s porous flow): per cell, with M_f the fluid mass
 * of the cell's fluid particles, each solid particle p in the cell asks for
 * d_p = min(rate dt m_s,p, max(0, capacity m_s,p - m_abs,p)); the cell gives
 * D = min(sum d_p, max_fraction M_f); solid particle p gains d_p D / sum d
 * and fluid particle q loses m_q D / M_f, so the cell's total mass is kept.
 * Cells are decided in FP32 as for the sort (fx, fy, fz: FP32 positions).  */
void or_absorb(int64_t nf, const float *fx, const float *fy, const float *fz, double *fmass,
               int64_t ns, const float *sx, const float *sy, const float *sz,
               const double *smass, double *mass_abs, int nx, int ny, int nz, double dx,
               double dt, double rate, double capacity, double max_fraction)
{
    size_t nc = (size_t)nx * ny * nz;
    double *Mf = calloc(nc, sizeof(double)), *Dd = calloc(nc, sizeof(double));
    uint32_t *kf = malloc((size_t)(nf > 0 ? nf : 1) * sizeof(uint32_t));
    uint32_t *ks = malloc((size_t)(ns > 0 ? ns : 1) * sizeof(uint32_t));
    or_keys(nf, fx, fy, fz, nx, ny, nz, dx, kf);
    or_keys(ns, sx, sy, sz, nx, ny, nz, dx, ks);
    for (int64_t q = 0; q < nf; ++q) Mf[kf[q]] += fmass[q];
    double *d = malloc((size_t)(ns > 0 ? ns : 1) * sizeof(double));
    for (int64_t p = 0; p < ns; ++p) {
        double room = capacity * smass[p] - mass_abs[p];
        double want = rate * dt * smass[p];
        d[p] = room > 0.0 ? (want < room ? want : room) : 0.0;
        Dd[ks[p]] += d[p];
    }
    for (int64_t p = 0; p < ns; ++p) {
        size_t c = ks[p];
        double D = Dd[c] < max_fraction * Mf[c] ? Dd[c] : max_fraction * Mf[c];
        if (D > 0.0) mass_abs[p] += d[p] * D / Dd[c];
    }
    for (int64_t q = 0; q < nf; ++q) {
        size_t c = kf[q];
        double D = Dd[c] < max_fraction * Mf[c] ? Dd[c] : max_fraction * Mf[c];
        if (D > 0.0) fmass[q] -= fmass[q] * D / Mf[c];
    }
    free(Mf); free(Dd); free(kf); free(ks); free(d);
}

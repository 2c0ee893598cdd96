// adjoint.cu -- adjoint (transposed) transfers for differentiating through
// steps of PolyPIC (constant map, single phase, FP32 coefficients).
//
// Forward, per particle p and face grid a (physical units, z = x_i - x_p):
//   P2G  m_ia  += mt W_ia,   mv_ia += mt sum_abc c_abc Fx_a Fy_b Fz_c
//   G2P  c'_abc = sum_i Gx_a Gy_b Gz_c v_ia,   x'_a = clamp(x_a + dt c'_000)
// with per-axis factors (t = particle offset from the middle node in cells,
// q = 1 - 4t^2, F^1 and phi the dimensionless closed forms of polypic_internal):
//   F0 = W, F1 = dx F^1, F2 = dx^2 phi (1, -2, 1)          (P2G, W f_a)
//   G0 = W, G1 = 4 F^1 / dx, G2 = (1, -2, 1) / (2 dx^2)   (fit, W f_a / d_a)
// and their x-derivatives (dt/dx = 1/dx):
//   dW/dt = (t - 1/2, -2t, t + 1/2)
//   dF^1/dt = (3q/8, (12t^2 - 3)/4, 3q/8)
//   dphi/dt = -t q (7 - 12 t^2) / 4,   dG2/dx = 0 (the quadratic fit weights
//   do not depend on t).
//
// G2P adjoint: mu_abc = lc'_abc (+ dt lx'_a on the constant mode if x'_a was
// not clamped);  lv_ia += sum_abc mu_abc G_a G_b G_c  (a P2G-shaped scatter,
// done by the deterministic P2G kernel);  lx_b += (lx'_b if not clamped)
// + sum_a sum_abc mu_abc sum_i d/dx_b(G_a G_b G_c) v_ia  (gathered here).
// P2G adjoint: lc_abc = mt sum_i F_a F_b F_c lmv_ia;  lx_b += mt sum_a sum_i
// [d/dx_b(W W W) lm_ia + sum_abc c_abc d/dx_b(F_a F_b F_c) lmv_ia].
#include "adjoint.cuh"
#include "p2g.cuh"

namespace polypic {

constexpr int kAdjThreads = 256;
template <int A> struct ATile {
    static constexpr int X = A == 0 ? 11 : 10, Y = A == 1 ? 11 : 10, Z = A == 2 ? 7 : 6;
    static constexpr int N = X * Y * Z;
};
constexpr int kATileOff1 = ATile<0>::N, kATileOff2 = ATile<0>::N + ATile<1>::N;
constexpr int kATileFloats = ATile<0>::N + ATile<1>::N + ATile<2>::N;

struct AxisFac {
    float W[3], dW[3];    // W and dW/dx
    float F1[3], dF1[3];  // dimensionless F^1 and dF^1/dt
    float phi, dphi;      // phi and dphi/dt
    bool guard;
};

__device__ __forceinline__ AxisFac axis_fac(const Axis &ax) {
    AxisFac f;
    const float t = ax.t;
    const Stencil1D s = stencil_1d(t);
    const float q = (1.0f - 2.0f * t) * (1.0f + 2.0f * t);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        f.W[k] = s.W[k];
        f.F1[k] = s.F1[k];
    }
    f.dW[0] = t - 0.5f;
    f.dW[1] = -2.0f * t;
    f.dW[2] = t + 0.5f;
    f.dF1[0] = 0.375f * q;
    f.dF1[1] = (12.0f * t * t - 3.0f) * 0.25f;
    f.dF1[2] = 0.375f * q;
    f.phi = s.phi;
    f.dphi = -t * q * (7.0f - 12.0f * t * t) * 0.25f;
    f.guard = ax.guard;
    return f;
}

// P2G factor rows (physical) and their x-derivatives.
template <int D>
__device__ __forceinline__ void p2g_rows(const AxisFac &f, float dx, float inv_dx, float (&F)[D][3],
                                         float (&dF)[D][3]) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        F[0][k] = f.W[k];
        dF[0][k] = f.dW[k] * inv_dx;
    }
    if constexpr (D > 1) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            F[1][k] = dx * f.F1[k];
            dF[1][k] = f.dF1[k];
        }
    }
    if constexpr (D > 2) {
        const float p = dx * dx * f.phi, dp = dx * f.dphi;
        F[2][0] = p;
        F[2][1] = -2.0f * p;
        F[2][2] = p;
        dF[2][0] = dp;
        dF[2][1] = -2.0f * dp;
        dF[2][2] = dp;
    }
}

// Fit factor rows (physical) and their x-derivatives.
template <int D>
__device__ __forceinline__ void fit_rows_d(const AxisFac &f, float inv_dx, float (&G)[D][3],
                                           float (&dG)[D][3]) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        G[0][k] = f.W[k];
        dG[0][k] = f.dW[k] * inv_dx;
    }
    if constexpr (D > 1) {
        const float a = 4.0f * inv_dx, b = 4.0f * inv_dx * inv_dx;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            G[1][k] = a * f.F1[k];
            dG[1][k] = b * f.dF1[k];
        }
    }
    if constexpr (D > 2) {
        const float h = f.guard ? 0.0f : 0.5f * inv_dx * inv_dx;
        G[2][0] = h;
        G[2][1] = -2.0f * h;
        G[2][2] = h;
        dG[2][0] = dG[2][1] = dG[2][2] = 0.0f;
    }
}

// sum_abc mu_abc sum_i d/dx_b (X_a Y_b Z_c)(i) v(i) for b = x, y, z, with the
// contraction over x first, then y, then z, streamed over a.
template <int R, int D>
__device__ __forceinline__ void adj_position(const float (&X)[D][3], const float (&dX)[D][3],
                                             const float (&Y)[D][3], const float (&dY)[D][3],
                                             const float (&Z)[D][3], const float (&dZ)[D][3],
                                             const float (&v)[3][3][3], const float (&mu)[D][D][D],
                                             float &Dx, float &Dy, float &Dz) {
#pragma unroll
    for (int a = 0; a < D; ++a) {
        float U1[3][3], U1d[3][3];  // [ky][kz]
#pragma unroll
        for (int ky = 0; ky < 3; ++ky)
#pragma unroll
            for (int kz = 0; kz < 3; ++kz) {
                U1[ky][kz] = fmaf(X[a][0], v[0][ky][kz], fmaf(X[a][1], v[1][ky][kz], X[a][2] * v[2][ky][kz]));
                U1d[ky][kz] = fmaf(dX[a][0], v[0][ky][kz], fmaf(dX[a][1], v[1][ky][kz], dX[a][2] * v[2][ky][kz]));
            }
#pragma unroll
        for (int b = 0; b < D; ++b) {
            float U2[3], U2dy[3], U2dx[3];
#pragma unroll
            for (int kz = 0; kz < 3; ++kz) {
                U2[kz] = fmaf(Y[b][0], U1[0][kz], fmaf(Y[b][1], U1[1][kz], Y[b][2] * U1[2][kz]));
                U2dy[kz] = fmaf(dY[b][0], U1[0][kz], fmaf(dY[b][1], U1[1][kz], dY[b][2] * U1[2][kz]));
                U2dx[kz] = fmaf(Y[b][0], U1d[0][kz], fmaf(Y[b][1], U1d[1][kz], Y[b][2] * U1d[2][kz]));
            }
#pragma unroll
            for (int kz = 0; kz < 3; ++kz) {
                float M = 0.0f, Md = 0.0f;
#pragma unroll
                for (int c = 0; c < D; ++c)
                    if (has_mode(R, a, b, c)) {
                        M = fmaf(mu[a][b][c], Z[c][kz], M);
                        Md = fmaf(mu[a][b][c], dZ[c][kz], Md);
                    }
                Dx = fmaf(M, U2dx[kz], Dx);
                Dy = fmaf(M, U2dy[kz], Dy);
                Dz = fmaf(Md, U2[kz], Dz);
            }
        }
    }
}

// out_abc = sum_i X_a Y_b Z_c v(i) for the modes of the set.
template <int R, int D>
__device__ __forceinline__ void contract_modes(const float (&X)[D][3], const float (&Y)[D][3],
                                               const float (&Z)[D][3], const float (&v)[3][3][3],
                                               float (&out)[D][D][D]) {
#pragma unroll
    for (int a = 0; a < D; ++a) {
        float U1[3][3];
#pragma unroll
        for (int ky = 0; ky < 3; ++ky)
#pragma unroll
            for (int kz = 0; kz < 3; ++kz)
                U1[ky][kz] = fmaf(X[a][0], v[0][ky][kz], fmaf(X[a][1], v[1][ky][kz], X[a][2] * v[2][ky][kz]));
#pragma unroll
        for (int b = 0; b < D; ++b) {
            float U2[3];
#pragma unroll
            for (int kz = 0; kz < 3; ++kz)
                U2[kz] = fmaf(Y[b][0], U1[0][kz], fmaf(Y[b][1], U1[1][kz], Y[b][2] * U1[2][kz]));
#pragma unroll
            for (int c = 0; c < D; ++c)
                out[a][b][c] = has_mode(R, a, b, c)
                                   ? fmaf(Z[c][0], U2[0], fmaf(Z[c][1], U2[1], Z[c][2] * U2[2]))
                                   : 0.0f;
        }
    }
}

// Stage the footprints (three face grids) of `src` around tile (tx, ty, tz).
__device__ __forceinline__ void stage_tile(const GridGeom &g, const float *const src[3], int ox,
                                           int oy, int oz, float *dst) {
    const int dims[3][3] = {{ATile<0>::X, ATile<0>::Y, ATile<0>::Z},
                            {ATile<1>::X, ATile<1>::Y, ATile<1>::Z},
                            {ATile<2>::X, ATile<2>::Y, ATile<2>::Z}};
    const int off[3] = {0, kATileOff1, kATileOff2};
    for (int a = 0; a < 3; ++a) {
        const int X = dims[a][0], Y = dims[a][1], Z = dims[a][2];
        const int dX = g.n[0] + (a == 0), dY = g.n[1] + (a == 1), dZ = g.n[2] + (a == 2);
        for (int i = threadIdx.x; i < X * Y * Z; i += kAdjThreads) {
            const int lx = i % X, ly = (i / X) % Y, lz = i / (X * Y);
            const int gx = ox + lx, gy = oy + ly, gz = oz + lz;
            float v = 0.0f;
            if (gx >= 0 && gx < dX && gy >= 0 && gy < dY && gz >= 0 && gz < dZ)
                v = src[a][((int64_t)gz * dY + gy) * dX + gx];
            dst[off[a] + i] = v;
        }
    }
}

template <int A>
__device__ __forceinline__ void read_stencil(const float *tile, int lx, int ly, int lz,
                                             float (&v)[3][3][3]) {
    const float *t = tile + (A == 0 ? 0 : A == 1 ? kATileOff1 : kATileOff2);
#pragma unroll
    for (int kz = 0; kz < 3; ++kz)
#pragma unroll
        for (int ky = 0; ky < 3; ++ky)
#pragma unroll
            for (int kx = 0; kx < 3; ++kx)
                v[kx][ky][kz] = t[((lz + kz) * ATile<A>::Y + (ly + ky)) * ATile<A>::X + lx + kx];
}

struct ParticleAxes {
    bool ok;
    int cell[3];
    Axis ctr[3], fce[3];
};

__device__ __forceinline__ ParticleAxes particle_axes(const GridGeom &g, float px, float py,
                                                      float pz, int tx, int ty, int tz) {
    ParticleAxes P;
    const float v[3] = {cell_coord(px, g.inv_dx), cell_coord(py, g.inv_dx), cell_coord(pz, g.inv_dx)};
    P.ok = coord_valid(v[0], g.n[0]) && coord_valid(v[1], g.n[1]) && coord_valid(v[2], g.n[2]);
    const int org[3] = {8 * tx, 8 * ty, 4 * tz}, ext[3] = {8, 8, 4};
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        P.cell[b] = cell_index(v[b], g.n[b]);
        P.ok = P.ok && P.cell[b] >= org[b] && P.cell[b] < org[b] + ext[b];
        P.ctr[b] = axis_decide(v[b], false);
        P.fce[b] = axis_decide(v[b], true);
    }
    return P;
}

// ---------------------------------------------------------------- G2P adjoint gather
template <int R, int A>
__device__ __forceinline__ void g2p_adj_component(const AdjG2PArgs &G, const ParticleAxes &pa,
                                                  const float *tile, int ox, int oy, int oz,
                                                  uint32_t j, float px_a, float (&lx)[3]) {
    constexpr int D = axis_degrees(R);
    const Axis &ax = A == 0 ? pa.fce[0] : pa.ctr[0];
    const Axis &ay = A == 1 ? pa.fce[1] : pa.ctr[1];
    const Axis &az = A == 2 ? pa.fce[2] : pa.ctr[2];
    float X[D][3], dX[D][3], Y[D][3], dY[D][3], Z[D][3], dZ[D][3];
    fit_rows_d<D>(axis_fac(ax), G.inv_dx, X, dX);
    fit_rows_d<D>(axis_fac(ay), G.inv_dx, Y, dY);
    fit_rows_d<D>(axis_fac(az), G.inv_dx, Z, dZ);
    float v[3][3][3];
    read_stencil<A>(tile, ax.base - ox, ay.base - oy, az.base - oz, v);
    // the forward velocity fit (constant mode) decides whether x'_A was clamped
    float c0 = 0.0f;
#pragma unroll
    for (int kz = 0; kz < 3; ++kz)
#pragma unroll
        for (int ky = 0; ky < 3; ++ky) {
            const float yz = Y[0][ky] * Z[0][kz];
#pragma unroll
            for (int kx = 0; kx < 3; ++kx) c0 = fmaf(X[0][kx] * yz, v[kx][ky][kz], c0);
        }
    const float xn = fmaf(G.dt, c0, px_a);
    const bool clamped = xn < G.g.lo[A] || xn > G.g.hi[A];
    const float lxo = __ldg(G.bar_x[A] + j);
    // all loads of the component first (read-only path), then the stores:
    // the loads go out together instead of one per store
    const int64_t cnt = G.count;
    const float *__restrict__ bc = G.bar_c + (int64_t)A * R * cnt + j;
    float *__restrict__ mo = G.mu + (int64_t)A * R * cnt + j;
    float mu[D][D][D];
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b)
#pragma unroll
            for (int c = 0; c < D; ++c)
                mu[a][b][c] = has_mode(R, a, b, c) ? __ldg(bc + mode_index(a, b, c) * cnt) : 0.0f;
    if (!clamped) mu[0][0][0] = fmaf(G.dt, lxo, mu[0][0][0]);
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b)
#pragma unroll
            for (int c = 0; c < D; ++c)
                if (has_mode(R, a, b, c)) mo[mode_index(a, b, c) * cnt] = mu[a][b][c];
    float Dx = 0.0f, Dy = 0.0f, Dz = 0.0f;
    adj_position<R, D>(X, dX, Y, dY, Z, dZ, v, mu, Dx, Dy, Dz);
    lx[0] += Dx;
    lx[1] += Dy;
    lx[2] += Dz;
    if (!clamped) lx[A] += lxo;
}

template <int R>
__global__ void __launch_bounds__(kAdjThreads) k_g2p_adjoint(AdjG2PArgs G) {
    __shared__ float s_tile[kATileFloats];
    const GridGeom &g = G.g;
    const uint32_t tile = blockIdx.x;
    const uint32_t jb = G.cell_start[tile * 256], je = G.cell_start[tile * 256 + 256];
    if (jb == je) return;
    const int tx = (int)(tile % (uint32_t)g.tiles[0]);
    const int ty = (int)((tile / (uint32_t)g.tiles[0]) % (uint32_t)g.tiles[1]);
    const int tz = (int)(tile / ((uint32_t)g.tiles[0] * (uint32_t)g.tiles[1]));
    const int ox = 8 * tx - 1, oy = 8 * ty - 1, oz = 4 * tz - 1;
    stage_tile(g, G.vel, ox, oy, oz, s_tile);
    __syncthreads();
    // software pipeline: the next particle's index and position load while
    // this one is computed
    uint32_t j = jb + threadIdx.x;
    uint32_t pn = j < je ? G.perm[j] : 0u;
    float nx = 0.0f, ny = 0.0f, nz = 0.0f;
    if (j < je) {
        nx = G.x[0][pn];
        ny = G.x[1][pn];
        nz = G.x[2][pn];
    }
    for (; j < je; j += kAdjThreads) {
        const uint32_t p = pn;
        const float px = nx, py = ny, pz = nz;
        if (j + kAdjThreads < je) {
            pn = G.perm[j + kAdjThreads];
            nx = G.x[0][pn];
            ny = G.x[1][pn];
            nz = G.x[2][pn];
        }
        const ParticleAxes pa = particle_axes(g, px, py, pz, tx, ty, tz);
        float lx[3] = {0.0f, 0.0f, 0.0f};
        if (pa.ok) {
            g2p_adj_component<R, 0>(G, pa, s_tile, ox, oy, oz, j, px, lx);
            g2p_adj_component<R, 1>(G, pa, s_tile, ox, oy, oz, j, py, lx);
            g2p_adj_component<R, 2>(G, pa, s_tile, ox, oy, oz, j, pz, lx);
        } else {
            atomicOr(G.status, kFlagOutOfDomain);
            for (int a = 0; a < 3; ++a)
                for (int r = 0; r < R; ++r) G.mu[((int64_t)a * R + r) * G.count + j] = 0.0f;
        }
        if (G.accumulate) {  // three loads, then three stores
            const float o0 = G.out_x[0][p], o1 = G.out_x[1][p], o2 = G.out_x[2][p];
            lx[0] += o0;
            lx[1] += o1;
            lx[2] += o2;
        }
#pragma unroll
        for (int b = 0; b < 3; ++b) G.out_x[b][p] = lx[b];
    }
}

// ---------------------------------------------------------------- P2G adjoint gather
template <int R, int A>
__device__ __forceinline__ void p2g_adj_component(const AdjP2GArgs &Q, const ParticleAxes &pa,
                                                  const float *tile_m, const float *tile_v, int ox,
                                                  int oy, int oz, uint32_t p, float mt,
                                                  float (&lx)[3]) {
    constexpr int D = axis_degrees(R);
    const Axis &ax = A == 0 ? pa.fce[0] : pa.ctr[0];
    const Axis &ay = A == 1 ? pa.fce[1] : pa.ctr[1];
    const Axis &az = A == 2 ? pa.fce[2] : pa.ctr[2];
    const AxisFac fx = axis_fac(ax), fy = axis_fac(ay), fz = axis_fac(az);
    float X[D][3], dX[D][3], Y[D][3], dY[D][3], Z[D][3], dZ[D][3];
    p2g_rows<D>(fx, Q.dx, Q.inv_dx, X, dX);
    p2g_rows<D>(fy, Q.dx, Q.inv_dx, Y, dY);
    p2g_rows<D>(fz, Q.dx, Q.inv_dx, Z, dZ);
    const int lx0 = ax.base - ox, ly0 = ay.base - oy, lz0 = az.base - oz;
    float lmv[3][3][3], lm[3][3][3];
    read_stencil<A>(tile_v, lx0, ly0, lz0, lmv);
    read_stencil<A>(tile_m, lx0, ly0, lz0, lm);
    const int64_t cnt = Q.count;
    // the component's coefficients first (read-only path, all in flight at
    // once), then the coefficient adjoint and its stores
    const float *__restrict__ cin = Q.coeff + (int64_t)A * R * cnt + p;
    float *__restrict__ cout = Q.out_c + (int64_t)A * R * cnt + p;
    float c[D][D][D];
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b)
#pragma unroll
            for (int cc = 0; cc < D; ++cc)
                c[a][b][cc] = has_mode(R, a, b, cc) ? __ldg(cin + mode_index(a, b, cc) * cnt) : 0.0f;
    float lc[D][D][D];
    contract_modes<R, D>(X, Y, Z, lmv, lc);
    if (Q.accumulate) {  // the old values, all loaded before the first store
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
            for (int b = 0; b < D; ++b)
#pragma unroll
                for (int cc = 0; cc < D; ++cc)
                    lc[a][b][cc] = has_mode(R, a, b, cc)
                                       ? fmaf(mt, lc[a][b][cc], cout[mode_index(a, b, cc) * cnt])
                                       : 0.0f;
    } else {
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
            for (int b = 0; b < D; ++b)
#pragma unroll
                for (int cc = 0; cc < D; ++cc) lc[a][b][cc] *= mt;
    }
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b)
#pragma unroll
            for (int cc = 0; cc < D; ++cc)
                if (has_mode(R, a, b, cc)) cout[mode_index(a, b, cc) * cnt] = lc[a][b][cc];
    // position terms: momentum through the modes, mass through the weights
    float Dx = 0.0f, Dy = 0.0f, Dz = 0.0f;
    adj_position<R, D>(X, dX, Y, dY, Z, dZ, lmv, c, Dx, Dy, Dz);
    float Wx[1][3], dWx[1][3], Wy[1][3], dWy[1][3], Wz[1][3], dWz[1][3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        Wx[0][k] = X[0][k]; dWx[0][k] = dX[0][k];
        Wy[0][k] = Y[0][k]; dWy[0][k] = dY[0][k];
        Wz[0][k] = Z[0][k]; dWz[0][k] = dZ[0][k];
    }
    const float one[1][1][1] = {{{1.0f}}};
    adj_position<1, 1>(Wx, dWx, Wy, dWy, Wz, dWz, lm, one, Dx, Dy, Dz);
    lx[0] = fmaf(mt, Dx, lx[0]);
    lx[1] = fmaf(mt, Dy, lx[1]);
    lx[2] = fmaf(mt, Dz, lx[2]);
}

template <int R>
__global__ void __launch_bounds__(kAdjThreads) k_p2g_adjoint(AdjP2GArgs Q) {
    extern __shared__ float s_adj[];
    float *tile_m = s_adj, *tile_v = s_adj + kATileFloats;
    const GridGeom &g = Q.g;
    const uint32_t tile = blockIdx.x;
    const uint32_t jb = Q.cell_start[tile * 256], je = Q.cell_start[tile * 256 + 256];
    if (jb == je) return;
    const int tx = (int)(tile % (uint32_t)g.tiles[0]);
    const int ty = (int)((tile / (uint32_t)g.tiles[0]) % (uint32_t)g.tiles[1]);
    const int tz = (int)(tile / ((uint32_t)g.tiles[0] * (uint32_t)g.tiles[1]));
    const int ox = 8 * tx - 1, oy = 8 * ty - 1, oz = 4 * tz - 1;
    stage_tile(g, Q.lm, ox, oy, oz, tile_m);
    stage_tile(g, Q.lmv, ox, oy, oz, tile_v);
    __syncthreads();
    // software pipeline: the next particle's index, position and mass load
    // while this one is computed
    uint32_t j = jb + threadIdx.x;
    uint32_t pn = j < je ? Q.perm[j] : 0u;
    float nx = 0.0f, ny = 0.0f, nz = 0.0f, nm = 0.0f;
    if (j < je) {
        nx = Q.x[0][pn];
        ny = Q.x[1][pn];
        nz = Q.x[2][pn];
        nm = Q.mass[pn] + (Q.mass_abs ? Q.mass_abs[pn] : 0.0f);
    }
    for (; j < je; j += kAdjThreads) {
        const uint32_t p = pn;
        const float px = nx, py = ny, pz = nz, mt = nm;
        if (j + kAdjThreads < je) {
            pn = Q.perm[j + kAdjThreads];
            nx = Q.x[0][pn];
            ny = Q.x[1][pn];
            nz = Q.x[2][pn];
            nm = Q.mass[pn] + (Q.mass_abs ? Q.mass_abs[pn] : 0.0f);
        }
        const ParticleAxes pa = particle_axes(g, px, py, pz, tx, ty, tz);
        float lx[3] = {0.0f, 0.0f, 0.0f};
        if (pa.ok) {
            p2g_adj_component<R, 0>(Q, pa, tile_m, tile_v, ox, oy, oz, p, mt, lx);
            p2g_adj_component<R, 1>(Q, pa, tile_m, tile_v, ox, oy, oz, p, mt, lx);
            p2g_adj_component<R, 2>(Q, pa, tile_m, tile_v, ox, oy, oz, p, mt, lx);
        } else {
            atomicOr(Q.status, kFlagOutOfDomain);
            for (int a = 0; a < 3; ++a)
                for (int r = 0; r < R; ++r) {
                    float *o = Q.out_c + ((int64_t)a * R + r) * Q.count + p;
                    if (!Q.accumulate) *o = 0.0f;
                }
        }
        if (Q.accumulate) {  // three loads, then three stores
            const float o0 = Q.out_x[0][p], o1 = Q.out_x[1][p], o2 = Q.out_x[2][p];
            lx[0] += o0;
            lx[1] += o1;
            lx[2] += o2;
        }
#pragma unroll
        for (int b = 0; b < 3; ++b) Q.out_x[b][p] = lx[b];
    }
}

// ---------------------------------------------------------------- drivers
size_t adjoint_scratch_bytes(int64_t count, int R) {
    return (size_t)count * 3 * R * sizeof(float) + 512;
}

cudaError_t adjoint_g2p(const GridGeom &g, int64_t num_keys, int R, float dx,
                        const polypic_grid *grid, const polypic_particles *in, float dt,
                        const polypic_particles *bar_out, polypic_grid *bar_grid,
                        polypic_particles *bar_in, bool accumulate, uint32_t *status,
                        Workspace &ws, cudaStream_t s) {
    const int64_t tiles = num_keys / 256;
    if (in->count == 0) {  // nothing scatters: the grid adjoint is 0 (or unchanged)
        if (!accumulate)
            for (int a = 0; a < 3; ++a) {
                const size_t n = (size_t)(g.n[0] + (a == 0)) * (g.n[1] + (a == 1)) * (g.n[2] + (a == 2));
                cudaError_t e = cudaMemsetAsync(bar_grid->vel[a], 0, n * sizeof(float), s);
                if (e != cudaSuccess) return e;
            }
        return cudaSuccess;
    }
    float *mu = ws.take<float>((size_t)in->count * 3 * R);
    P2GArgs P{};
    P.scratch = ws.take<float>((size_t)tiles * kTileFloats);
    P.tile_live = ws.take<uint8_t>((size_t)tiles);
    if (ws.overflow) return cudaErrorInvalidValue;

    AdjG2PArgs G{};
    G.g = g;
    G.count = in->count;
    G.dt = dt;
    G.inv_dx = 1.0f / dx;
    for (int a = 0; a < 3; ++a) {
        G.vel[a] = grid->vel[a];
        G.x[a] = in->x[a];
        G.bar_x[a] = bar_out->x[a];
        G.out_x[a] = bar_in->x[a];
    }
    G.bar_c = static_cast<const float *>(bar_out->coeff);
    G.perm = in->perm;
    G.cell_start = in->cell_start;
    G.mu = mu;
    G.status = status;
    G.accumulate = accumulate;
    cudaError_t e = cudaErrorInvalidValue;
    if (R == 1) { k_g2p_adjoint<1><<<(int)tiles, kAdjThreads, 0, s>>>(G); e = cudaGetLastError(); }
    if (R == 4) { k_g2p_adjoint<4><<<(int)tiles, kAdjThreads, 0, s>>>(G); e = cudaGetLastError(); }
    if (R == 8) { k_g2p_adjoint<8><<<(int)tiles, kAdjThreads, 0, s>>>(G); e = cudaGetLastError(); }
    if (R == 27) { k_g2p_adjoint<27><<<(int)tiles, kAdjThreads, 0, s>>>(G); e = cudaGetLastError(); }
    if (e != cudaSuccess) return e;

    P.g = g;
    P.count = in->count;
    P.x = in->x[0];
    P.y = in->x[1];
    P.z = in->x[2];
    P.perm = in->perm;
    P.cell_start = in->cell_start;
    P.status = status;
    P.nblocks = (uint32_t)(num_keys / 32);
    P.s1 = P.s2 = 1.0f;  // the scatter's fit rows carry their own 1/dx powers
    P.mu = mu;
    P.inv_dx = 1.0f / dx;
    P.inv_dx2 = 1.0f / (dx * dx);
    return p2g_adjoint_scatter(P, bar_grid->vel, accumulate, R, s);
}

cudaError_t adjoint_p2g(const GridGeom &g, int64_t num_keys, int R, float dx,
                        const polypic_particles *in, const polypic_grid *bar_grid,
                        polypic_particles *bar_in, bool accumulate, uint32_t *status,
                        Workspace &ws, cudaStream_t s) {
    (void)ws;
    if (in->count == 0) return cudaSuccess;
    AdjP2GArgs Q{};
    Q.g = g;
    Q.count = in->count;
    Q.dx = dx;
    Q.inv_dx = 1.0f / dx;
    for (int a = 0; a < 3; ++a) {
        Q.lm[a] = bar_grid->mass[a];
        Q.lmv[a] = bar_grid->mom[a];
        Q.x[a] = in->x[a];
        Q.out_x[a] = bar_in->x[a];
    }
    Q.mass = in->mass;
    Q.mass_abs = in->mass_abs;
    Q.coeff = static_cast<const float *>(in->coeff);
    Q.out_c = static_cast<float *>(bar_in->coeff);
    Q.perm = in->perm;
    Q.cell_start = in->cell_start;
    Q.status = status;
    Q.accumulate = accumulate;
    const int64_t tiles = num_keys / 256;
    const int smem = 2 * kATileFloats * (int)sizeof(float);
#define POLYPIC_ADJ_CASE(RR)                                                        \
    if (R == RR) {                                                                  \
        k_p2g_adjoint<RR><<<(int)tiles, kAdjThreads, smem, s>>>(Q);                \
        return cudaGetLastError();                                                  \
    }
    POLYPIC_ADJ_CASE(1)
    POLYPIC_ADJ_CASE(4)
    POLYPIC_ADJ_CASE(8)
    POLYPIC_ADJ_CASE(27)
#undef POLYPIC_ADJ_CASE
    return cudaErrorInvalidValue;
}

}  // namespace polypic

// g2p_fit.cuh -- the G2P fit from a staged velocity footprint (Eqs 6-8,
// Section 3.3), used by the G2P kernels of g2p.cu.
//
// The fit is the transpose of P2G's sum factorisation with per-axis weights
//   G0_k = W_k,  G1_k = W_k z_k / mu2 = 4 F1_k,  G2_k = W_k g_k / d_2 = (1,-2,1)/2
// (z in cells): the quadratic fit is half the second difference for every t,
// so no denominator is formed; the guard zeroes G2 on a guarded axis.
#pragma once
#include "polypic_internal.cuh"

namespace polypic {

constexpr int kG2PThreads = 256;
// Staged footprint of a tile on face grid A, with a halo of H cells on every
// side: nodes [8 tx - 1 - H, ...) x [8 ty - 1 - H, ...) x [4 tz - 1 - H, ...);
// dims (11,10,6) (10,11,6) (10,10,7) for H = 0.
template <int H> struct Shape {
    template <int A> struct D {
        static constexpr int X = (A == 0 ? 11 : 10) + 2 * H, Y = (A == 1 ? 11 : 10) + 2 * H,
                             Z = (A == 2 ? 7 : 6) + 2 * H, N = X * Y * Z;
    };
    static constexpr int kOff1 = D<0>::N, kOff2 = D<0>::N + D<1>::N;
    static constexpr int kFloats = D<0>::N + D<1>::N + D<2>::N;
};
template <int A> using Tile = Shape<0>::D<A>;
constexpr int kVelTileOff1 = Shape<0>::kOff1, kVelTileOff2 = Shape<0>::kOff2;
constexpr int kVelTileFloats = Shape<0>::kFloats;

// Stages the three velocity footprints of tile (tx, ty, tz) with halo H
// (nodes outside a grid read as 0); the caller synchronises.
template <int H>
__device__ __forceinline__ void stage_velocity(const GridGeom &g, const float *const vel[3],
                                               int tx, int ty, int tz, float *s_tile) {
    const int ox = 8 * tx - 1 - H, oy = 8 * ty - 1 - H, oz = 4 * tz - 1 - H;
    auto stage = [&](int a, int X, int Y, int Z, int off) {
        const int dX = g.n[0] + (a == 0), dY = g.n[1] + (a == 1), dZ = g.n[2] + (a == 2);
        const float *src = vel[a];
        for (int i = threadIdx.x; i < X * Y * Z; i += blockDim.x) {
            const int lx = i % X, ly = (i / X) % Y, lz = i / (X * Y);
            const int gx = ox + lx, gy = oy + ly, gz = oz + lz;
            float v = 0.0f;
            if (gx >= 0 && gx < dX && gy >= 0 && gy < dY && gz >= 0 && gz < dZ)
                v = src[((int64_t)gz * dY + gy) * dX + gx];
            s_tile[off + i] = v;
        }
    };
    using S = Shape<H>;
    stage(0, S::template D<0>::X, S::template D<0>::Y, S::template D<0>::Z, 0);
    stage(1, S::template D<1>::X, S::template D<1>::Y, S::template D<1>::Z, S::kOff1);
    stage(2, S::template D<2>::X, S::template D<2>::Y, S::template D<2>::Z, S::kOff2);
}

__device__ __forceinline__ float2 gbc(float x) { return make_float2(x, x); }

// inv1 = 1/dx, inv2 = 1/dx^2 give physical coefficients; 1 and 1 give c dx^L.
template <int D>
__device__ __forceinline__ void fit_factors(const Stencil1D &s, bool guard, float inv1,
                                            float inv2, float (&G)[D][3]) {
#pragma unroll
    for (int k = 0; k < 3; ++k) G[0][k] = s.W[k];
    if constexpr (D > 1) {
        const float f = 4.0f * inv1;
#pragma unroll
        for (int k = 0; k < 3; ++k) G[1][k] = f * s.F1[k];
    }
    if constexpr (D > 2) {
        const float h = guard ? 0.0f : 0.5f * inv2;
        G[2][0] = h;
        G[2][1] = -2.0f * h;
        G[2][2] = h;
    }
}

// Eq 10's gradient form of the linear modes (4 modes only): the degree-1
// factor of an axis becomes dW_k/dx_p = (t - 1/2, -2t, t + 1/2) / dx, the
// x_p-derivative of the B-spline weights (inv1 = 1/dx, or 1 for c dx).
template <int D>
__device__ __forceinline__ void grad_w_factors(float t, float inv1, float (&G)[D][3]) {
    static_assert(D == 2, "the gradient form replaces the linear modes of the 4-mode set");
    G[1][0] = (t - 0.5f) * inv1;
    G[1][1] = -2.0f * t * inv1;
    G[1][2] = (t + 0.5f) * inv1;
}

// Fit of component A for one particle; Chat receives the dimensionless
// coefficients c dx^L in canonical order (only the first R entries are set).
// t: the staged values of face grid A, rows of TX nodes, planes of TY rows;
// (lx, ly, lz): the stencil's lowest node in it.  GRADW (4 modes): the
// linear modes take Eq 10's weight gradients; (tx, ty, tz) are the axes' t.
// PACK: the x and y contractions run two rows at a time through packed FP32
// FMAs, with the same bits as the scalar form (faster where the fit, not the
// coefficient stores, bounds the kernel: the 16-bit formats).
template <int R, int A, int TX, int TY, bool GRADW = false, bool PACK = false>
__device__ __forceinline__ void g2p_component(const float *t, int lx, int ly, int lz,
                                              const Stencil1D &sx, bool gx, const Stencil1D &sy,
                                              bool gy, const Stencil1D &sz, bool gz, float inv1,
                                              float inv2, float (&Chat)[R], float tx = 0.0f,
                                              float ty = 0.0f, float tz = 0.0f) {
    constexpr int D = axis_degrees(R);
    float Gx[D][3], Gy[D][3], Gz[D][3];
    fit_factors<D>(sx, gx, inv1, inv2, Gx);
    fit_factors<D>(sy, gy, inv1, inv2, Gy);
    fit_factors<D>(sz, gz, inv1, inv2, Gz);
    if constexpr (GRADW) {
        grad_w_factors<D>(tx, inv1, Gx);
        grad_w_factors<D>(ty, inv1, Gy);
        grad_w_factors<D>(tz, inv1, Gz);
    }
    float U2[D][D][3];
    if constexpr (!PACK) {
        // contract x
        float U1[D][3][3];
#pragma unroll
        for (int kz = 0; kz < 3; ++kz)
#pragma unroll
            for (int ky = 0; ky < 3; ++ky) {
                const float *row = t + ((lz + kz) * TY + (ly + ky)) * TX + lx;
                const float v0 = row[0], v1 = row[1], v2 = row[2];
#pragma unroll
                for (int a = 0; a < D; ++a)
                    U1[a][ky][kz] = fmaf(Gx[a][0], v0, fmaf(Gx[a][1], v1, Gx[a][2] * v2));
            }
        // contract y
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
            for (int b = 0; b < D; ++b)
#pragma unroll
                for (int kz = 0; kz < 3; ++kz)
                    U2[a][b][kz] = fmaf(Gy[b][0], U1[a][0][kz],
                                        fmaf(Gy[b][1], U1[a][1][kz], Gy[b][2] * U1[a][2][kz]));
    } else {
        // contract x, then y; the rows kz = 0, 1 travel as float2 pairs through
        // packed FP32 FMAs (each lane rounds as fmaf does, in the same order, so
        // the values carry the same bits as scalar FMAs), the row kz = 2 scalar
        float2 U1p[D][3];
        float U1s[D][3];
#pragma unroll
        for (int ky = 0; ky < 3; ++ky) {
            const float *r0 = t + ((lz + 0) * TY + (ly + ky)) * TX + lx;
            const float *r1 = t + ((lz + 1) * TY + (ly + ky)) * TX + lx;
            const float *r2 = t + ((lz + 2) * TY + (ly + ky)) * TX + lx;
            const float2 v0 = make_float2(r0[0], r1[0]), v1 = make_float2(r0[1], r1[1]),
                         v2 = make_float2(r0[2], r1[2]);
            const float w0 = r2[0], w1 = r2[1], w2 = r2[2];
#pragma unroll
            for (int a = 0; a < D; ++a) {
                U1p[a][ky] = __ffma2_rn(gbc(Gx[a][0]), v0,
                                        __ffma2_rn(gbc(Gx[a][1]), v1, __fmul2_rn(gbc(Gx[a][2]), v2)));
                U1s[a][ky] = fmaf(Gx[a][0], w0, fmaf(Gx[a][1], w1, Gx[a][2] * w2));
            }
        }
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
            for (int b = 0; b < D; ++b) {
                const float2 p = __ffma2_rn(
                    gbc(Gy[b][0]), U1p[a][0],
                    __ffma2_rn(gbc(Gy[b][1]), U1p[a][1], __fmul2_rn(gbc(Gy[b][2]), U1p[a][2])));
                U2[a][b][0] = p.x;
                U2[a][b][1] = p.y;
                U2[a][b][2] = fmaf(Gy[b][0], U1s[a][0],
                                   fmaf(Gy[b][1], U1s[a][1], Gy[b][2] * U1s[a][2]));
            }
    }
    // contract z
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b)
#pragma unroll
            for (int c = 0; c < D; ++c)
                if (has_mode(R, a, b, c))
                    Chat[mode_index(a, b, c)] = fmaf(Gz[c][0], U2[a][b][0],
                                                     fmaf(Gz[c][1], U2[a][b][1], Gz[c][2] * U2[a][b][2]));
}

}  // namespace polypic

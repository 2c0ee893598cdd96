// p2g_kernel.cuh -- the per-particle pieces of the P2G transfer (Eqs 1-5,
// 13, 15-19) used by the tile kernel of p2g_tiles.cuh: cp.async staging of a
// particle, the sum-factorised accumulation into a lane's padded 4 x 3 x 3
// footprint, and the slot of a lane's particle in a round.
#pragma once
#include "p2g.cuh"

namespace polypic {


template <int A> struct TileReg {
    static constexpr int X = tile_x(A), Y = tile_y(A), Z = tile_z(A);
};

// 1-D factors of one axis: F[a][k] = W_k f_a(z_k) (z in cells), a < D.
template <int D>
__device__ __forceinline__ void axis_factors(const Stencil1D &s, float (&F)[D][3]) {
#pragma unroll
    for (int k = 0; k < 3; ++k) F[0][k] = s.W[k];
    if constexpr (D > 1) {
#pragma unroll
        for (int k = 0; k < 3; ++k) F[1][k] = s.F1[k];
    }
    if constexpr (D > 2) {
        F[2][0] = s.phi;
        F[2][1] = -2.0f * s.phi;
        F[2][2] = s.phi;
    }
}

// Degrees (a, b, c) along (x, y, z) of the tensor entry (du, dv, dw) for the
// component-A ordering u = A, (v, w) = the other two axes in increasing order.
template <int A> __host__ __device__ constexpr int deg_x(int du, int dv, int dw) {
    return A == 0 ? du : dv;
}
template <int A> __host__ __device__ constexpr int deg_y(int du, int dv, int dw) {
    return A == 0 ? dv : (A == 1 ? du : dw);
}
template <int A> __host__ __device__ constexpr int deg_z(int du, int dv, int dw) {
    return A == 2 ? du : dw;
}

// ---------------------------------------------------------------- staging
// Each lane prefetches its next particles with cp.async (4-byte copies) into
// a private multi-stage buffer laid out [stage][value][lane] (conflict-free):
// x, y, z, m, m_abs, s_p, the particle index, then the coefficient words: one
// per mode for FP32, one per pair of modes for the 16-bit formats (whose
// words hold two codes).  With Eq 12's affine map (AFF) six more words
// follow: the linear-mode coefficients of the two other components (their C
// rows).
__host__ __device__ constexpr int coeff_words(int R, int FMT) {
    return FMT == POLYPIC_COEFF_F32 ? R : (R + 1) / 2;
}
template <int R, bool AFF = false, int FMT = POLYPIC_COEFF_F32> struct Stage {
    static constexpr int kX = 0, kY = 1, kZ = 2, kM = 3, kMabs = 4, kScale = 5, kIdx = 6, kC = 7;
    static constexpr int kL = kC + coeff_words(R, FMT);
    static constexpr int NV = kL + (AFF ? 6 : 0);
};

__device__ __forceinline__ void cp_async4(float *dst, const void *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <int R, int FMT, int A, bool ADJ, bool AFF = false>
__device__ __forceinline__ void stage_particle(const P2GArgs &P, uint32_t p, uint32_t slot,
                                               float *st, int lane) {
    using S = Stage<R, AFF, FMT>;
    cp_async4(st + S::kX * 32 + lane, P.x + p);
    cp_async4(st + S::kY * 32 + lane, P.y + p);
    cp_async4(st + S::kZ * 32 + lane, P.z + p);
    if constexpr (ADJ) {
        // adjoint scatter: unit weight, coefficients mu (slot order) from scratch
        st[S::kM * 32 + lane] = 1.0f;
        const float *c = P.mu + (int64_t)A * R * P.count + slot;
#pragma unroll
        for (int r = 0; r < R; ++r, c += P.count) cp_async4(st + (S::kC + r) * 32 + lane, c);
        return;
    }
    cp_async4(st + S::kM * 32 + lane, P.mass + p);
    if (P.mass_abs) cp_async4(st + S::kMabs * 32 + lane, P.mass_abs + p);
    reinterpret_cast<uint32_t *>(st)[S::kIdx * 32 + lane] = p;
    if constexpr (FMT == POLYPIC_COEFF_F32) {
        // row r of component A starts (A R + r) * count floats in
        const float *c = reinterpret_cast<const float *>(P.coeff) + (int64_t)A * R * P.count + p;
#pragma unroll
        for (int r = 0; r < R; ++r, c += P.count) cp_async4(st + (S::kC + r) * 32 + lane, c);
        if constexpr (AFF) {
            const float *cf = reinterpret_cast<const float *>(P.coeff) + p;
#pragma unroll
            for (int o = 0; o < 2; ++o) {
                const int a2 = o < A ? o : o + 1;  // the other two components, ascending
#pragma unroll
                for (int b = 0; b < 3; ++b)
                    cp_async4(st + (S::kL + 3 * o + b) * 32 + lane,
                              cf + ((int64_t)a2 * R + 1 + b) * P.count);
            }
        }
    } else {
        // 16-bit codes: word (A H + k, p), H = (R + 1) / 2, holds modes 2k and 2k + 1
        cp_async4(st + S::kScale * 32 + lane, P.scale + p);
        constexpr int H = coeff_words(R, FMT);
        const uint32_t *w = reinterpret_cast<const uint32_t *>(P.coeff) + (int64_t)A * H * P.count + p;
#pragma unroll
        for (int k = 0; k < H; ++k, w += P.count) cp_async4(st + (S::kC + k) * 32 + lane, w);
    }
}

// A lane's footprint on face grid A: 4 x 3 x 3 nodes (d along the face axis,
// the lowest node cell - 1; kv, kw along the other two axes), mass and
// momentum.  The kw = 0, 1 entries are float2 pairs so that packed FP32 FMAs
// update both at once; each lane of a packed FMA rounds as fmaf does, so the
// sums carry the same bits as scalar FMAs in the same order.
struct Foot {
    float2 m2[4][3], v2[4][3];  // kw = 0 (x), kw = 1 (y)
    float m1[4][3], v1[4][3];   // kw = 2
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int d = 0; d < 4; ++d)
#pragma unroll
            for (int kv = 0; kv < 3; ++kv) {
                m2[d][kv] = v2[d][kv] = make_float2(0.0f, 0.0f);
                m1[d][kv] = v1[d][kv] = 0.0f;
            }
    }
    __device__ __forceinline__ float m(int d, int kv, int kw) const {
        return kw == 0 ? m2[d][kv].x : (kw == 1 ? m2[d][kv].y : m1[d][kv]);
    }
    __device__ __forceinline__ float v(int d, int kv, int kw) const {
        return kw == 0 ? v2[d][kv].x : (kw == 1 ? v2[d][kv].y : v1[d][kv]);
    }
    __device__ __forceinline__ void add(int d, int kv, int kw, float dm, float dv) {
        if (kw == 0) {
            m2[d][kv].x += dm;
            v2[d][kv].x += dv;
        } else if (kw == 1) {
            m2[d][kv].y += dm;
            v2[d][kv].y += dv;
        } else {
            m1[d][kv] += dm;
            v1[d][kv] += dv;
        }
    }
};

__device__ __forceinline__ float2 bcast(float x) { return make_float2(x, x); }

// One particle's contribution to the lane's padded footprint on grid A.
// fu: stencil along A (face offset), fv / fw: the other two axes (centre).
// Fit factors of the G2P least-squares fit in physical units (the adjoint
// scatter): G0 = W, G1 = 4 F1 / dx, G2 = (1, -2, 1) / (2 dx^2), zero when guarded.
template <int D>
__device__ __forceinline__ void fit_rows(const Stencil1D &s, bool guard, float inv1, float inv2,
                                         float (&G)[D][3]) {
#pragma unroll
    for (int k = 0; k < 3; ++k) G[0][k] = s.W[k];
    if constexpr (D > 1) {
#pragma unroll
        for (int k = 0; k < 3; ++k) G[1][k] = 4.0f * inv1 * s.F1[k];
    }
    if constexpr (D > 2) {
        const float h = guard ? 0.0f : 0.5f * inv2;
        G[2][0] = h;
        G[2][1] = -2.0f * h;
        G[2][2] = h;
    }
}

// Eq 12's affine map: M = (I + dt C)^-1 with C_ab = c_{a, 1+b} (the linear
// modes of all three components, component A's own row from its staged
// coefficients), the identity when |det(I + dt C)| < 1e-6.
template <int R, int A>
__device__ __forceinline__ void affine_inverse(const float *st, int lane, float dt,
                                               float (&M)[3][3]) {
    using S = Stage<R, true>;
    float C[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const int slot = a == A ? S::kC + 1 + b : S::kL + 3 * (a < A ? a : a - 1) + b;
            C[a][b] = fmaf(dt, st[slot * 32 + lane], a == b ? 1.0f : 0.0f);
        }
    const float m00 = C[1][1] * C[2][2] - C[1][2] * C[2][1];
    const float m01 = C[0][2] * C[2][1] - C[0][1] * C[2][2];
    const float m02 = C[0][1] * C[1][2] - C[0][2] * C[1][1];
    const float m10 = C[1][2] * C[2][0] - C[1][0] * C[2][2];
    const float m11 = C[0][0] * C[2][2] - C[0][2] * C[2][0];
    const float m12 = C[0][2] * C[1][0] - C[0][0] * C[1][2];
    const float m20 = C[1][0] * C[2][1] - C[1][1] * C[2][0];
    const float m21 = C[0][1] * C[2][0] - C[0][0] * C[2][1];
    const float m22 = C[0][0] * C[1][1] - C[0][1] * C[1][0];
    const float det = C[0][0] * m00 + C[0][1] * m10 + C[0][2] * m20;
    if (fabsf(det) < 1e-6f) {
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) M[a][b] = a == b ? 1.0f : 0.0f;
        return;
    }
    const float id = 1.0f / det;
    M[0][0] = m00 * id; M[0][1] = m01 * id; M[0][2] = m02 * id;
    M[1][0] = m10 * id; M[1][1] = m11 * id; M[1][2] = m12 * id;
    M[2][0] = m20 * id; M[2][1] = m21 * id; M[2][2] = m22 * id;
}

// The 4-mode set under the map: sum_r c_r s_r(M z) = c_0 + sum_g (sum_b
// c_{1+b} M_bg) z_g, so component A's linear coefficients become (M^T c)_g.
template <int R, int A>
__device__ __forceinline__ void affine_linear(const float *st, int lane, float dt,
                                              float (&cl)[3]) {
    using S = Stage<R, true>;
    float M[3][3];
    affine_inverse<R, A>(st, lane, dt, M);
    const float c1 = st[(S::kC + 1) * 32 + lane], c2 = st[(S::kC + 2) * 32 + lane],
                c3 = st[(S::kC + 3) * 32 + lane];
#pragma unroll
    for (int g = 0; g < 3; ++g) cl[g] = c1 * M[0][g] + c2 * M[1][g] + c3 * M[2][g];
}

// 8 and 27 modes under the map are not separable per axis: every stencil node
// evaluates s_r(xi) = f_a(xi_x) f_b(xi_y) f_c(xi_z) at xi = M z, with
// f_2(xi) = xi^2 - kappa xi - mu2 from the particle's own (unmapped) axis
// constants kappa = dx t (1 - 4t^2), mu2 = dx^2 / 4, and adds
// mt w(node) sum_r c_r s_r(xi) into the padded footprint (FP32, physical c).
template <int R, int A>
__device__ __forceinline__ void accumulate_mapped(const P2GArgs &P, const float *st, int lane,
                                                  float mt, int shift, float tu, float tv,
                                                  float tw, const Stencil1D &fu,
                                                  const Stencil1D &fv, const Stencil1D &fw,
                                                  Foot &F) {
    using S = Stage<R, true>;
    constexpr int D = axis_degrees(R);
    float M[3][3];
    affine_inverse<R, A>(st, lane, P.map_dt, M);
    const float dx = P.dxpow[1], mu2 = 0.25f * P.dxpow[2];
    // axes u (= A), v, w as x, y, z indices, and each axis's node offsets
    constexpr int U = A, V = A == 0 ? 1 : 0, Wx = A == 2 ? 1 : 2;
    const float t3[3] = {tu, tv, tw};
    float kap[3];   // by x, y, z
    float Mz[3][3][3];  // [axis u/v/w][node k][component of xi]
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        const int ax = e == 0 ? U : (e == 1 ? V : Wx);
        const float t = t3[e];
        kap[ax] = dx * t * ((1.0f - 2.0f * t) * (1.0f + 2.0f * t));
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float z = ((float)(k - 1) - t) * dx;
#pragma unroll
            for (int g = 0; g < 3; ++g) Mz[e][k][g] = M[g][ax] * z;
        }
    }
    float c[R];
#pragma unroll
    for (int r = 0; r < R; ++r) c[r] = st[(S::kC + r) * 32 + lane];
#pragma unroll
    for (int ku = 0; ku < 3; ++ku)
#pragma unroll
        for (int kv = 0; kv < 3; ++kv)
#pragma unroll
            for (int kw = 0; kw < 3; ++kw) {
                float f[3][3];  // [axis x/y/z][degree]
#pragma unroll
                for (int g = 0; g < 3; ++g) {
                    const float xi = Mz[0][ku][g] + Mz[1][kv][g] + Mz[2][kw][g];
                    f[g][0] = 1.0f;
                    f[g][1] = xi;
                    f[g][2] = fmaf(xi, xi - kap[g], -mu2);
                }
                float Sn = 0.0f;
#pragma unroll
                for (int a = 0; a < D; ++a) {
                    float Sa = 0.0f;
#pragma unroll
                    for (int b = 0; b < D; ++b) {
                        float Sb = 0.0f;
#pragma unroll
                        for (int cc = 0; cc < D; ++cc)
                            if (has_mode(R, a, b, cc))
                                Sb = fmaf(c[mode_index(a, b, cc)], f[2][cc], Sb);
                        Sa = fmaf(Sb, f[1][b], Sa);
                    }
                    Sn = fmaf(Sa, f[0][a], Sn);
                }
                // node ku lands on footprint row ku + shift; both candidate
                // rows are static indices (the footprint stays in registers)
                const float w = mt * fu.W[ku] * fv.W[kv] * fw.W[kw];
                const float wS = w * Sn;
                F.add(ku, kv, kw, shift ? 0.0f : w, shift ? 0.0f : wS);
                F.add(ku + 1, kv, kw, shift ? w : 0.0f, shift ? wS : 0.0f);
            }
}

template <int R, int FMT, int A, bool ADJ, bool AFF = false>
__device__ __forceinline__ void accumulate(const P2GArgs &P, const float *st, int lane, float mt,
                                           int shift, const Stencil1D &fu, const Stencil1D &fv,
                                           const Stencil1D &fw, bool gu, bool gv, bool gw, Foot &F,
                                           float tu = 0.0f, float tv = 0.0f, float tw = 0.0f) {
    using S = Stage<R, AFF, FMT>;
    if constexpr (AFF && R > 4) {
        accumulate_mapped<R, A>(P, st, lane, mt, shift, tu, tv, tw, fu, fv, fw, F);
        return;
    }
    float cl[3] = {0.0f, 0.0f, 0.0f};
    if constexpr (AFF) affine_linear<R, A>(st, lane, P.map_dt, cl);
    constexpr int D = axis_degrees(R);
    const float cscale = FMT == POLYPIC_COEFF_F32 ? 1.0f : st[S::kScale * 32 + lane];
    float Fu[D][3], Fv[D][3], Fw[D][3];
    if constexpr (ADJ) {
        fit_rows<D>(fu, gu, P.inv_dx, P.inv_dx2, Fu);
        fit_rows<D>(fv, gv, P.inv_dx, P.inv_dx2, Fv);
        fit_rows<D>(fw, gw, P.inv_dx, P.inv_dx2, Fw);
    } else {
        axis_factors<D>(fu, Fu);
        axis_factors<D>(fv, Fv);
        axis_factors<D>(fw, Fw);
    }
    // FP32 coefficients are physical: the caller's stencils carry dx^a in
    // their degree-a factors.  The momentum weight (mass, and the 16-bit scale
    // s_p) goes into the u factors once.
    const float W0[3] = {Fu[0][0], Fu[0][1], Fu[0][2]};
    const float mom_scale = FMT == POLYPIC_COEFF_F32 ? mt : mt * cscale;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int k = 0; k < 3; ++k) Fu[a][k] *= mom_scale;
    // mass weights first (padded along u: node d = k + shift)
    if constexpr (!ADJ) {
        float w0, w1, w2;
        if constexpr (FMT == POLYPIC_COEFF_F32) {
            w0 = Fu[0][0];
            w1 = Fu[0][1];
            w2 = Fu[0][2];
        } else {
            w0 = mt * W0[0];
            w1 = mt * W0[1];
            w2 = mt * W0[2];
        }
        const float Wm[4] = {shift ? 0.0f : w0, shift ? w0 : w1, shift ? w1 : w2, shift ? w2 : 0.0f};
        const float2 fw0 = make_float2(Fw[0][0], Fw[0][1]);
#pragma unroll
        for (int kv = 0; kv < 3; ++kv) {
            const float2 wvw = __fmul2_rn(bcast(Fv[0][kv]), fw0);
            const float wvw2 = Fv[0][kv] * Fw[0][2];
#pragma unroll
            for (int d = 0; d < 4; ++d) {
                F.m2[d][kv] = __ffma2_rn(bcast(Wm[d]), wvw, F.m2[d][kv]);
                F.m1[d][kv] = fmaf(Wm[d], wvw2, F.m1[d][kv]);
            }
        }
    }
    (void)W0;
    // momentum, streamed over the degree du along u: contract w, then v, then
    // u into the padded footprint (kw = 0, 1 as packed pairs, kw = 2 scalar)
    float2 fw2[D];
#pragma unroll
    for (int dw = 0; dw < D; ++dw) fw2[dw] = make_float2(Fw[dw][0], Fw[dw][1]);
#pragma unroll
    for (int du = 0; du < D; ++du) {
        float C[D][D];
#pragma unroll
        for (int dv = 0; dv < D; ++dv)
#pragma unroll
            for (int dw = 0; dw < D; ++dw) {
                const int a = deg_x<A>(du, dv, dw), b = deg_y<A>(du, dv, dw),
                          c = deg_z<A>(du, dv, dw);
                C[dv][dw] = 0.0f;
                if (has_mode(R, a, b, c)) {
                    const int r = mode_index(a, b, c);
                    if constexpr (AFF) {
                        C[dv][dw] = r >= 1 && r <= 3 ? cl[r - 1] : st[(S::kC + r) * 32 + lane];
                    } else if constexpr (FMT == POLYPIC_COEFF_F32) {
                        C[dv][dw] = st[(S::kC + r) * 32 + lane];
                    } else {
                        // mode r is the low (r even) or high (r odd) half of word r / 2
                        const uint32_t word =
                            reinterpret_cast<const uint32_t *>(st)[(S::kC + r / 2) * 32 + lane];
                        C[dv][dw] = Codec<FMT>::decode((uint16_t)((r & 1) ? word >> 16 : word));
                    }
                }
            }
        float2 T1p[D];
        float T1s[D];
#pragma unroll
        for (int dv = 0; dv < D; ++dv) {
            float2 sp = make_float2(0.0f, 0.0f);
            float ss = 0.0f;
#pragma unroll
            for (int dw = 0; dw < D; ++dw)
                if (has_mode(R, deg_x<A>(du, dv, dw), deg_y<A>(du, dv, dw), deg_z<A>(du, dv, dw))) {
                    sp = __ffma2_rn(bcast(C[dv][dw]), fw2[dw], sp);
                    ss = fmaf(C[dv][dw], Fw[dw][2], ss);
                }
            T1p[dv] = sp;
            T1s[dv] = ss;
        }
        const float f0 = Fu[du][0], f1 = Fu[du][1], f2 = Fu[du][2];
        const float Gu[4] = {shift ? 0.0f : f0, shift ? f0 : f1, shift ? f1 : f2, shift ? f2 : 0.0f};
#pragma unroll
        for (int kv = 0; kv < 3; ++kv) {
            float2 tp = make_float2(0.0f, 0.0f);
            float ts = 0.0f;
#pragma unroll
            for (int dv = 0; dv < D; ++dv) {
                tp = __ffma2_rn(T1p[dv], bcast(Fv[dv][kv]), tp);
                ts = fmaf(T1s[dv], Fv[dv][kv], ts);
            }
#pragma unroll
            for (int d = 0; d < 4; ++d) {
                F.v2[d][kv] = __ffma2_rn(tp, bcast(Gu[d]), F.v2[d][kv]);
                F.v1[d][kv] = fmaf(ts, Gu[d], F.v1[d][kv]);
            }
        }
    }
}

// Slot of the lane's particle in round q (every lane must call it).
__device__ __forceinline__ uint32_t round_slot(uint32_t bs, uint32_t n_c, uint32_t q,
                                               unsigned lt) {
    const uint32_t before = __reduce_add_sync(0xffffffffu, min(n_c, q));
    const unsigned mask = __ballot_sync(0xffffffffu, n_c > q);
    return bs + before + __popc(mask & lt);
}

// Rounds in flight per lane (cp.async groups).  Two measured fastest at 27
// modes (three were 2% slower, four 8%: the ring takes shared memory from
// L1).
#ifndef POLYPIC_P2G_STAGES
#define POLYPIC_P2G_STAGES 2
#endif
constexpr int kStages = POLYPIC_P2G_STAGES;
}  // namespace polypic

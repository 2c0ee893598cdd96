// polypic_internal.cuh -- device-side building blocks shared by the kernels of
// libpolypic (sm_103a).  Nothing here is visible through the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "polypic.h"

namespace polypic {

// ---------------------------------------------------------------- status bits
enum : uint32_t {
    kFlagOutOfDomain = 1u,
    kFlagNonFinite = 2u,
    kFlagNotConverged = 4u,
    kFlagTimeout = 8u,
};

// ---------------------------------------------------------------- geometry
// Everything a kernel needs to know about the grid, passed by value.
struct GridGeom {
    int n[3];          // cells per axis
    int tiles[3];      // key tiles per axis: ceil(n / (8, 8, 4))
    float dx;          // cell width (FP32)
    float inv_dx;      // (float)(1.0 / dx), the FP32 decision factor
    float lo[3];       // advection clamp: 1.5 dx
    float hi[3];       // (n - 1.5) dx
};

struct polypic_ctx_impl;  // fwd

// Face grid a dims.
__host__ __device__ inline int face_dim(const GridGeom &g, int a, int b) {
    return g.n[b] + (a == b ? 1 : 0);
}

// ---------------------------------------------------------------- key layout
// key = tile * 256 + block_in_tile * 32 + cell_in_block; tiles 8x8x4 cells,
// blocks 4x4x2 cells, x fastest at every level.
__host__ __device__ inline uint32_t cell_key(const GridGeom &g, int i, int j, int k) {
    uint32_t tile = ((uint32_t)(k >> 2) * (uint32_t)g.tiles[1] + (uint32_t)(j >> 3)) *
                        (uint32_t)g.tiles[0] + (uint32_t)(i >> 3);
    uint32_t blk = ((i >> 2) & 1) | (((j >> 2) & 1) << 1) | (((k >> 1) & 1) << 2);
    uint32_t cell = (i & 3) | ((j & 3) << 2) | ((k & 1) << 4);
    return (tile << 8) | (blk << 5) | cell;
}

// Lowest cell (i, j, k) of block number b (b = key >> 5).
__host__ __device__ inline void block_origin(const GridGeom &g, uint32_t b, int &i0, int &j0,
                                             int &k0) {
    uint32_t tile = b >> 3, bit = b & 7u;
    uint32_t tx = tile % (uint32_t)g.tiles[0];
    uint32_t rest = tile / (uint32_t)g.tiles[0];
    uint32_t ty = rest % (uint32_t)g.tiles[1];
    uint32_t tz = rest / (uint32_t)g.tiles[1];
    i0 = (int)(tx * 8 + (bit & 1) * 4);
    j0 = (int)(ty * 8 + ((bit >> 1) & 1) * 4);
    k0 = (int)(tz * 4 + ((bit >> 2) & 1) * 2);
}

// Block number of the block whose origin is (4 bx, 4 by, 2 bz).
__host__ __device__ inline uint32_t block_of(const GridGeom &g, int bx, int by, int bz) {
    return cell_key(g, bx * 4, by * 4, bz * 2) >> 5;
}

// ---------------------------------------------------------------- FP32 decisions
// Rounded-per-operation FP32 arithmetic (no contraction into FMA) for every
// value that decides an integer.  __fmul_rn etc. are never fused.
__device__ __forceinline__ float cell_coord(float x, float inv_dx) { return __fmul_rn(x, inv_dx); }

__device__ __forceinline__ int cell_index(float v, int n) {
    float f = floorf(v);
    if (!(f >= 0.0f)) return 0;
    if (f > (float)(n - 1)) return n - 1;
    return (int)f;
}

// Valid region: 1 <= v < n - 1 (NaN fails).
__device__ __forceinline__ bool coord_valid(float v, int n) {
    return v >= 1.0f && v < (float)(n - 1);
}

// One axis of one particle on one face-grid type.
// face = true: offset o = 0 (the grid of this component), else o = 1/2.
struct Axis {
    int base;      // lowest stencil node
    float t;       // offset from the middle node, in cells, [-1/2, 1/2)
    bool guard;    // q = (1-2t)(1+2t) < 2^-10 in FP32
};

__device__ __forceinline__ Axis axis_decide(float v, bool face) {
    Axis a;
    float X = face ? v : __fsub_rn(v, 0.5f);
    float fb = floorf(__fsub_rn(X, 0.5f));
    a.base = (int)fb;
    a.t = __fsub_rn(X, __fadd_rn(fb, 1.0f));
    float tt = __fmul_rn(2.0f, a.t);
    float q = __fmul_rn(__fsub_rn(1.0f, tt), __fadd_rn(1.0f, tt));
    a.guard = q < 0x1p-10f;
    return a;
}

// ---------------------------------------------------------------- closed forms
// Dimensionless per-node factors of the quadratic B-spline stencil
// (z measured in cells):
//   W_k  = N(.)                 = (1/2 (1/2 - t)^2, 3/4 - t^2, 1/2 (1/2 + t)^2)
//   F1_k = W_k z_k              = (-(1+t)(1-2t)^2/8, t(4t^2-3)/4, (1-t)(1+2t)^2/8)
//   F2_k = W_k g(z_k)           = phi (1, -2, 1),  phi = q^2 (3 - 4t^2) / 32
// (q = 1 - 4t^2).  These follow from mu2 = 1/4, mu3/mu2 = t(1 - 4t^2) for
// this kernel; F2 carries the d_2 = q^2 (3 - 4t^2)/16 factor, so the fit of
// the quadratic mode needs no division:
//   G0_k = W_k, G1_k = F1_k / mu2 = 4 F1_k, G2_k = F2_k / d_2 = (1, -2, 1)/2.
struct Stencil1D {
    float W[3];
    float F1[3];
    float phi;
};

__device__ __forceinline__ Stencil1D stencil_1d(float t) {
    Stencil1D s;
    float a = 0.5f - t, b = 0.5f + t;
    s.W[0] = 0.5f * a * a;
    s.W[1] = 0.75f - t * t;
    s.W[2] = 0.5f * b * b;
    float om = 1.0f - 2.0f * t, op = 1.0f + 2.0f * t;
    s.F1[0] = -(1.0f + t) * om * om * 0.125f;
    s.F1[1] = t * (4.0f * t * t - 3.0f) * 0.25f;
    s.F1[2] = (1.0f - t) * op * op * 0.125f;
    float q = om * op;
    s.phi = q * q * (3.0f - 4.0f * t * t) * (1.0f / 32.0f);
    return s;
}

// The same factors with F1 and phi multiplied by s1 and s2 (s1 = dx and
// s2 = dx^2 turn them into physical units for FP32 coefficients), F1 formed
// as its definition W_k z_k with z = (-1 - t, -t, 1 - t) in cells.
__device__ __forceinline__ Stencil1D stencil_1d_scaled(float t, float s1, float s2) {
    Stencil1D s;
    float a = 0.5f - t, b = 0.5f + t;
    s.W[0] = 0.5f * a * a;
    s.W[1] = 0.75f - t * t;
    s.W[2] = 0.5f * b * b;
    s.F1[0] = s.W[0] * fmaf(-t, s1, -s1);
    s.F1[1] = s.W[1] * (-t * s1);
    s.F1[2] = s.W[2] * fmaf(-t, s1, s1);
    float q = (1.0f - 2.0f * t) * (1.0f + 2.0f * t);
    s.phi = q * q * (3.0f - 4.0f * t * t) * (s2 * (1.0f / 32.0f));
    return s;
}

// ---------------------------------------------------------------- modes
// Canonical mode index of the per-axis degrees (a, b, c), or -1.
__host__ __device__ constexpr int mode_index(int a, int b, int c) {
    if (a < 2 && b < 2 && c < 2) {
        const int idx = a + 2 * b + 4 * c;  // (000)(100)(010)(110)(001)(101)(011)(111)
        return idx == 0 ? 0 : idx == 1 ? 1 : idx == 2 ? 2 : idx == 4 ? 3
             : idx == 3 ? 4 : idx == 5 ? 5 : idx == 6 ? 6 : 7;
    }
    int r = 8;
    for (int cc = 0; cc < 3; ++cc)
        for (int bb = 0; bb < 3; ++bb)
            for (int aa = 0; aa < 3; ++aa)
                if (aa == 2 || bb == 2 || cc == 2) {
                    if (aa == a && bb == b && cc == c) return r;
                    ++r;
                }
    return -1;
}

__host__ __device__ constexpr bool has_mode(int R, int a, int b, int c) {
    return mode_index(a, b, c) >= 0 && mode_index(a, b, c) < R;
}

// Per-axis degree count of an R-mode set.
__host__ __device__ constexpr int axis_degrees(int R) { return R == 1 ? 1 : (R == 27 ? 3 : 2); }

// Total degree L_r of mode r (host + device).
__host__ __device__ constexpr int mode_degree(int r) {
    int rr = 0;
    for (int c = 0; c < 3; ++c)
        for (int b = 0; b < 3; ++b)
            for (int a = 0; a < 3; ++a)
                if (mode_index(a, b, c) == r) rr = a + b + c;
    return rr;
}

// ---------------------------------------------------------------- coefficient codec
template <int FMT> struct Codec;
template <> struct Codec<POLYPIC_COEFF_F32> {
    using T = float;
    __device__ static float load(const float *p) { return __ldg(p); }
};
template <> struct Codec<POLYPIC_COEFF_BF16> {
    using T = __nv_bfloat16;
    __device__ static float load(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
    __device__ static float decode(uint16_t bits) {
        return __bfloat162float(__ushort_as_bfloat16(bits));
    }
    __device__ static __nv_bfloat16 encode(float v) { return __float2bfloat16_rn(v); }
    __device__ static uint32_t bits(__nv_bfloat16 v) { return __bfloat16_as_ushort(v); }
};
template <> struct Codec<POLYPIC_COEFF_F16> {
    using T = __half;
    __device__ static float load(const __half *p) { return __half2float(*p); }
    __device__ static float decode(uint16_t bits) { return __half2float(__ushort_as_half(bits)); }
    __device__ static __half encode(float v) { return __float2half_rn(v); }
    __device__ static uint32_t bits(__half v) { return __half_as_ushort(v); }
};

// ---------------------------------------------------------------- launch helpers
// Carves 256-byte-aligned pieces out of the caller's workspace.  A request
// beyond its end returns nullptr and sets `overflow`; callers check before
// launching anything.
struct Workspace {
    char *base;
    size_t bytes;
    size_t used;
    bool overflow = false;
    template <class T> T *take(size_t count) {
        size_t off = (used + 255) & ~(size_t)255;
        if (off + count * sizeof(T) > bytes) {
            overflow = true;
            return nullptr;
        }
        used = off + count * sizeof(T);
        return reinterpret_cast<T *>(base + off);
    }
};

}  // namespace polypic

// The opaque context behind polypic_ctx.
namespace polypic {
struct PcgGraphs;
}

struct polypic_ctx {
    polypic_config cfg;
    polypic::GridGeom geom;
    int64_t num_keys;
    int device;
    uint32_t *d_status;   // device status word
    polypic::PcgGraphs *pcg_graphs = nullptr;   // the projection's captured batches
};

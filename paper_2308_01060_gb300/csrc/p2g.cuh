// p2g.cuh -- host-side entry points of the P2G transfer (p2g.cu).
#pragma once
#include "polypic_internal.cuh"

namespace polypic {

// Node region of one 4x4x2-cell block on face grid a: nodes
// [4bx - 1, 4bx - 1 + reg_x) x [4by - 1, ...) x [2bz - 1, 2bz - 1 + reg_z).
__host__ __device__ constexpr int reg_x(int a) { return a == 0 ? 7 : 6; }
__host__ __device__ constexpr int reg_y(int a) { return a == 1 ? 7 : 6; }
__host__ __device__ constexpr int reg_z(int a) { return a == 2 ? 5 : 4; }
__host__ __device__ constexpr int reg_size(int a) { return reg_x(a) * reg_y(a) * reg_z(a); }
// Scratch layout of one block: [a][mass | momentum][reg_size(a)].
__host__ __device__ constexpr int reg_off(int a, int which) {
    return (a >= 1 ? 2 * reg_size(0) : 0) + (a >= 2 ? 2 * reg_size(1) : 0) +
           which * reg_size(a);
}
constexpr int kRegionFloats = 2 * (reg_size(0) + reg_size(1) + reg_size(2));

// Node region of one 8x8x4-cell tile on face grid a (the union of its 8 block
// regions): nodes [8tx - 1, 8tx - 1 + tile_x) x [8ty - 1, ...) x [4tz - 1, ...).
__host__ __device__ constexpr int tile_x(int a) { return a == 0 ? 11 : 10; }
__host__ __device__ constexpr int tile_y(int a) { return a == 1 ? 11 : 10; }
__host__ __device__ constexpr int tile_z(int a) { return a == 2 ? 7 : 6; }
__host__ __device__ constexpr int tile_size(int a) { return tile_x(a) * tile_y(a) * tile_z(a); }
// Scratch layout of one tile: [a][mass | momentum][tile_size(a)].
__host__ __device__ constexpr int tile_off(int a, int which) {
    return (a >= 1 ? 2 * tile_size(0) : 0) + (a >= 2 ? 2 * tile_size(1) : 0) +
           which * tile_size(a);
}
constexpr int kTileFloats = 2 * (tile_size(0) + tile_size(1) + tile_size(2));

struct P2GArgs {
    GridGeom g;
    int64_t count;
    const float *x, *y, *z, *mass, *mass_abs;
    const void *coeff;
    const float *scale;        // 16-bit formats: per-particle s_p
    const uint32_t *perm, *cell_start;
    float *scratch;            // p2g_scratch_bytes(): one tile region per tile
    uint8_t *tile_live;        // one flag per tile, written by every CTA
    uint32_t *status;
    uint32_t nblocks;          // num_keys / 32
    float dxpow[7];            // dx^L, L = 0..6 (FP32 coefficients -> dimensionless)
    float s1, s2;              // stencil scales of F1 and phi: dx, dx^2 for FP32 P2G, else 1
    // Eq 12's affine map (4 modes, FP32): M = (I + map_dt C_p)^-1
    bool affine;
    float map_dt;
    // adjoint scatter only: mu [3][R][count] in slot order, 1/dx, 1/dx^2
    const float *mu;
    float inv_dx, inv_dx2;
};

size_t p2g_scratch_bytes(int64_t num_keys);

// Built-in fixed-size scratch for polypic_p2g_noalloc: device addresses of the
// tile regions and live flags in the current context (looked up again on
// every call outside a capture of `s`, cached per context for calls during
// one), and the number of tiles they hold.
cudaError_t p2g_builtin_scratch(cudaStream_t s, float **tiles, uint8_t **live);
int p2g_builtin_max_tiles();

// Writes all faces of gm[3] (mass) and gp[3] (momentum); with gv non-NULL
// also the single-phase grid update (v = mv/m + dt g, zero on wall faces).
// The phase is in block-interleaved slot order, read through perm.
// Reduces the tile regions already in P.scratch into gm, gp (added to them
// with `accumulate`).
cudaError_t p2g_reduce(const P2GArgs &P, float *gm[3], float *gp[3], bool accumulate,
                       cudaStream_t s);
// FP32 P2G whose result is added to gm, gp.
cudaError_t p2g_accumulate(const P2GArgs &P, float *gm[3], float *gp[3], int R, cudaStream_t s);
cudaError_t p2g(const P2GArgs &P, float *gm[3], float *gp[3], float *gv[3], float dt,
                const float gravity[3], int R, int fmt, cudaStream_t s);

// Adjoint of the G2P fit's grid dependence: lv_ia (+)= sum_p sum_r mu_pra
// G_r(x_ia - x_p), the same deterministic scatter with the fit factors
// G_r = w s_r / d_r and unit weight.  Reads positions through perm, mu in
// slot order.
cudaError_t p2g_adjoint_scatter(const P2GArgs &P, float *lv[3], bool accumulate, int R,
                                cudaStream_t s);

}  // namespace polypic

// g2p2g.cuh -- host side of the fused transfer (g2p2g.cu).
#pragma once
#include "p2g.cuh"

namespace polypic {

struct G2P2GArgs {
    P2GArgs p2g;                 // step n's sort, masses, P2G scratch and stencil scales
    const float *x, *y, *z;      // positions of step n (input order)
    const float *vel[3];         // v~ of step n
    float dt, inv1, inv2;        // advection step; 1/dx, 1/dx^2 (physical FP32 fit)
    float *ox, *oy, *oz, *omass, *omass_abs;   // state n + 1 in slot order
    float *ocoeff;               // [3][R][count]: written for movers only
    uint8_t *moved;              // [count] slot flags
};

struct SpillArgs {
    int64_t count, ntiles;
    int R;
    uint32_t capacity;
    const uint32_t *cell_start, *offsets;
    const uint8_t *moved;
    const float *ox, *oy, *oz, *omass, *omass_abs, *ocoeff;
    float *x, *y, *z, *mass, *mass_abs, *coeff;
};

cudaError_t g2p2g_tiles(const G2P2GArgs &Q, int R, cudaStream_t s);
cudaError_t count_and_scan_movers(const uint32_t *cell_start, const uint8_t *moved, int64_t ntiles,
                                  uint32_t *counts, uint32_t *offsets, cudaStream_t s);
cudaError_t compact_movers(const SpillArgs &S, cudaStream_t s);

}  // namespace polypic

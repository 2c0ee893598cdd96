// g2p.cuh -- host-side entry point of the G2P transfer (g2p.cu).
#pragma once
#include "polypic_internal.cuh"

namespace polypic {

struct G2PArgs {
    GridGeom g;
    int64_t count;
    float dt;
    const float *vel[3];
    const float *x, *y, *z, *mass, *mass_abs;
    const uint32_t *perm, *cell_start;
    float *ox, *oy, *oz, *omass, *omass_abs;
    void *ocoeff;
    float *oscale;
    uint32_t *status;
    float inv_dxpow[7];   // 1 / dx^L, L = 0..6
    bool grad_w;          // Eq 10's gradient form of the linear modes (4 modes)
};

cudaError_t g2p(const G2PArgs &A, int64_t num_tiles, int R, int fmt, cudaStream_t s);

}  // namespace polypic

// grid.cuh -- host-side entry points of the grid update (grid.cu) and the
// pressure projection (pcg.cu).
#pragma once
#include "polypic_internal.cuh"

namespace polypic {

struct GridUpdateArgs {
    GridGeom g;
    float dt;
    float gravity[3];
    float drag_k;
    const float *fm[3], *fp[3];
    float *fv[3];
    const float *sm[3], *sp[3];   // all NULL without a solid grid
    float *sv[3];
};

struct GridAdjointArgs {
    GridGeom g;
    float dt;
    float gravity[3];
    float drag_k;
    const float *fm[3], *fp[3], *lv[3];   // lv: dL/dv~ of the fluid (projected already)
    float *lm[3], *lp[3];
    const float *sm[3], *sp[3], *lsv[3];  // all NULL without a solid grid
    float *lsm[3], *lsp[3];
};

cudaError_t grid_update(const GridUpdateArgs &U, cudaStream_t s);
cudaError_t grid_update_adjoint(const GridAdjointArgs &U, cudaStream_t s);
// dst = src with the wall faces i_a in {0, n_a} zeroed (all three face grids)
cudaError_t wall_zeroed_copy(const GridGeom &g, const float *const src[3], float *const dst[3],
                             cudaStream_t s);

}  // namespace polypic

// adjoint.cuh -- adjoint transfers (adjoint.cu).
#pragma once
#include "polypic_internal.cuh"

namespace polypic {

struct AdjG2PArgs {
    GridGeom g;
    int64_t count;
    float dt, inv_dx;
    const float *vel[3];          // forward grid velocity v~
    const float *x[3];            // forward input positions (storage order)
    const float *bar_x[3];        // dL/dx' (slot order)
    const float *bar_c;           // dL/dc' [3][R][count] (slot order)
    const uint32_t *perm, *cell_start;
    float *mu;                    // out: effective coefficient adjoint (slot order)
    float *out_x[3];              // out: dL/dx (storage order)
    uint32_t *status;
    bool accumulate;
};

struct AdjP2GArgs {
    GridGeom g;
    int64_t count;
    float dx, inv_dx;
    const float *lm[3], *lmv[3];  // dL/dm, dL/d(mv) on the face grids
    const float *x[3];            // forward positions (storage order)
    const float *mass, *mass_abs;
    const float *coeff;           // forward coefficients [3][R][count]
    const uint32_t *perm, *cell_start;
    float *out_c;                 // out: dL/dc [3][R][count] (storage order)
    float *out_x[3];              // out: dL/dx (storage order)
    uint32_t *status;
    bool accumulate;
};

size_t adjoint_scratch_bytes(int64_t count, int R);

cudaError_t adjoint_g2p(const GridGeom &g, int64_t num_keys, int R, float dx,
                        const polypic_grid *grid, const polypic_particles *in, float dt,
                        const polypic_particles *bar_out, polypic_grid *bar_grid,
                        polypic_particles *bar_in, bool accumulate, uint32_t *status,
                        Workspace &ws, cudaStream_t s);

cudaError_t adjoint_p2g(const GridGeom &g, int64_t num_keys, int R, float dx,
                        const polypic_particles *in, const polypic_grid *bar_grid,
                        polypic_particles *bar_in, bool accumulate, uint32_t *status,
                        Workspace &ws, cudaStream_t s);

}  // namespace polypic

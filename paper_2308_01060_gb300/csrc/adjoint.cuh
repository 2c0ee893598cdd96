// adjoint.cuh -- adjoint transfers (adjoint.cu).
#pragma once
#include "polypic_internal.cuh"

namespace polypic {

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

// pcg.cuh -- pressure projection (pcg.cu).
#pragma once
#include "polypic_internal.cuh"

namespace polypic {

size_t pcg_scratch_bytes(const GridGeom &g);

// The captured CUDA graphs of a context's CG iteration batches (pcg.cu).
struct PcgGraphs;
void pcg_graphs_free(PcgGraphs *g);

// Projects vel[3] in place onto the discretely divergence-free fields on the
// cells that hold fluid particles (cell_start of the fluid phase).  With
// `graphs`, full batches of CG iterations replay CUDA graphs captured once
// per workspace layout and kept there (freed by pcg_graphs_free).
polypic_status pcg_project(const GridGeom &g, int64_t num_keys, const uint32_t *cell_start,
                           float *vel[3], float dt, float rho, int maxiter, double rtol,
                           uint32_t *status, Workspace &ws, cudaStream_t s,
                           PcgGraphs **graphs = nullptr);

}  // namespace polypic

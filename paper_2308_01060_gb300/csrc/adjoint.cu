// adjoint.cu -- adjoint transfers (placeholder until the kernels land).
#include "adjoint.cuh"

namespace polypic {

cudaError_t adjoint_g2p(const GridGeom &, int64_t, int, float, const polypic_grid *,
                        const polypic_particles *, float, const polypic_particles *,
                        polypic_grid *, polypic_particles *, bool, uint32_t *, Workspace &,
                        cudaStream_t) {
    return cudaErrorNotSupported;
}

cudaError_t adjoint_p2g(const GridGeom &, int64_t, int, float, const polypic_particles *,
                        const polypic_grid *, polypic_particles *, bool, uint32_t *,
                        Workspace &, cudaStream_t) {
    return cudaErrorNotSupported;
}

}  // namespace polypic

// pcg.cu -- pressure projection (placeholder until the PCG kernels land).
#include "pcg.cuh"

namespace polypic {

size_t pcg_scratch_bytes(const GridGeom &g) { (void)g; return 0; }

polypic_status pcg_project(const GridGeom &, int64_t, const uint32_t *, float *[3], float, float,
                           int, double, uint32_t *, Workspace &, cudaStream_t) {
    return POLYPIC_ERR_UNSUPPORTED;
}

}  // namespace polypic

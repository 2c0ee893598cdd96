// p2g_tiles_aff.cu -- the P2G tile kernels with Eq 12's affine map (FP32 coefficients).
#include "p2g_tiles.cuh"

namespace polypic {

cudaError_t launch_tiles_aff27(const P2GArgs &P, int grid, cudaStream_t s);

cudaError_t launch_tiles_aff(const P2GArgs &P, int R, int grid, cudaStream_t s) {
    if (R == 4) return launch_tiles<4, POLYPIC_COEFF_F32, false, true>(P, grid, s);
    if (R == 8) return launch_tiles<8, POLYPIC_COEFF_F32, false, true>(P, grid, s);
    if (R == 27) return launch_tiles_aff27(P, grid, s);
    return cudaErrorInvalidValue;
}

}  // namespace polypic

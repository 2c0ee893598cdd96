// p2g_tiles_teams.cu -- the FP32 P2G tile kernels with the lane-team schedule,
// used for the solid phase (a sheet fills few of a block's cells).
#include "p2g_tiles.cuh"

namespace polypic {

cudaError_t launch_tiles_teams(const P2GArgs &P, int R, int grid, cudaStream_t s) {
    if (R == 1) return launch_tiles<1, POLYPIC_COEFF_F32, false>(P, grid, s);
    if (R == 4) return launch_tiles<4, POLYPIC_COEFF_F32, false, false, true>(P, grid, s);
    if (R == 8) return launch_tiles<8, POLYPIC_COEFF_F32, false, false, true>(P, grid, s);
    if (R == 27) return launch_tiles<27, POLYPIC_COEFF_F32, false, false, true>(P, grid, s);
    return cudaErrorInvalidValue;
}

}  // namespace polypic

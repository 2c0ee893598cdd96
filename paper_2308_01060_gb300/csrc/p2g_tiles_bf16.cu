// p2g_tiles_bf16.cu -- the P2G tile kernels for BF16 coefficient codes.
#include "p2g_tiles.cuh"

namespace polypic {

cudaError_t launch_tiles_bf16(const P2GArgs &P, int R, int grid, cudaStream_t s) {
    if (R == 1) return launch_tiles<1, POLYPIC_COEFF_BF16, false>(P, grid, s);
    if (R == 4) return launch_tiles<4, POLYPIC_COEFF_BF16, false>(P, grid, s);
    if (R == 8) return launch_tiles<8, POLYPIC_COEFF_BF16, false>(P, grid, s);
    if (R == 27) return launch_tiles<27, POLYPIC_COEFF_BF16, false>(P, grid, s);
    return cudaErrorInvalidValue;
}

}  // namespace polypic

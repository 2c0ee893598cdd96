// p2g_tiles_f16.cu -- the P2G tile kernels for FP16 coefficient codes, and the 16-bit dispatch.
#include "p2g_tiles.cuh"

namespace polypic {

cudaError_t launch_tiles_bf16(const P2GArgs &P, int R, int grid, cudaStream_t s);

cudaError_t launch_tiles_16(const P2GArgs &P, int R, int fmt, int grid, cudaStream_t s) {
    if (fmt == POLYPIC_COEFF_BF16) return launch_tiles_bf16(P, R, grid, s);
    if (fmt != POLYPIC_COEFF_F16) return cudaErrorInvalidValue;
    if (R == 1) return launch_tiles<1, POLYPIC_COEFF_F16, false>(P, grid, s);
    if (R == 4) return launch_tiles<4, POLYPIC_COEFF_F16, false>(P, grid, s);
    if (R == 8) return launch_tiles<8, POLYPIC_COEFF_F16, false>(P, grid, s);
    if (R == 27) return launch_tiles<27, POLYPIC_COEFF_F16, false>(P, grid, s);
    return cudaErrorInvalidValue;
}

}  // namespace polypic

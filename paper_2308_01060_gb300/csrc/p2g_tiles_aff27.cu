// p2g_tiles_aff27.cu -- the 27-mode P2G tile kernel with Eq 12's affine map
// (per-node evaluation of the mapped modes; its own translation unit, the
// largest of the library).
#include "p2g_tiles.cuh"

namespace polypic {

cudaError_t launch_tiles_aff27(const P2GArgs &P, int grid, cudaStream_t s) {
    return launch_tiles<27, POLYPIC_COEFF_F32, false, true>(P, grid, s);
}

}  // namespace polypic

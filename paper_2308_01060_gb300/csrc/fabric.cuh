// fabric.cuh -- host side of the fabric and absorption stand-ins (fabric.cu).
#pragma once
#include "polypic_internal.cuh"

namespace polypic {

struct FabricForceArgs {
    int64_t count;
    const float *x[3];
    const float *mass, *mass_abs;
    float *vel[3];          // mode 0 of each component's coefficients (FP32), updated in place
    const uint32_t *id;     // lattice id per slot
    int m;
    float h, k_stretch, k_shear, k_bend, damping, dt;
};

struct AbsorbCall {
    int64_t num_keys;
    const uint32_t *fluid_cell_start, *fluid_perm;
    const uint32_t *solid_cell_start, *solid_perm;
    float *fluid_mass;
    const float *solid_mass;
    float *mass_abs;
    float rate, dt, capacity, max_fraction;
};

size_t fabric_scratch_bytes(int64_t count, int m);
cudaError_t fabric_forces(const FabricForceArgs &a, Workspace &ws, cudaStream_t s);
cudaError_t absorb(const AbsorbCall &a, cudaStream_t s);
cudaError_t gather_ids(const uint32_t *in, const uint32_t *perm, int64_t count, uint32_t *out,
                       cudaStream_t s);

}  // namespace polypic

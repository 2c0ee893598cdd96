// ordered.cuh -- host-side entry points of the kernels for ordered phases
// (ordered.cu): particle arrays kept in their own slot order, so that P2G
// reads them contiguously.
#pragma once
#include "polypic_internal.cuh"
#include "sort.cuh"

namespace polypic {

// Advection of an ordered phase with the grid velocity (the PIC part of the
// G2P fit, v_p = c_p0) and the key of every new position, counted into
// `counts` with an arrival rank (the key producer of the next order).
struct AdvectArgs {
    GridGeom g;
    int64_t count;
    float dt;
    const float *vel[3];
    const float *x, *y, *z;        // the ordered phase
    const uint32_t *cell_start;    // its cell starts
    uint32_t *key, *rank;          // key of each advected position and its arrival rank
    uint32_t *counts;              // per-key counts (zeroed by the caller)
    uint32_t *num_crowded;         // zeroed here for the sort that follows
    uint32_t *num_far;             // zeroed here for the G2P that follows
    uint32_t *status;
};
cudaError_t advect(const AdvectArgs &A, int64_t num_tiles, cudaStream_t s);

// G2P of an ordered phase into the next order: slot j of the output holds
// input particle perm[j], fitted at its old position, advected again with
// the velocity mode of that fit (the very value k_advect computed, from the
// same arithmetic on the same nodes) and given the key k_advect sorted it by.
struct OrderedG2PArgs {
    GridGeom g;
    int64_t count;
    float dt;
    const float *vel[3];
    const float *x, *y, *z, *mass, *mass_abs;   // the input phase (old order)
    const uint32_t *key_new;                    // keys of the advected positions (old order)
    const uint32_t *perm, *cell_start;          // the next order
    float *ox, *oy, *oz, *omass, *omass_abs;
    void *ocoeff;
    float *oscale;
    uint32_t *okey;
    uint32_t *far, *num_far;  // slots whose old cell is outside the staged halo
    uint32_t *status;
    float inv_dxpow[7];  // 1 / dx^L, L = 0..6
};
cudaError_t g2p_ordered(const OrderedG2PArgs &A, int64_t num_tiles, int R, int fmt,
                        cudaStream_t s);

// out slot j <- in particle perm[j] for every array of a phase (coefficient
// elements of `elem` bytes, rows of `count`).
struct GatherArgs {
    int64_t count;
    int rows;   // coefficient rows, 3 N_r
    int elem;   // bytes per coefficient: 4 or 2
    const uint32_t *perm;
    const float *x[3], *mass, *mass_abs, *scale;
    const void *coeff;
    const uint32_t *key;
    float *ox[3], *omass, *omass_abs, *oscale;
    void *ocoeff;
    uint32_t *okey;
};
cudaError_t gather_phase(const GatherArgs &A, cudaStream_t s);

}  // namespace polypic

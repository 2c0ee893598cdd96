// sort.cuh -- host-side entry points of the cell sort (sort.cu).
#pragma once
#include "polypic_internal.cuh"

namespace polypic {

constexpr int kScanThreads = 256;
constexpr int kScanTile = 4096;
// Cells holding at most this many particles are ordered by per-lane
// selection (quadratic in the population); larger ones by a CTA radix sort.
constexpr int kSelectMax = 64;

size_t scan_scratch_words(int64_t L);

// Exclusive prefix sum of L uint32 (in may equal out); scratch holds
// scan_scratch_words(L) words.
cudaError_t exclusive_scan(const uint32_t *in, uint32_t *out, int64_t L, uint32_t *scratch,
                           cudaStream_t s);

size_t sort_scratch_bytes(int64_t count, int64_t num_keys);

cudaError_t sort_particles(const GridGeom &g, int64_t num_keys, int64_t count, const float *x,
                           const float *y, const float *z, uint32_t *key, uint32_t *perm,
                           uint32_t *cell_start, uint32_t *status, Workspace &ws,
                           cudaStream_t s);

}  // namespace polypic

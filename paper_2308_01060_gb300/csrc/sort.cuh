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

// Scratch of one sort, carved from the caller's workspace.
struct SortScratch {
    uint32_t *key;          // key of each input particle (when the caller has no array)
    uint32_t *rank;         // arrival rank of each input particle in its cell
    uint32_t *arrival;      // particles in cell order, arrival order inside a cell
    uint32_t *radix;        // second buffer of the crowded-cell radix sort
    uint32_t *crowded;      // cells holding more than kSelectMax particles ...
    uint32_t *num_crowded;  // ... and their number (zeroed by the key producer)
    uint32_t *cscan;        // scratch of the count scan
};
size_t sort_scratch_bytes(int64_t count, int64_t num_keys);
bool take_sort_scratch(Workspace &ws, int64_t count, int64_t num_keys, SortScratch &S);

// From the per-key counts in cell_start (written by a key producer together
// with key and S.rank): cell_start becomes the exclusive prefix, perm the
// block-interleaved slot order (perm[j] = input index of the particle in slot j).
cudaError_t finish_order(int64_t num_keys, int64_t count, const uint32_t *key,
                         uint32_t *cell_start, uint32_t *perm, const SortScratch &S,
                         cudaStream_t s);

// The whole sort of particles by the cell of their positions.
cudaError_t sort_particles(const GridGeom &g, int64_t num_keys, int64_t count, const float *x,
                           const float *y, const float *z, uint32_t *key, uint32_t *perm,
                           uint32_t *cell_start, uint32_t *status, Workspace &ws,
                           cudaStream_t s);

}  // namespace polypic

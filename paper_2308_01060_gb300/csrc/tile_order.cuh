// tile_order.cuh -- the grouped slot order of ordered particle phases: how the
// 256 cells of a key tile are dealt to the lanes of the transfer kernels.
//
// A transfer lane owns one cell and visits its particles in rounds (round r:
// every lane's r-th particle), so a warp costs as many rounds as its fullest
// cell.  To keep a warp's lanes equally busy, the cells of a tile are ranked
// by particle count -- bucket q = min(n, 31) descending, ties by cell index
// ascending -- and rank 32 g + l becomes lane l of group g (g = 0..7).  The
// particles of a tile are stored group by group (g ascending), each group
// round by round (round r lists the r-th particle, in stable order, of every
// lane whose cell holds more than r), each round by lane.  The ranking is a
// function of the cell counts alone, so the sort that writes this order and
// the transfers that read it derive it independently from cell_start.
#pragma once
#include "polypic_internal.cuh"

namespace polypic {

constexpr int kTileCells = 256;
constexpr int kGroups = 8;
constexpr int kBuckets = 32;

struct TileOrder {
    uint32_t n[kTileCells];          // particle count of the cell at each rank
    uint16_t cell[kTileCells];       // tile-local index (key - 256 tile) at each rank
    uint32_t gstart[kGroups + 1];    // first slot of each group; gstart[8] = end of the tile
    uint32_t wc[kGroups][kBuckets];  // per 32-cell chunk: bucket counts, then their prefixes
    uint32_t above[kBuckets];        // cells of the tile in higher buckets
};

// Ranks the cells of `tile` into `o` (shared memory).  Every thread of the
// CTA (kThreads of them) must call it; it ends with a barrier.
template <int kThreads>
__device__ __forceinline__ void rank_tile(const uint32_t *__restrict__ cs, uint32_t tile,
                                          TileOrder &o) {
    static_assert(kTileCells % kThreads == 0 && kThreads % 32 == 0, "whole warps, whole tile");
    constexpr int kPer = kTileCells / kThreads;
    const int tid = threadIdx.x, lane = tid & 31;
    const unsigned lt = (1u << lane) - 1u;
    const uint32_t t0 = tile * kTileCells;
    for (int i = tid; i < kGroups * kBuckets; i += kThreads) (&o.wc[0][0])[i] = 0;
    __syncthreads();
    uint32_t n[kPer], q[kPer], wr[kPer];
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        const int c = tid + k * kThreads;  // its 32-cell chunk c >> 5 is warp-uniform
        n[k] = cs[t0 + c + 1] - cs[t0 + c];
        q[k] = min(n[k], (uint32_t)(kBuckets - 1));
        const unsigned peers = __match_any_sync(0xffffffffu, q[k]);
        wr[k] = (uint32_t)__popc(peers & lt);
        if (lane == __ffs(peers) - 1) o.wc[c >> 5][q[k]] = (uint32_t)__popc(peers);
    }
    __syncthreads();
    if (tid < kBuckets) {  // warp 0, lane = bucket
        uint32_t run = 0;
#pragma unroll
        for (int ch = 0; ch < kGroups; ++ch) {
            const uint32_t v = o.wc[ch][tid];
            o.wc[ch][tid] = run;
            run += v;
        }
        uint32_t s = run;  // cells in buckets >= this one
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t t = __shfl_down_sync(0xffffffffu, s, off);
            if (tid + off < 32) s += t;
        }
        o.above[tid] = s - run;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        const int c = tid + k * kThreads;
        const uint32_t rank = o.above[q[k]] + o.wc[c >> 5][q[k]] + wr[k];
        o.n[rank] = n[k];
        o.cell[rank] = (uint16_t)c;
    }
    __syncthreads();
    if (tid < 32) {
        uint32_t run = cs[t0];
#pragma unroll
        for (int g = 0; g < kGroups; ++g) {
            const uint32_t tot = __reduce_add_sync(0xffffffffu, o.n[32 * g + tid]);
            if (tid == 0) o.gstart[g] = run;
            run += tot;
        }
        if (tid == 0) o.gstart[kGroups] = run;
    }
    __syncthreads();
}

// Tile-local cell coordinates of tile-local key c (inverse of cell_key).
__device__ __forceinline__ void local_cell(uint32_t c, int &i, int &j, int &k) {
    i = (int)((c & 3u) | (((c >> 5) & 1u) << 2));
    j = (int)(((c >> 2) & 3u) | (((c >> 6) & 1u) << 2));
    k = (int)(((c >> 4) & 1u) | (((c >> 7) & 1u) << 1));
}

}  // namespace polypic

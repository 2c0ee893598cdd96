// sort.cu -- bit-exact stable sort of particles by cell key.
//
// The paper has no sort; it is the device that makes the transfers
// deterministic and coalesced.  No kernel waits on another CTA:
//   1. k_keys:     key of every particle (FP32 cell decision), domain check,
//                  per-key counts with integer atomics, one per run of equal
//                  keys along a lane (exact: integer addition is order
//                  independent), whose return values give each particle an
//                  arrival rank inside its cell;
//   2. scan:       exclusive prefix sum of the counts -> cell_start;
//   3. k_scatter:  particle p to cell_start[key] + arrival rank, so every
//                  cell's particles fill its range in a timing-dependent order;
//   4. k_cell_order / k_crowded_cells: the stable order inside each cell is
//                  ascending particle index (unique, so it is compared
//                  bit-exactly with a CPU stable sort); it is recovered from
//                  the arrival order by selection (small cells) or a CTA radix
//                  sort (crowded cells) and written straight into the slot
//                  order of the transfers: inside every block of 32 keys the
//                  stable order is dealt round-robin over the keys (round r =
//                  each key's r-th particle), so that a warp whose lanes own
//                  the 32 cells reads one contiguous run of slots per round.
#include "sort.cuh"

namespace polypic {

// ---------------------------------------------------------------- keys
// A warp takes kKeyRuns x 32 consecutive particles, lane l the particles
// l, l + 32, l + 64, ... of its chunk.  In the slot order the previous step's
// G2P wrote, a full round of a block is 32 consecutive slots of 32 different
// cells, so a lane's successive particles tend to share a cell: each run of
// equal keys along a lane takes one atomicAdd of its length (integer, exact)
// and ranks its particles from the returned count.
constexpr int kKeyRuns = 8;

__global__ void __launch_bounds__(256) k_keys(int64_t n, const float *__restrict__ x,
                                              const float *__restrict__ y,
                                              const float *__restrict__ z, GridGeom g,
                                              uint32_t *__restrict__ key,
                                              uint32_t *__restrict__ rank,
                                              uint32_t *__restrict__ counts,
                                              uint32_t *__restrict__ num_crowded,
                                              uint32_t *__restrict__ status) {
    const int lane = threadIdx.x & 31;
    const int64_t base = ((int64_t)blockIdx.x * 8 + (threadIdx.x >> 5)) * (32 * kKeyRuns) + lane;
    if (blockIdx.x == 0 && threadIdx.x == 0) *num_crowded = 0;
    uint32_t k[kKeyRuns];
    bool bad = false;
#pragma unroll
    for (int m = 0; m < kKeyRuns; ++m) {
        const int64_t p = base + 32 * m;
        k[m] = 0;
        if (p < n) {
            const float vx = cell_coord(x[p], g.inv_dx);
            const float vy = cell_coord(y[p], g.inv_dx);
            const float vz = cell_coord(z[p], g.inv_dx);
            bad |= !(coord_valid(vx, g.n[0]) && coord_valid(vy, g.n[1]) && coord_valid(vz, g.n[2]));
            k[m] = cell_key(g, cell_index(vx, g.n[0]), cell_index(vy, g.n[1]),
                            cell_index(vz, g.n[2]));
            key[p] = k[m];
        }
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(status, kFlagOutOfDomain);
    // runs of equal keys along the lane (the live particles are a prefix)
    bool start[kKeyRuns];
    uint32_t len[kKeyRuns], old[kKeyRuns];
#pragma unroll
    for (int m = 0; m < kKeyRuns; ++m)
        start[m] = base + 32 * m < n && (m == 0 || k[m] != k[m - 1]);
    len[kKeyRuns - 1] = base + 32 * (kKeyRuns - 1) < n ? 1u : 0u;
#pragma unroll
    for (int m = kKeyRuns - 2; m >= 0; --m) {
        const bool cont = base + 32 * (m + 1) < n && !start[m + 1];  // run goes on at m + 1
        len[m] = base + 32 * m < n ? (cont ? len[m + 1] + 1u : 1u) : 0u;
    }
#pragma unroll
    for (int m = 0; m < kKeyRuns; ++m) old[m] = start[m] ? atomicAdd(&counts[k[m]], len[m]) : 0u;
    uint32_t r = 0;
#pragma unroll
    for (int m = 0; m < kKeyRuns; ++m) {
        const int64_t p = base + 32 * m;
        if (p < n) {
            r = start[m] ? old[m] : r + 1u;
            rank[p] = r;
        }
    }
}

// ---------------------------------------------------------------- scan
// Block-level exclusive scan of 256 per-thread totals; returns the thread's
// exclusive prefix and writes the block total to *total.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *s_warp,
                                                         uint32_t *total) {
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_warp[w] = incl;
    __syncthreads();
    if (w == 0) {
        int nw = blockDim.x >> 5;
        uint32_t s = lane < nw ? s_warp[lane] : 0u;
        uint32_t si = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t t = __shfl_up_sync(0xffffffffu, si, o);
            if (lane >= o) si += t;
        }
        if (lane < nw) s_warp[lane] = si - s;
        if (lane == nw - 1) s_warp[32] = si;
    }
    __syncthreads();
    uint32_t r = s_warp[w] + incl - v;
    *total = s_warp[32];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t *__restrict__ in,
                                                              int64_t L,
                                                              uint32_t *__restrict__ sums) {
    __shared__ uint32_t s_warp[33];
    int64_t base = (int64_t)blockIdx.x * kScanTile;
    uint32_t acc = 0;
    for (int i = threadIdx.x; i < kScanTile; i += kScanThreads) {
        int64_t idx = base + i;
        if (idx < L) acc += in[idx];
    }
    uint32_t total;
    block_exclusive_scan(acc, s_warp, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// Single-CTA exclusive scan of nb block sums (nb <= kScanThreads * 256).
__global__ void __launch_bounds__(kScanThreads) k_scan_top(uint32_t *__restrict__ sums, int nb) {
    __shared__ uint32_t s_warp[33];
    int per = (nb + kScanThreads - 1) / kScanThreads;
    int beg = threadIdx.x * per;
    uint32_t acc = 0;
    for (int i = 0; i < per; ++i)
        if (beg + i < nb) acc += sums[beg + i];
    uint32_t total;
    uint32_t run = block_exclusive_scan(acc, s_warp, &total);
    for (int i = 0; i < per; ++i)
        if (beg + i < nb) {
            uint32_t v = sums[beg + i];
            sums[beg + i] = run;
            run += v;
        }
}

// Exclusive scan of one kScanTile chunk plus its block offset, in place
// (in may equal out).
__global__ void __launch_bounds__(kScanThreads) k_scan_down(const uint32_t *in, uint32_t *out,
                                                            int64_t L,
                                                            const uint32_t *__restrict__ sums) {
    __shared__ uint32_t s_data[kScanTile];
    __shared__ uint32_t s_warp[33];
    int64_t base = (int64_t)blockIdx.x * kScanTile;
    for (int i = threadIdx.x; i < kScanTile; i += kScanThreads) {
        int64_t idx = base + i;
        s_data[i] = idx < L ? in[idx] : 0u;
    }
    __syncthreads();
    constexpr int kPer = kScanTile / kScanThreads;
    uint32_t loc[kPer];
    uint32_t acc = 0;
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
        loc[i] = s_data[threadIdx.x * kPer + i];
        acc += loc[i];
    }
    uint32_t total;
    uint32_t run = block_exclusive_scan(acc, s_warp, &total) + sums[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
        s_data[threadIdx.x * kPer + i] = run;
        run += loc[i];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kScanTile; i += kScanThreads) {
        int64_t idx = base + i;
        if (idx < L) out[idx] = s_data[i];
    }
}

size_t scan_scratch_words(int64_t L) { return (size_t)((L + kScanTile - 1) / kScanTile) + 1; }

cudaError_t exclusive_scan(const uint32_t *in, uint32_t *out, int64_t L, uint32_t *scratch,
                           cudaStream_t s) {
    if (L <= 0) return cudaSuccess;
    int nb = (int)((L + kScanTile - 1) / kScanTile);
    if (nb > kScanThreads * 256) return cudaErrorInvalidValue;
    k_scan_reduce<<<nb, kScanThreads, 0, s>>>(in, L, scratch);
    k_scan_top<<<1, kScanThreads, 0, s>>>(scratch, nb);
    k_scan_down<<<nb, kScanThreads, 0, s>>>(in, out, L, scratch);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- scatter
// Every particle to cell_start[key] + its arrival rank: each cell's particles
// land in its range, in an order that depends on the atomics' timing.
__global__ void __launch_bounds__(256) k_scatter(int64_t n, const uint32_t *__restrict__ key,
                                                 const uint32_t *__restrict__ rank,
                                                 const uint32_t *__restrict__ cs,
                                                 uint32_t *__restrict__ out) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) out[cs[key[p]] + rank[p]] = (uint32_t)p;
}

// ---------------------------------------------------------------- cell order
// The block-interleaved layout deals the 32 cells of a block round-robin:
// round r lists the r-th particle (ascending input index, i.e. the stable
// order) of every cell holding more than r, cells ascending, from the block's
// first slot on.  One warp per block.  The particle in round r of cell c sits
// at slot S(r) + |{c' < c : n_c' > r}|, S(r) = sum over the block's cells of
// min(n, r); a warp tabulates S and the live masks once.  Each particle's
// round is its rank in its cell: the number of smaller indices in the cell's
// arrival-ordered range (indices are distinct).  The warp's lanes share the
// block's particles (lane l takes l, l + 32, ...), so a warp costs the sum of
// n^2 over its cells / 32 loads, not the fullest cell's n^2.  Cells holding
// more than kSelectMax particles are listed for k_crowded_cells instead and
// their slots are left to it.
__global__ void __launch_bounds__(256) k_cell_order(const uint32_t *__restrict__ in,
                                                    const uint32_t *__restrict__ cs,
                                                    uint32_t *__restrict__ out, uint32_t nblocks,
                                                    uint32_t *__restrict__ crowded,
                                                    uint32_t *__restrict__ num_crowded) {
    __shared__ uint32_t s_tab[8][2][kSelectMax];
    __shared__ uint32_t s_start[8][33];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t b = blockIdx.x * 8 + w;
    if (b >= nblocks) return;  // warp-uniform
    const uint32_t k = b * 32 + lane;
    const uint32_t s0 = cs[k], n = cs[k + 1] - s0;
    const uint32_t base = cs[b * 32], end = cs[b * 32 + 32];
    const bool select = n <= (uint32_t)kSelectMax;
    if (!select) crowded[atomicAdd(num_crowded, 1u)] = k;
    const uint32_t maxn = __reduce_max_sync(0xffffffffu, select ? n : 0u);
    uint32_t *tabS = s_tab[w][0], *tabM = s_tab[w][1];
    for (uint32_t r = 0; r < maxn; ++r) {
        const uint32_t sr = __reduce_add_sync(0xffffffffu, min(n, r));
        const uint32_t mr = __ballot_sync(0xffffffffu, n > r);
        if (lane == 0) {
            tabS[r] = sr;
            tabM[r] = mr;
        }
    }
    s_start[w][lane] = s0;
    if (lane == 0) s_start[w][32] = end;
    __syncwarp();
    for (uint32_t i = base + lane; i < end; i += 32) {
        // the cell of arrival slot i: the last lane whose start is <= i
        int c = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1)
            if (s_start[w][c + step] <= i) c += step;
        const uint32_t cs0 = s_start[w][c], cn = s_start[w][c + 1] - cs0;
        if (cn > (uint32_t)kSelectMax) continue;  // a crowded cell
        const uint32_t e = __ldg(in + i);
        uint32_t rank = 0;
        for (uint32_t j = 0; j < cn; ++j) rank += __ldg(in + cs0 + j) < e ? 1u : 0u;
        out[base + tabS[rank] + __popc(tabM[rank] & ((1u << c) - 1u))] = e;
    }
}

// Cells holding more than kSelectMax particles, one CTA per cell: a stable
// LSD radix sort of the cell's indices (8-bit digits, ranked in chunks of 256
// in order) between its range of `a` and of `b`, then the dealt slots.
// Linear in the cell's population, so a crowded cell costs what its particles
// cost.  Launched with a fixed grid; CTAs beyond the list exit at once.
__global__ void __launch_bounds__(256) k_crowded_cells(const uint32_t *__restrict__ crowded,
                                                       const uint32_t *__restrict__ num_crowded,
                                                       uint32_t *a, uint32_t *b,
                                                       const uint32_t *__restrict__ cs,
                                                       uint32_t *__restrict__ out, int value_bits) {
    __shared__ uint32_t s_base[256];
    __shared__ uint32_t s_wc[8][256];
    __shared__ uint32_t s_warp[33];
    __shared__ uint32_t s_n[32];
    __shared__ uint32_t s_lane, s_setbase;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const uint32_t total_cells = *num_crowded;
    for (uint32_t ci = blockIdx.x; ci < total_cells; ci += gridDim.x) {
        const uint32_t k = crowded[ci];
        const uint32_t s0 = cs[k], n = cs[k + 1] - s0;
        uint32_t *src = a + s0, *dst = b + s0;
        for (int shift = 0; shift < value_bits; shift += 8) {
            // digit histogram -> exclusive digit starts
            s_base[tid] = 0;
#pragma unroll
            for (int ww = 0; ww < 8; ++ww) s_wc[ww][tid] = 0;
            __syncthreads();
            for (uint32_t i = tid; i < n; i += 256) atomicAdd(&s_base[(src[i] >> shift) & 255u], 1u);
            __syncthreads();
            uint32_t total;
            const uint32_t start = block_exclusive_scan(s_base[tid], s_warp, &total);
            s_base[tid] = start;
            __syncthreads();
            // stable scatter, 256 indices per chunk in order
            for (uint32_t c0 = 0; c0 < n; c0 += 256) {
                const uint32_t i = c0 + tid;
                const bool valid = i < n;
                const uint32_t v = valid ? src[i] : 0u;
                const uint32_t d = valid ? (v >> shift) & 255u : 256u;
                const unsigned peers = __match_any_sync(0xffffffffu, d);
                if (valid && lane == __ffs(peers) - 1) s_wc[w][d] = (uint32_t)__popc(peers);
                __syncthreads();
                uint32_t run = 0;
#pragma unroll
                for (int ww = 0; ww < 8; ++ww) {
                    const uint32_t c = s_wc[ww][tid];
                    s_wc[ww][tid] = run;
                    run += c;
                }
                __syncthreads();
                if (valid) dst[s_base[d] + s_wc[w][d] + (uint32_t)__popc(peers & lt)] = v;
                __syncthreads();
                s_base[tid] += run;
#pragma unroll
                for (int ww = 0; ww < 8; ++ww) s_wc[ww][tid] = 0;
                __syncthreads();
            }
            uint32_t *t = src;
            src = dst;
            dst = t;
        }
        // the cell's lane set: its 32 counts, its lane and the set's first slot
        {
            const uint32_t blk = k >> 5;
            if (tid < 32) s_n[tid] = cs[blk * 32 + tid + 1] - cs[blk * 32 + tid];
            if (tid == 0) {
                s_lane = k & 31u;
                s_setbase = cs[blk * 32];
            }
        }
        __syncthreads();
        const uint32_t l = s_lane, base = s_setbase;
        for (uint32_t q = tid; q < n; q += 256) {
            uint32_t before = 0, pos = 0;
#pragma unroll 8
            for (uint32_t ll = 0; ll < 32; ++ll) {
                const uint32_t nl = s_n[ll];
                before += min(nl, q);
                pos += (ll < l && nl > q) ? 1u : 0u;
            }
            out[base + before + pos] = src[q];
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- driver
static int value_bits(int64_t count) {
    int b = 8;
    while (b < 32 && ((int64_t)1 << b) < count) b += 8;
    return b;
}

static int64_t crowded_capacity(int64_t count) { return count / (kSelectMax + 1) + 1; }

size_t sort_scratch_bytes(int64_t count, int64_t num_keys) {
    size_t words = 0;
    words += 4 * (size_t)count + 4 * 64;                       // key, rank, arrival, radix
    words += (size_t)crowded_capacity(count) + 1 + 2 * 64;     // crowded-cell list and its length
    words += scan_scratch_words(num_keys + 1) + 64;            // cell-count scan
    return words * sizeof(uint32_t) + 8 * 256;
}

bool take_sort_scratch(Workspace &ws, int64_t count, int64_t num_keys, SortScratch &S) {
    S.key = ws.take<uint32_t>(count);
    S.rank = ws.take<uint32_t>(count);
    S.arrival = ws.take<uint32_t>(count);
    S.radix = ws.take<uint32_t>(count);
    S.crowded = ws.take<uint32_t>(crowded_capacity(count));
    S.num_crowded = ws.take<uint32_t>(1);
    S.cscan = ws.take<uint32_t>(scan_scratch_words(num_keys + 1));
    return !ws.overflow;
}

cudaError_t finish_order(int64_t num_keys, int64_t count, const uint32_t *key,
                         uint32_t *cell_start, uint32_t *perm, const SortScratch &S,
                         cudaStream_t s) {
    cudaError_t e = exclusive_scan(cell_start, cell_start, num_keys + 1, S.cscan, s);
    if (e != cudaSuccess) return e;
    const int pblocks = (int)((count + 255) / 256);
    k_scatter<<<pblocks, 256, 0, s>>>(count, key, S.rank, cell_start, S.arrival);
    const int64_t cap = crowded_capacity(count);
    const int cgrid = (int)(cap < 304 ? cap : 304);
    const uint32_t nblocks = (uint32_t)(num_keys / 32);
    k_cell_order<<<(nblocks + 7) / 8, 256, 0, s>>>(S.arrival, cell_start, perm, nblocks,
                                                   S.crowded, S.num_crowded);
    k_crowded_cells<<<cgrid, 256, 0, s>>>(S.crowded, S.num_crowded, S.arrival, S.radix,
                                          cell_start, perm, value_bits(count));
    return cudaGetLastError();
}

cudaError_t sort_particles(const GridGeom &g, int64_t num_keys, int64_t count, const float *x,
                           const float *y, const float *z, uint32_t *key, uint32_t *perm,
                           uint32_t *cell_start, uint32_t *status, Workspace &ws,
                           cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(cell_start, 0, sizeof(uint32_t) * (num_keys + 1), s);
    if (e != cudaSuccess) return e;
    if (count == 0) return cudaSuccess;
    SortScratch S;
    if (!take_sort_scratch(ws, count, num_keys, S)) return cudaErrorInvalidValue;
    if (!key) key = S.key;
    k_keys<<<(int)((count + 256 * kKeyRuns - 1) / (256 * kKeyRuns)), 256, 0, s>>>(
        count, x, y, z, g, key, S.rank, cell_start, S.num_crowded, status);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return finish_order(num_keys, count, key, cell_start, perm, S, s);
}

}  // namespace polypic

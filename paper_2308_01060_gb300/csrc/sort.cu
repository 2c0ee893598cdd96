// sort.cu -- bit-exact stable sort of particles by cell key.
//
// The paper has no sort; it is the device that makes the transfers
// deterministic and coalesced.  Four pieces, none of which waits on another
// CTA (reduce-then-scan only):
//   1. k_keys:   key of every particle (FP32 cell decision), domain check,
//                per-key counts with warp-aggregated integer atomics
//                (integer addition is order independent, so counts are exact);
//   2. scan:     exclusive prefix sum of the counts -> cell_start;
//   3. radix:    LSD radix sort of (key, index) pairs, 8 bits or fewer per
//                pass; each pass = per-tile digit histograms, a device-wide
//                scan of the digit-major histogram table, and a stable
//                scatter that ranks equal digits with __match_any_sync.
//                Stability makes the permutation unique, so it is compared
//                bit-exactly with a CPU stable sort;
//   4. interleave: inside every block of 32 keys the stable order is dealt
//                round-robin over the keys (round r = each key's r-th
//                particle), so that a warp whose lanes own the 32 cells reads
//                one contiguous run of slots per round.
#include "sort.cuh"

namespace polypic {

// ---------------------------------------------------------------- keys
__global__ void __launch_bounds__(256) k_keys(int64_t n, const float *__restrict__ x,
                                              const float *__restrict__ y,
                                              const float *__restrict__ z, GridGeom g,
                                              uint32_t *__restrict__ key,
                                              uint32_t *__restrict__ counts,
                                              uint32_t *__restrict__ status) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool live = p < n;
    uint32_t k = 0;
    bool bad = false;
    if (live) {
        float vx = cell_coord(x[p], g.inv_dx);
        float vy = cell_coord(y[p], g.inv_dx);
        float vz = cell_coord(z[p], g.inv_dx);
        bad = !(coord_valid(vx, g.n[0]) && coord_valid(vy, g.n[1]) && coord_valid(vz, g.n[2]));
        k = cell_key(g, cell_index(vx, g.n[0]), cell_index(vy, g.n[1]), cell_index(vz, g.n[2]));
        key[p] = k;
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, kFlagOutOfDomain);
    unsigned active = __ballot_sync(0xffffffffu, live);
    if (live) {
        unsigned peers = __match_any_sync(active, k);
        if ((int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&counts[k], (uint32_t)__popc(peers));
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

// ---------------------------------------------------------------- radix
// Each CTA owns kRadixTile consecutive keys; warp w owns the kRadixItems*32
// keys starting at tile + w * kRadixItems * 32, visited 32 at a time.
__global__ void __launch_bounds__(kRadixThreads) k_radix_up(const uint32_t *__restrict__ keys,
                                                            int64_t n, int shift, int bits,
                                                            uint32_t *__restrict__ hist,
                                                            int ntiles) {
    __shared__ uint32_t s_hist[256];
    int radix = 1 << bits;
    for (int i = threadIdx.x; i < 256; i += kRadixThreads) s_hist[i] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kRadixTile;
    for (int i = threadIdx.x; i < kRadixTile; i += kRadixThreads) {
        int64_t idx = base + i;
        if (idx < n) atomicAdd(&s_hist[(keys[idx] >> shift) & (uint32_t)(radix - 1)], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < radix; d += kRadixThreads)
        hist[(int64_t)d * ntiles + blockIdx.x] = s_hist[d];
}

template <bool FIRST, bool LAST>
__global__ void __launch_bounds__(kRadixThreads) k_radix_down(
    const uint32_t *__restrict__ keys_in, const uint32_t *__restrict__ vals_in,
    uint32_t *__restrict__ keys_out, uint32_t *__restrict__ vals_out, int64_t n, int shift,
    int bits, const uint32_t *__restrict__ offsets, int ntiles) {
    constexpr int kWarps = kRadixThreads / 32;
    __shared__ uint32_t s_warp[kWarps][256];
    __shared__ uint32_t s_off[256];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const uint32_t mask = (1u << bits) - 1u;
    for (int i = tid; i < kWarps * 256; i += kRadixThreads) (&s_warp[0][0])[i] = 0;
    for (int d = tid; d < 256; d += kRadixThreads)
        s_off[d] = d <= (int)mask ? offsets[(int64_t)d * ntiles + blockIdx.x] : 0u;
    __syncthreads();

    const int64_t base = (int64_t)blockIdx.x * kRadixTile + (int64_t)w * (kRadixItems * 32);
    const unsigned lt = (1u << lane) - 1u;
    uint32_t k[kRadixItems], v[kRadixItems], loc[kRadixItems];
    int dg[kRadixItems];
#pragma unroll
    for (int r = 0; r < kRadixItems; ++r) {
        int64_t idx = base + r * 32 + lane;
        bool valid = idx < n;
        k[r] = valid ? keys_in[idx] : 0u;
        v[r] = valid ? (FIRST ? (uint32_t)idx : vals_in[idx]) : 0u;
        int d = valid ? (int)((k[r] >> shift) & mask) : 256;  // 256: no digit
        dg[r] = d;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        uint32_t prior = d < 256 ? s_warp[w][d] : 0u;
        __syncwarp();
        if (d < 256 && lane == __ffs(peers) - 1) s_warp[w][d] = prior + (uint32_t)__popc(peers);
        __syncwarp();
        loc[r] = prior + (uint32_t)__popc(peers & lt);
    }
    __syncthreads();
    // exclusive prefix of each digit's count over the warps (warp order = key order)
    for (int d = tid; d <= (int)mask; d += kRadixThreads) {
        uint32_t run = 0;
#pragma unroll
        for (int ww = 0; ww < kWarps; ++ww) {
            uint32_t c = s_warp[ww][d];
            s_warp[ww][d] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRadixItems; ++r) {
        int d = dg[r];
        if (d < 256) {
            uint32_t pos = s_off[d] + s_warp[w][d] + loc[r];
            if (!LAST) keys_out[pos] = k[r];
            vals_out[pos] = v[r];
        }
    }
}

// ---------------------------------------------------------------- block interleave
// Slot order used by the transfers: inside each block of 32 keys, round r
// lists the r-th particle (stable order) of every key holding more than r
// particles, keys ascending.  One warp per block, lane = key.
__global__ void __launch_bounds__(256) k_block_interleave(const uint32_t *__restrict__ in,
                                                          const uint32_t *__restrict__ cs,
                                                          uint32_t *__restrict__ out,
                                                          uint32_t nblocks) {
    const int lane = threadIdx.x & 31;
    const uint32_t b = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (b >= nblocks) return;
    const uint32_t k = b * 32 + lane;
    const uint32_t s0 = cs[k], n = cs[k + 1] - s0, base = cs[b * 32];
    const uint32_t maxn = __reduce_max_sync(0xffffffffu, n);
    const unsigned lt = (1u << lane) - 1u;
    uint32_t off = 0;
    for (uint32_t r = 0; r < maxn; ++r) {
        const unsigned mask = __ballot_sync(0xffffffffu, n > r);
        if (n > r) out[base + off + __popc(mask & lt)] = in[s0 + r];
        off += __popc(mask);
    }
}

// ---------------------------------------------------------------- driver
int key_bits(int64_t num_keys) {
    int b = 1;
    while (((int64_t)1 << b) < num_keys) ++b;
    return b;
}

size_t sort_scratch_bytes(int64_t count, int64_t num_keys) {
    int64_t ntiles = (count + kRadixTile - 1) / kRadixTile;
    size_t words = 0;
    words += 5 * (size_t)count + 64;                          // key/value ping-pong + stable perm
    words += 256 * (size_t)ntiles + 64;                       // digit histograms
    words += scan_scratch_words(256 * ntiles) + 64;           // their scan
    words += scan_scratch_words(num_keys + 1) + 64;           // cell-count scan
    return words * sizeof(uint32_t) + 8 * 256;
}

cudaError_t sort_particles(const GridGeom &g, int64_t num_keys, int64_t count, const float *x,
                           const float *y, const float *z, uint32_t *key, uint32_t *perm,
                           uint32_t *cell_start, uint32_t *status, Workspace &ws,
                           cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(cell_start, 0, sizeof(uint32_t) * (num_keys + 1), s);
    if (e != cudaSuccess) return e;
    if (count == 0) return cudaSuccess;
    int64_t ntiles = (count + kRadixTile - 1) / kRadixTile;
    uint32_t *ka = ws.take<uint32_t>(count), *va = ws.take<uint32_t>(count);
    uint32_t *kb = ws.take<uint32_t>(count), *vb = ws.take<uint32_t>(count);
    uint32_t *stable = ws.take<uint32_t>(count);
    uint32_t *hist = ws.take<uint32_t>(256 * ntiles);
    uint32_t *hscan = ws.take<uint32_t>(scan_scratch_words(256 * ntiles));
    uint32_t *cscan = ws.take<uint32_t>(scan_scratch_words(num_keys + 1));
    if (ws.overflow) return cudaErrorInvalidValue;

    int kblocks = (int)((count + 255) / 256);
    k_keys<<<kblocks, 256, 0, s>>>(count, x, y, z, g, key, cell_start, status);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = exclusive_scan(cell_start, cell_start, num_keys + 1, cscan, s)) != cudaSuccess) return e;

    int bits = key_bits(num_keys);
    int passes = (bits + 7) / 8;
    int per = (bits + passes - 1) / passes;
    const uint32_t *kin = key;
    const uint32_t *vin = nullptr;
    int shift = 0;
    for (int pass = 0; pass < passes; ++pass) {
        int pb = (shift + per <= bits) ? per : bits - shift;
        bool first = pass == 0, last = pass == passes - 1;
        uint32_t *kout = (pass & 1) ? kb : ka;
        uint32_t *vout = last ? stable : ((pass & 1) ? vb : va);
        k_radix_up<<<(int)ntiles, kRadixThreads, 0, s>>>(kin, count, shift, pb, hist, (int)ntiles);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = exclusive_scan(hist, hist, ((int64_t)1 << pb) * ntiles, hscan, s)) != cudaSuccess)
            return e;
        if (first && last)
            k_radix_down<true, true><<<(int)ntiles, kRadixThreads, 0, s>>>(
                kin, vin, kout, vout, count, shift, pb, hist, (int)ntiles);
        else if (first)
            k_radix_down<true, false><<<(int)ntiles, kRadixThreads, 0, s>>>(
                kin, vin, kout, vout, count, shift, pb, hist, (int)ntiles);
        else if (last)
            k_radix_down<false, true><<<(int)ntiles, kRadixThreads, 0, s>>>(
                kin, vin, kout, vout, count, shift, pb, hist, (int)ntiles);
        else
            k_radix_down<false, false><<<(int)ntiles, kRadixThreads, 0, s>>>(
                kin, vin, kout, vout, count, shift, pb, hist, (int)ntiles);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        kin = kout;
        vin = vout;
        shift += pb;
    }
    const uint32_t nblocks = (uint32_t)(num_keys / 32);
    k_block_interleave<<<(nblocks + 7) / 8, 256, 0, s>>>(stable, cell_start, perm, nblocks);
    return cudaGetLastError();
}

}  // namespace polypic

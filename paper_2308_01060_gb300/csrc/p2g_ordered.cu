// p2g_ordered.cu -- P2G of ordered phases (Eqs 1-5, 13, 15-19): the particle
// arrays are in their own slot order (tile_order.cuh), so there is no perm to
// follow and the lanes of a warp own cells of similar population.
//
//   * one CTA of 8 warps per tile; warp g owns group g of the tile's cells
//     ranked by count, lane = cell.  In round r the lanes read the r-th
//     particle of their cells from slots gstart[g] + (earlier rounds) + lane
//     rank: one contiguous run of the particle arrays, read directly;
//   * per pass (face grid A) a lane accumulates its cell's padded 4 x 3 x 3
//     footprint in registers (p2g_kernel.cuh), the warp adds its 32 footprints
//     into its own tile region in 36 phases (distinct cells hit distinct
//     nodes), and the CTA adds the 8 warp regions in warp order into the tile
//     region in scratch, which k_p2g_reduce sums over tiles as for the
//     block-interleaved kernel.  No float atomics: bit-identical runs.
//   * one cp.async stream per warp runs through the three passes.
#include "p2g_kernel.cuh"
#include "tile_order.cuh"

namespace polypic {

constexpr int kOrdWarps = kGroups;  // warp g = group g
// A warp's region for one pass: mass and momentum of one face grid's tile.
constexpr int kPassFloats = 2 * (tile_size(2) > tile_size(0) ? tile_size(2) : tile_size(0));
static_assert(tile_size(1) == tile_size(0), "face grids 0 and 1 have equal tile regions");

template <int R> constexpr int ordered_smem_bytes() {
    return (kOrdWarps * kPassFloats + kOrdWarps * kStages * Stage<R>::NV * 32) * 4;
}
static_assert(ordered_smem_bytes<27>() <= 200 * 1024, "ordered P2G staging exceeds a CTA");

template <int A> __device__ __forceinline__ int tile_index(int ix, int iy, int iz) {
    return (iz * tile_y(A) + iy) * tile_x(A) + ix;
}

// Issue side of a warp's stream: pass ia, round ir, its slot sn (ia == 3: done).
struct OPipe {
    int ia;
    uint32_t ir, sn;
    int ring;  // stage holding the next round to consume
};

template <int R, int FMT>
__device__ __forceinline__ void opipe_issue(const P2GArgs &P, OPipe &q, uint32_t gs, uint32_t n,
                                            uint32_t maxn, unsigned lt, float *st, int lane) {
    if (q.ia < 3 && n > q.ir) {  // q.ia is warp-uniform
        if (q.ia == 0) stage_particle<R, FMT, 0, false>(P, q.sn, q.sn, st, lane);
        else if (q.ia == 1) stage_particle<R, FMT, 1, false>(P, q.sn, q.sn, st, lane);
        else stage_particle<R, FMT, 2, false>(P, q.sn, q.sn, st, lane);
    }
    cp_async_commit();
    if (q.ia < 3 && ++q.ir == maxn) {
        q.ir = 0;
        ++q.ia;
    }
    if (q.ia < 3) q.sn = round_slot(gs, n, q.ir, lt);
}

// One pass of a warp: its group's rounds on face grid A, then the merge of
// the lanes' footprints into the warp's region.
template <int R, int FMT, int A>
__device__ __forceinline__ void opass(const P2GArgs &P, OPipe &q, uint32_t gs, uint32_t n,
                                      uint32_t maxn, int ci, int cj, int ck, int gi, int gj,
                                      int gk, int lane, float *reg, float *stage, bool &bad) {
    constexpr int N = tile_size(A);
    if (maxn == 0) return;  // warp-uniform
    using S = Stage<R>;
    for (int i = lane; i < 2 * N; i += 32) reg[i] = 0.0f;
    __syncwarp();
    float am[4][3][3], av[4][3][3];
#pragma unroll
    for (int d = 0; d < 4; ++d)
#pragma unroll
        for (int kv = 0; kv < 3; ++kv)
#pragma unroll
            for (int kw = 0; kw < 3; ++kw) am[d][kv][kw] = av[d][kv][kw] = 0.0f;
    const unsigned lt = (1u << lane) - 1u;
    for (uint32_t r = 0; r < maxn; ++r) {
        float *st = stage + q.ring * S::NV * 32;
        cp_async_wait<kStages - 1>();
        if (n > r) {
            const float px = st[S::kX * 32 + lane], py = st[S::kY * 32 + lane],
                        pz = st[S::kZ * 32 + lane];
            float mt = st[S::kM * 32 + lane];
            if (P.mass_abs) mt += st[S::kMabs * 32 + lane];
            const float v0 = cell_coord(px, P.g.inv_dx), v1 = cell_coord(py, P.g.inv_dx),
                        v2 = cell_coord(pz, P.g.inv_dx);
            const bool ok = coord_valid(v0, P.g.n[0]) && coord_valid(v1, P.g.n[1]) &&
                            coord_valid(v2, P.g.n[2]) && (int)floorf(v0) == gi &&
                            (int)floorf(v1) == gj && (int)floorf(v2) == gk;
            if (ok) {
                const float vu = A == 0 ? v0 : (A == 1 ? v1 : v2);
                const float vv = A == 0 ? v1 : v0;
                const float vw = A == 2 ? v1 : v2;
                const Axis au = axis_decide(vu, true), av_ = axis_decide(vv, false),
                           aw = axis_decide(vw, false);
                const int cu = A == 0 ? gi : (A == 1 ? gj : gk);
                const int shift = au.base - (cu - 1);
                accumulate<R, FMT, A, false>(P, st, lane, mt, shift, stencil_1d_scaled(au.t, P.s1, P.s2),
                                             stencil_1d_scaled(av_.t, P.s1, P.s2), stencil_1d_scaled(aw.t, P.s1, P.s2), au.guard,
                                             av_.guard, aw.guard, am, av);
            } else {
                bad = true;
            }
        }
        // refill the stage just consumed with the next round of the stream
        opipe_issue<R, FMT>(P, q, gs, n, maxn, lt, st, lane);
        q.ring = q.ring + 1 == kStages ? 0 : q.ring + 1;
    }
    // merge into the warp's tile region, one node offset per phase
    const int cu = A == 0 ? ci : (A == 1 ? cj : ck);
    const int cv = A == 0 ? cj : ci;
    const int cw = A == 2 ? cj : ck;
#pragma unroll
    for (int d = 0; d < 4; ++d)
#pragma unroll
        for (int kv = 0; kv < 3; ++kv)
#pragma unroll
            for (int kw = 0; kw < 3; ++kw) {
                const int nu = cu + d, nv = cv + kv, nw = cw + kw;
                const int ix = A == 0 ? nu : nv;
                const int iy = A == 0 ? nv : (A == 1 ? nu : nw);
                const int iz = A == 2 ? nu : nw;
                const int idx = tile_index<A>(ix, iy, iz);
                reg[idx] += am[d][kv][kw];
                reg[N + idx] += av[d][kv][kw];
                __syncwarp();
            }
}

// The CTA adds the used warp regions of pass A, in warp order, into the
// tile region in scratch.
template <int A>
__device__ __forceinline__ void merge_pass(const float *s_reg, const bool *used, float *dst) {
    constexpr int N = tile_size(A);
    for (int i = threadIdx.x; i < N; i += kOrdWarps * 32) {
        float sm = 0.0f, sv = 0.0f;
#pragma unroll
        for (int w = 0; w < kOrdWarps; ++w) {
            if (!used[w]) continue;
            sm += s_reg[w * kPassFloats + i];
            sv += s_reg[w * kPassFloats + N + i];
        }
        dst[tile_off(A, 0) + i] = sm;
        dst[tile_off(A, 1) + i] = sv;
    }
}

template <int R, int FMT>
// 27 modes: one CTA per SM (the compiler's register allocation); fewer modes
// fit two CTAs per SM.
__global__ void __launch_bounds__(kOrdWarps * 32, (R == 27 ? 1 : 2)) k_p2g_ordered(P2GArgs P) {
    extern __shared__ float smem[];
    __shared__ TileOrder o;
    __shared__ bool s_used[kOrdWarps];
    float *s_reg = smem;                                   // [8][kPassFloats]
    float *s_stage = smem + kOrdWarps * kPassFloats;       // [8][kStages][NV][32]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const uint32_t tile = blockIdx.x;
    const bool tile_empty =
        P.cell_start[tile * kTileCells] == P.cell_start[tile * kTileCells + kTileCells];
    if (threadIdx.x == 0) P.tile_live[tile] = tile_empty ? 0 : 1;
    if (tile_empty) return;  // CTA-uniform
    rank_tile<kOrdWarps * 32>(P.cell_start, tile, o);
    const uint32_t rk = (uint32_t)threadIdx.x;  // rank 32 g + lane
    const uint32_t n = o.n[rk], gs = o.gstart[warp];
    const uint32_t maxn = __reduce_max_sync(0xffffffffu, n);
    int ci, cj, ck;
    local_cell(o.cell[rk], ci, cj, ck);
    const int tx = (int)(tile % (uint32_t)P.g.tiles[0]);
    const int ty = (int)((tile / (uint32_t)P.g.tiles[0]) % (uint32_t)P.g.tiles[1]);
    const int tz = (int)(tile / ((uint32_t)P.g.tiles[0] * (uint32_t)P.g.tiles[1]));
    const int gi = 8 * tx + ci, gj = 8 * ty + cj, gk = 4 * tz + ck;
    if (lane == 0) s_used[warp] = maxn > 0;
    float *reg = s_reg + warp * kPassFloats;
    float *stage = s_stage + warp * kStages * Stage<R>::NV * 32;
    float *dst = P.scratch + (size_t)tile * kTileFloats;

    OPipe q;
    q.ia = maxn > 0 ? 0 : 3;
    q.ir = 0;
    q.ring = 0;
    q.sn = round_slot(gs, n, 0, lt);
#pragma unroll
    for (int k = 0; k < kStages; ++k)
        opipe_issue<R, FMT>(P, q, gs, n, maxn, lt, stage + k * Stage<R>::NV * 32, lane);
    bool bad = false;
    opass<R, FMT, 0>(P, q, gs, n, maxn, ci, cj, ck, gi, gj, gk, lane, reg, stage, bad);
    __syncthreads();
    merge_pass<0>(s_reg, s_used, dst);
    __syncthreads();
    opass<R, FMT, 1>(P, q, gs, n, maxn, ci, cj, ck, gi, gj, gk, lane, reg, stage, bad);
    __syncthreads();
    merge_pass<1>(s_reg, s_used, dst);
    __syncthreads();
    opass<R, FMT, 2>(P, q, gs, n, maxn, ci, cj, ck, gi, gj, gk, lane, reg, stage, bad);
    __syncthreads();
    merge_pass<2>(s_reg, s_used, dst);
    cp_async_wait<0>();
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(P.status, kFlagOutOfDomain);
}

template <int R, int FMT>
static cudaError_t launch_ordered(const P2GArgs &P, int ntiles, cudaStream_t s) {
    constexpr int smem = ordered_smem_bytes<R>();
    static int configured_device = -1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (configured_device != dev) {
        e = cudaFuncSetAttribute(k_p2g_ordered<R, FMT>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        configured_device = dev;
    }
    k_p2g_ordered<R, FMT><<<ntiles, kOrdWarps * 32, smem, s>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_p2g_ordered(const P2GArgs &P, int R, int fmt, int ntiles, cudaStream_t s) {
#define POLYPIC_P2GO_CASE(RR, FF) \
    if (R == RR && fmt == FF) return launch_ordered<RR, FF>(P, ntiles, s);
    POLYPIC_P2GO_CASE(1, POLYPIC_COEFF_F32)
    POLYPIC_P2GO_CASE(4, POLYPIC_COEFF_F32)
    POLYPIC_P2GO_CASE(8, POLYPIC_COEFF_F32)
    POLYPIC_P2GO_CASE(27, POLYPIC_COEFF_F32)
    POLYPIC_P2GO_CASE(1, POLYPIC_COEFF_BF16)
    POLYPIC_P2GO_CASE(4, POLYPIC_COEFF_BF16)
    POLYPIC_P2GO_CASE(8, POLYPIC_COEFF_BF16)
    POLYPIC_P2GO_CASE(27, POLYPIC_COEFF_BF16)
    POLYPIC_P2GO_CASE(1, POLYPIC_COEFF_F16)
    POLYPIC_P2GO_CASE(4, POLYPIC_COEFF_F16)
    POLYPIC_P2GO_CASE(8, POLYPIC_COEFF_F16)
    POLYPIC_P2GO_CASE(27, POLYPIC_COEFF_F16)
#undef POLYPIC_P2GO_CASE
    return cudaErrorInvalidValue;
}

}  // namespace polypic

// g2p2g.cu -- the fused transfer: G2P of step n (the fit of Section 3.3 and
// the advection) and P2G of step n + 1 (Eqs 1-5, 13) in one pass, so that the
// new coefficients of a particle that stays in its cell never reach HBM.
//
// The P2G of step n + 1 needs the particles grouped by their new cells.  A
// particle that stays in its cell keeps its place in step n's lane-per-cell
// rounds, so the kernel runs the P2G tile scheme on step n's sort: one CTA
// per 8x8x4-cell tile (its velocity footprint staged in shared memory, as
// for G2P), one warp per 4x4x2-cell block, one lane per cell.  For component
// pass A and round r the lane fits its particle from the staged grid (pass 0
// also fits the velocity modes of the other two components and advects,
// writing x^{n+1}, which passes 1 and 2 read back), then accumulates the
// particle's contribution at x^{n+1} into its 4 x 3 x 3 register footprint;
// the footprints merge into the tile region exactly as in P2G.  A particle
// whose new position lies in another cell (a mover) is not accumulated: its
// coefficients are written to the output state and it is flagged, and the
// host routes the movers through a compact spill set, the ordinary sort and
// P2G, whose reduction adds onto the grid.  Every sum runs in a fixed order:
// the result is bit-identical from run to run.
#include "g2p2g.cuh"
#include "g2p_fit.cuh"
#include "p2g_tiles.cuh"

namespace polypic {

namespace {

template <int R, int A>
__device__ __forceinline__ void fit_component(const float *s_tile, int ox, int oy, int oz,
                                              const Axis (&ac)[3], const Axis (&af)[3],
                                              const Stencil1D (&sc)[3], const Stencil1D (&sf)[3],
                                              float inv1, float inv2, float (&C)[R]) {
    if constexpr (A == 0)
        g2p_component<R, 0, Tile<0>::X, Tile<0>::Y>(s_tile, af[0].base - ox, ac[1].base - oy,
                                                    ac[2].base - oz, sf[0], af[0].guard, sc[1],
                                                    ac[1].guard, sc[2], ac[2].guard, inv1, inv2, C);
    else if constexpr (A == 1)
        g2p_component<R, 1, Tile<1>::X, Tile<1>::Y>(s_tile + kVelTileOff1, ac[0].base - ox,
                                                    af[1].base - oy, ac[2].base - oz, sc[0],
                                                    ac[0].guard, sf[1], af[1].guard, sc[2],
                                                    ac[2].guard, inv1, inv2, C);
    else
        g2p_component<R, 2, Tile<2>::X, Tile<2>::Y>(s_tile + kVelTileOff2, ac[0].base - ox,
                                                    ac[1].base - oy, af[2].base - oz, sc[0],
                                                    ac[0].guard, sc[1], ac[1].guard, sf[2],
                                                    af[2].guard, inv1, inv2, C);
}

// One component pass of one block: the rounds of the lane's cell, then the
// 36-phase merge of the footprints into the block region.
template <int R, int A>
__device__ __forceinline__ void fused_pass(const G2P2GArgs &Q, const float *s_tile, int ox, int oy,
                                           int oz, uint32_t bs, uint32_t n_c, uint32_t maxn,
                                           int ci, int cj, int ck, int gi, int gj, int gk,
                                           int lane, float *reg, float *st, bool &bad) {
    using S = Stage<R, false, POLYPIC_COEFF_F32>;
    const P2GArgs &P = Q.p2g;
    const GridGeom &g = P.g;
    Foot F;
    F.zero();
    const unsigned lt = (1u << lane) - 1u;
    const int64_t cnt = P.count;
    for (uint32_t r = 0; r < maxn; ++r) {
        const uint32_t slot = round_slot(bs, n_c, r, lt);
        if (n_c > r) {
            const uint32_t p = P.perm[slot];
            const float px = Q.x[p], py = Q.y[p], pz = Q.z[p];
            const float m = P.mass[p], mabs = P.mass_abs ? P.mass_abs[p] : 0.0f;
            const float v0 = cell_coord(px, g.inv_dx), v1 = cell_coord(py, g.inv_dx),
                        v2 = cell_coord(pz, g.inv_dx);
            const bool in_cell = coord_valid(v0, g.n[0]) && coord_valid(v1, g.n[1]) &&
                                 coord_valid(v2, g.n[2]) && (int)floorf(v0) == gi &&
                                 (int)floorf(v1) == gj && (int)floorf(v2) == gk;
            if (!in_cell) {
                bad = true;
                if (A == 0) Q.moved[slot] = 0;
            } else {
                const float vv[3] = {v0, v1, v2};
                Axis ac[3], af[3];
                Stencil1D sc[3], sf[3];
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    ac[b] = axis_decide(vv[b], false);
                    af[b] = axis_decide(vv[b], true);
                    sc[b] = stencil_1d(ac[b].t);
                    sf[b] = stencil_1d(af[b].t);
                }
                float C[R];
                fit_component<R, A>(s_tile, ox, oy, oz, ac, af, sc, sf, Q.inv1, Q.inv2, C);
                float x1, y1, z1;
                if constexpr (A == 0) {
                    // the velocity is mode 0 of each component (the same bits as
                    // G2P's full fit: mode 0 contracts the same rows in order)
                    float c1[1], c2[1];
                    fit_component<1, 1>(s_tile, ox, oy, oz, ac, af, sc, sf, Q.inv1, Q.inv2, c1);
                    fit_component<1, 2>(s_tile, ox, oy, oz, ac, af, sc, sf, Q.inv1, Q.inv2, c2);
                    if (!(isfinite(C[0]) && isfinite(c1[0]) && isfinite(c2[0])))
                        atomicOr(P.status, kFlagNonFinite);
                    x1 = fminf(fmaxf(fmaf(Q.dt, C[0], px), g.lo[0]), g.hi[0]);
                    y1 = fminf(fmaxf(fmaf(Q.dt, c1[0], py), g.lo[1]), g.hi[1]);
                    z1 = fminf(fmaxf(fmaf(Q.dt, c2[0], pz), g.lo[2]), g.hi[2]);
                    Q.ox[slot] = x1;
                    Q.oy[slot] = y1;
                    Q.oz[slot] = z1;
                    Q.omass[slot] = m;
                    if (Q.omass_abs) Q.omass_abs[slot] = mabs;
                } else {
                    x1 = Q.ox[slot];
                    y1 = Q.oy[slot];
                    z1 = Q.oz[slot];
                }
                const float w0 = cell_coord(x1, g.inv_dx), w1 = cell_coord(y1, g.inv_dx),
                            w2 = cell_coord(z1, g.inv_dx);
                const bool stays = (int)floorf(w0) == gi && (int)floorf(w1) == gj &&
                                   (int)floorf(w2) == gk;
                if (!stays) {
                    // a mover: its coefficients go out for the spill P2G
                    float *oc = Q.ocoeff + (int64_t)A * R * cnt + slot;
#pragma unroll
                    for (int k = 0; k < R; ++k, oc += cnt) *oc = C[k];
                    if (A == 0) Q.moved[slot] = 1;
                } else {
                    if (A == 0) Q.moved[slot] = 0;
#pragma unroll
                    for (int k = 0; k < R; ++k) st[(S::kC + k) * 32 + lane] = C[k];
                    const float wu = A == 0 ? w0 : (A == 1 ? w1 : w2);
                    const float wv = A == 0 ? w1 : w0;
                    const float ww = A == 2 ? w1 : w2;
                    const Axis au = axis_decide(wu, true), av_ = axis_decide(wv, false),
                               aw = axis_decide(ww, false);
                    const int cu = A == 0 ? gi : (A == 1 ? gj : gk);
                    const int shift = au.base - (cu - 1);
                    accumulate<R, POLYPIC_COEFF_F32, A, false, false>(
                        P, st, lane, m + mabs, shift, stencil_1d_scaled(au.t, P.s1, P.s2),
                        stencil_1d_scaled(av_.t, P.s1, P.s2), stencil_1d_scaled(aw.t, P.s1, P.s2),
                        au.guard, av_.guard, aw.guard, F);
                }
            }
        }
    }
    // merge the 32 footprints into the block region, one node offset per phase
    const int cu = A == 0 ? ci : (A == 1 ? cj : ck);
    const int cv = A == 0 ? cj : ci;
    const int cw = A == 2 ? cj : ck;
    float *rm = reg + reg_off(A, 0);
    float *rv = reg + reg_off(A, 1);
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
                const int idx = region_index<A>(ix, iy, iz);
                rm[idx] += F.m(d, kv, kw);
                rv[idx] += F.v(d, kv, kw);
                __syncwarp();
            }
}

template <int R>
__global__ void __launch_bounds__(kP2GWarps * 32, 1) k_g2p2g(G2P2GArgs Q) {
    extern __shared__ float smem[];
    __shared__ bool s_empty[kP2GWarps];
    using S = Stage<R, false, POLYPIC_COEFF_F32>;
    float *s_reg = smem;                                         // [8][kRegionFloats]
    float *s_stage = smem + kP2GWarps * kRegionFloats;            // [8][NV][32]
    float *s_tile = s_stage + kP2GWarps * S::NV * 32;             // staged velocity
    const P2GArgs &P = Q.p2g;
    const GridGeom &g = P.g;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t tile = blockIdx.x;
    const bool tile_empty = P.cell_start[tile * 256] == P.cell_start[tile * 256 + 256];
    if (threadIdx.x == 0) P.tile_live[tile] = tile_empty ? 0 : 1;
    if (tile_empty) return;  // CTA-uniform
    const int tx = (int)(tile % (uint32_t)g.tiles[0]);
    const int ty = (int)((tile / (uint32_t)g.tiles[0]) % (uint32_t)g.tiles[1]);
    const int tz = (int)(tile / ((uint32_t)g.tiles[0] * (uint32_t)g.tiles[1]));
    const int ox = 8 * tx - 1, oy = 8 * ty - 1, oz = 4 * tz - 1;
    stage_velocity<0>(g, Q.vel, tx, ty, tz, s_tile);
    __syncthreads();

    const uint32_t b = tile * kP2GWarps + warp;
    const uint32_t k = b * 32 + lane;
    const uint32_t n_c = P.cell_start[k + 1] - P.cell_start[k];
    const uint32_t bs = P.cell_start[b * 32];
    const uint32_t maxn = __reduce_max_sync(0xffffffffu, n_c);
    float *reg = s_reg + warp * kRegionFloats;
    float *st = s_stage + warp * S::NV * 32;
    if (lane == 0) s_empty[warp] = maxn == 0;
    if (maxn > 0) {
        for (int i = lane; i < kRegionFloats; i += 32) reg[i] = 0.0f;
        __syncwarp();
        int i0, j0, k0;
        block_origin(g, b, i0, j0, k0);
        const int ci = lane & 3, cj = (lane >> 2) & 3, ck = lane >> 4;
        const int gi = i0 + ci, gj = j0 + cj, gk = k0 + ck;
        bool bad = false;
        fused_pass<R, 0>(Q, s_tile, ox, oy, oz, bs, n_c, maxn, ci, cj, ck, gi, gj, gk, lane, reg,
                         st, bad);
        fused_pass<R, 1>(Q, s_tile, ox, oy, oz, bs, n_c, maxn, ci, cj, ck, gi, gj, gk, lane, reg,
                         st, bad);
        fused_pass<R, 2>(Q, s_tile, ox, oy, oz, bs, n_c, maxn, ci, cj, ck, gi, gj, gk, lane, reg,
                         st, bad);
        if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(P.status, kFlagOutOfDomain);
    }
    __syncthreads();
    float *dst = P.scratch + (size_t)tile * kTileFloats;
    merge_tile<0>(s_reg, s_empty, dst);
    merge_tile<1>(s_reg, s_empty, dst);
    merge_tile<2>(s_reg, s_empty, dst);
}

template <int R> constexpr int fused_smem_bytes() {
    return (kP2GWarps * kRegionFloats + kP2GWarps * Stage<R, false, POLYPIC_COEFF_F32>::NV * 32 +
            kVelTileFloats) * 4;
}
static_assert(fused_smem_bytes<27>() <= 227 * 1024, "fused transfer exceeds shared memory");

// Movers per tile: the flags of the tile's slot range.
__global__ void __launch_bounds__(256) k_count_movers(const uint32_t *cell_start,
                                                      const uint8_t *moved, uint32_t *counts) {
    const uint32_t tile = blockIdx.x;
    const uint32_t jb = cell_start[tile * 256], je = cell_start[tile * 256 + 256];
    uint32_t c = 0;
    for (uint32_t j = jb + threadIdx.x; j < je; j += 256) c += moved[j];
    c = __reduce_add_sync(0xffffffffu, c);
    __shared__ uint32_t s[8];
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < 8; ++w) t += s[w];
        counts[tile] = t;
    }
}

// Exclusive scan of the per-tile counts in one CTA; offsets[ntiles] = total.
__global__ void __launch_bounds__(1024) k_scan_movers(const uint32_t *counts, int64_t ntiles,
                                                      uint32_t *offsets) {
    __shared__ uint32_t s_w[32];
    __shared__ uint32_t s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t base = 0; base < ntiles; base += 1024) {
        const int64_t i = base + threadIdx.x;
        const uint32_t v = i < ntiles ? counts[i] : 0u;
        uint32_t x = v;  // inclusive warp scan
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_w[warp] = x;
        __syncthreads();
        if (warp == 0) {
            uint32_t t = s_w[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            s_w[lane] = t;  // inclusive over warps
        }
        __syncthreads();
        const uint32_t before = (warp > 0 ? s_w[warp - 1] : 0u) + x - v;
        if (i < ntiles) offsets[i] = s_carry + before;
        __syncthreads();
        if (threadIdx.x == 0) s_carry += s_w[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) offsets[ntiles] = s_carry;
}

// The movers of each tile, in slot order, to the spill set at the tile's
// offset: positions, masses, the 3R coefficients (rows of the spill's own
// count, the total number of movers).  Per chunk of 256 slots the CTA first
// lists its movers in shared memory, then copies their coefficients with
// every thread busy (consecutive threads write consecutive spill entries of
// one row).  Nothing is written past `capacity`.
__global__ void __launch_bounds__(256) k_compact_movers(SpillArgs S) {
    __shared__ uint32_t s_w[8];
    __shared__ uint32_t s_src[256];
    const uint32_t tile = blockIdx.x;
    const uint32_t jb = S.cell_start[tile * 256], je = S.cell_start[tile * 256 + 256];
    const uint32_t total = S.offsets[S.ntiles];
    if (total > S.capacity) return;
    uint32_t next = S.offsets[tile];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int rows = 3 * S.R;
    for (uint32_t j0 = jb; j0 < je; j0 += 256) {
        const uint32_t j = j0 + threadIdx.x;
        const bool mv = j < je && S.moved[j];
        const unsigned bal = __ballot_sync(0xffffffffu, mv);
        if (lane == 0) s_w[warp] = __popc(bal);
        __syncthreads();
        uint32_t before = 0, all = 0;
        for (int w = 0; w < 8; ++w) {
            before += w < warp ? s_w[w] : 0u;
            all += s_w[w];
        }
        if (mv) {
            const uint32_t i = before + __popc(bal & ((1u << lane) - 1u));
            const uint32_t d = next + i;
            s_src[i] = j;
            S.x[d] = S.ox[j];
            S.y[d] = S.oy[j];
            S.z[d] = S.oz[j];
            S.mass[d] = S.omass[j];
            if (S.mass_abs) S.mass_abs[d] = S.omass_abs[j];
        }
        __syncthreads();
        for (uint32_t item = threadIdx.x; item < all * (uint32_t)rows; item += 256) {
            const uint32_t i = item % all, r = item / all;
            S.coeff[(int64_t)r * total + next + i] = S.ocoeff[(int64_t)r * S.count + s_src[i]];
        }
        next += all;
        __syncthreads();
    }
}

}  // namespace

cudaError_t g2p2g_tiles(const G2P2GArgs &Q, int R, cudaStream_t s) {
    const int grid = (int)(Q.p2g.nblocks / kP2GWarps);
#define POLYPIC_FUSED_CASE(RR)                                                               \
    if (R == RR) {                                                                          \
        const cudaError_t e = cudaFuncSetAttribute(                                         \
            k_g2p2g<RR>, cudaFuncAttributeMaxDynamicSharedMemorySize, fused_smem_bytes<RR>()); \
        if (e != cudaSuccess) return e;                                                     \
        k_g2p2g<RR><<<grid, kP2GWarps * 32, fused_smem_bytes<RR>(), s>>>(Q);                \
        return cudaGetLastError();                                                          \
    }
    POLYPIC_FUSED_CASE(1)
    POLYPIC_FUSED_CASE(4)
    POLYPIC_FUSED_CASE(8)
    POLYPIC_FUSED_CASE(27)
#undef POLYPIC_FUSED_CASE
    return cudaErrorInvalidValue;
}

cudaError_t count_and_scan_movers(const uint32_t *cell_start, const uint8_t *moved, int64_t ntiles,
                                  uint32_t *counts, uint32_t *offsets, cudaStream_t s) {
    k_count_movers<<<(unsigned)ntiles, 256, 0, s>>>(cell_start, moved, counts);
    k_scan_movers<<<1, 1024, 0, s>>>(counts, ntiles, offsets);
    return cudaGetLastError();
}

cudaError_t compact_movers(const SpillArgs &S, cudaStream_t s) {
    k_compact_movers<<<(unsigned)S.ntiles, 256, 0, s>>>(S);
    return cudaGetLastError();
}

}  // namespace polypic

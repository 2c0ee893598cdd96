// p2g.cu -- deterministic particle-to-grid transfer (Eqs 1-5, 13, 15-19).
//
//   m_ia  = sum_p mt_p w_ipa
//   mv_ia = sum_p mt_p w_ipa sum_{r<R} c_pra s_r(x_ia - x_p)
//
// Work decomposition (no float atomics anywhere, so the result is
// bit-identical from run to run):
//   * one CTA per 8x8x4-cell tile, one warp per 4x4x2-cell block of it, one
//     lane per cell.  Particles are in block-interleaved slot order (see
//     sort.cu), so in round r the lanes read the r-th particle of their cell
//     from one contiguous run of slots: coalesced loads, no reduction across
//     lanes;
//   * a lane accumulates its cell's footprint on face grid A in registers:
//     4 x 3 x 3 nodes (the particle's stencil is 3 nodes wide on every axis,
//     but its lowest node along A is cell - 1 or cell), mass and momentum.
//     The mode sum uses sum factorisation with the padded axis contracted
//     last: 81 + 81 + 108 FMA per particle and component for 27 modes;
//   * after the last round the warp adds the 32 cell footprints into its
//     block region in 36 phases (one node offset per phase: distinct cells
//     hit distinct nodes), then the CTA adds its 8 block regions into the
//     tile region in ascending block order and writes it to scratch;
//   * k_p2g_reduce (one CTA per tile, the nodes it owns on the three face
//     grids) sums the at most 8 tile regions covering each node in ascending
//     tile order and writes the grids.
#include <mutex>

#include "p2g_kernel.cuh"

namespace polypic {

constexpr int kP2GWarps = 8;

template <int A> struct Reg {
    static constexpr int X = reg_x(A), Y = reg_y(A), Z = reg_z(A);
};

// Index in block region A of node (ix, iy, iz) relative to the region origin.
template <int A>
__device__ __forceinline__ int region_index(int ix, int iy, int iz) {
    return (iz * Reg<A>::Y + iy) * Reg<A>::X + ix;
}

template <int R, bool AFF = false> constexpr int p2g_smem_bytes() {
    return (kP2GWarps * kRegionFloats + kP2GWarps * kStages * Stage<R, AFF>::NV * 32) * 4;
}
static_assert(p2g_smem_bytes<27>() <= 227 * 1024, "P2G staging exceeds the shared memory of a CTA");

// The rounds of the three component passes form one stream (pass 0 rounds
// 0 .. maxn-1, then pass 1, then pass 2) that flows through the stage ring
// without draining: while a pass finishes and merges, the first rounds of the
// next one are already in flight.  `ia` / `ir` name the next round to issue,
// `sn` / `pn` its slot and particle index (loaded one round ahead).
struct Pipe {
    int ia;
    uint32_t ir, sn, pn;
    int ring;  // stage holding the next round to consume
};

template <int R, int FMT, bool ADJ, bool AFF>
__device__ __forceinline__ void pipe_issue(const P2GArgs &P, Pipe &q, uint32_t bs, uint32_t n_c,
                                           uint32_t maxn, unsigned lt, float *st, int lane) {
    if (q.ia < 3 && n_c > q.ir) {  // q.ia is warp-uniform
        if (q.ia == 0) stage_particle<R, FMT, 0, ADJ, AFF>(P, q.pn, q.sn, st, lane);
        else if (q.ia == 1) stage_particle<R, FMT, 1, ADJ, AFF>(P, q.pn, q.sn, st, lane);
        else stage_particle<R, FMT, 2, ADJ, AFF>(P, q.pn, q.sn, st, lane);
    }
    cp_async_commit();
    if (q.ia < 3 && ++q.ir == maxn) {
        q.ir = 0;
        ++q.ia;
    }
    if (q.ia < 3) {
        q.sn = round_slot(bs, n_c, q.ir, lt);
        q.pn = n_c > q.ir ? P.perm[q.sn] : 0u;
    }
}

template <int R, int FMT, int A, bool ADJ, bool AFF>
__device__ __forceinline__ void p2g_pass(const P2GArgs &P, Pipe &q, uint32_t bs, uint32_t n_c,
                                         uint32_t maxn, int ci, int cj, int ck, int gi, int gj,
                                         int gk, int lane, float *reg, float *stage, bool &bad) {
    using S = Stage<R, AFF>;
    const bool interior = gi >= 1 && gi <= P.g.n[0] - 2 && gj >= 1 && gj <= P.g.n[1] - 2 &&
                          gk >= 1 && gk <= P.g.n[2] - 2;
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
        if (n_c > r) {
            const float px = st[S::kX * 32 + lane], py = st[S::kY * 32 + lane],
                        pz = st[S::kZ * 32 + lane];
            float mt = st[S::kM * 32 + lane];
            if (!ADJ && P.mass_abs) mt += st[S::kMabs * 32 + lane];
            const float v0 = cell_coord(px, P.g.inv_dx), v1 = cell_coord(py, P.g.inv_dx),
                        v2 = cell_coord(pz, P.g.inv_dx);
            // in an interior cell, being in the cell implies the valid region
            const bool ok = (interior || (coord_valid(v0, P.g.n[0]) && coord_valid(v1, P.g.n[1]) &&
                                          coord_valid(v2, P.g.n[2]))) &&
                            (int)floorf(v0) == gi && (int)floorf(v1) == gj && (int)floorf(v2) == gk;
            if (ok) {
                const float vu = A == 0 ? v0 : (A == 1 ? v1 : v2);
                const float vv = A == 0 ? v1 : v0;
                const float vw = A == 2 ? v1 : v2;
                const Axis au = axis_decide(vu, true), av_ = axis_decide(vv, false),
                           aw = axis_decide(vw, false);
                const int cu = A == 0 ? gi : (A == 1 ? gj : gk);
                const int shift = au.base - (cu - 1);
                accumulate<R, FMT, A, ADJ, AFF>(P, st, lane, mt, shift, stencil_1d_scaled(au.t, P.s1, P.s2),
                                           stencil_1d_scaled(av_.t, P.s1, P.s2), stencil_1d_scaled(aw.t, P.s1, P.s2), au.guard,
                                           av_.guard, aw.guard, am, av, au.t, av_.t, aw.t);
            } else {
                bad = true;
            }
        }
        // refill the stage just consumed with the next round of the stream
        pipe_issue<R, FMT, ADJ, AFF>(P, q, bs, n_c, maxn, lt, st, lane);
        q.ring = q.ring + 1 == kStages ? 0 : q.ring + 1;
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
                rm[idx] += am[d][kv][kw];
                rv[idx] += av[d][kv][kw];
                __syncwarp();
            }
}

// All three passes of one block: the prologue fills the ring once.
template <int R, int FMT, bool ADJ, bool AFF>
__device__ __forceinline__ void p2g_block(const P2GArgs &P, uint32_t bs, uint32_t n_c,
                                          uint32_t maxn, int ci, int cj, int ck, int gi, int gj,
                                          int gk, int lane, float *reg, float *stage, bool &bad) {
    const unsigned lt = (1u << lane) - 1u;
    Pipe q;
    q.ia = 0;
    q.ir = 0;
    q.ring = 0;
    q.sn = round_slot(bs, n_c, 0, lt);
    q.pn = n_c > 0 ? P.perm[q.sn] : 0u;
#pragma unroll
    for (int k = 0; k < kStages; ++k)
        pipe_issue<R, FMT, ADJ, AFF>(P, q, bs, n_c, maxn, lt, stage + k * Stage<R, AFF>::NV * 32,
                                     lane);
    p2g_pass<R, FMT, 0, ADJ, AFF>(P, q, bs, n_c, maxn, ci, cj, ck, gi, gj, gk, lane, reg, stage, bad);
    p2g_pass<R, FMT, 1, ADJ, AFF>(P, q, bs, n_c, maxn, ci, cj, ck, gi, gj, gk, lane, reg, stage, bad);
    p2g_pass<R, FMT, 2, ADJ, AFF>(P, q, bs, n_c, maxn, ci, cj, ck, gi, gj, gk, lane, reg, stage, bad);
    cp_async_wait<0>();
}

// Adds block region A of warp w into the tile region (written to dst).
template <int A>
__device__ __forceinline__ void merge_tile(const float *smem_regions, const bool *empty,
                                           float *dst) {
    constexpr int N = TileReg<A>::X * TileReg<A>::Y * TileReg<A>::Z;
    for (int i = threadIdx.x; i < N; i += kP2GWarps * 32) {
        const int lx = i % TileReg<A>::X, ly = (i / TileReg<A>::X) % TileReg<A>::Y,
                  lz = i / (TileReg<A>::X * TileReg<A>::Y);
        float sm = 0.0f, sv = 0.0f;
#pragma unroll
        for (int w = 0; w < kP2GWarps; ++w) {
            if (empty[w]) continue;
            const int bx = lx - 4 * (w & 1), by = ly - 4 * ((w >> 1) & 1), bz = lz - 2 * (w >> 2);
            if (bx < 0 || bx >= Reg<A>::X || by < 0 || by >= Reg<A>::Y || bz < 0 || bz >= Reg<A>::Z)
                continue;
            const float *r = smem_regions + w * kRegionFloats;
            const int idx = region_index<A>(bx, by, bz);
            sm += r[reg_off(A, 0) + idx];
            sv += r[reg_off(A, 1) + idx];
        }
        dst[tile_off(A, 0) + i] = sm;
        dst[tile_off(A, 1) + i] = sv;
    }
}

template <int R, int FMT, bool ADJ, bool AFF>
// 27 modes keep the compiler's register allocation (one CTA per SM measured
// faster); fewer modes fit two CTAs per SM without spills, except the
// per-node evaluation of the affine map.
__global__ void __launch_bounds__(kP2GWarps * 32, (R == 27 || (AFF && R > 4) ? 1 : 2))
    k_p2g_tiles(P2GArgs P) {
    extern __shared__ float smem[];
    __shared__ bool s_empty[kP2GWarps];
    float *s_reg = smem;                                     // [8][kRegionFloats]
    float *s_stage = smem + kP2GWarps * kRegionFloats;        // [8][kStages][NV][32]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t tile = blockIdx.x;
    const bool tile_empty = P.cell_start[tile * 256] == P.cell_start[tile * 256 + 256];
    if (threadIdx.x == 0) P.tile_live[tile] = tile_empty ? 0 : 1;
    if (tile_empty) return;  // CTA-uniform

    const uint32_t b = tile * kP2GWarps + warp;
    const uint32_t k = b * 32 + lane;
    const uint32_t cs0 = P.cell_start[k];
    const uint32_t n_c = P.cell_start[k + 1] - cs0;
    const uint32_t bs = P.cell_start[b * 32];
    const uint32_t maxn = __reduce_max_sync(0xffffffffu, n_c);
    float *reg = s_reg + warp * kRegionFloats;
    float *stage = s_stage + warp * kStages * Stage<R, AFF>::NV * 32;
    if (lane == 0) s_empty[warp] = maxn == 0;
    if (maxn > 0) {
        for (int i = lane; i < kRegionFloats; i += 32) reg[i] = 0.0f;
        __syncwarp();
        int i0, j0, k0;
        block_origin(P.g, b, i0, j0, k0);
        const int ci = lane & 3, cj = (lane >> 2) & 3, ck = lane >> 4;
        const int gi = i0 + ci, gj = j0 + cj, gk = k0 + ck;
        bool bad = false;
        p2g_block<R, FMT, ADJ, AFF>(P, bs, n_c, maxn, ci, cj, ck, gi, gj, gk, lane, reg, stage, bad);
        if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(P.status, kFlagOutOfDomain);
    }
    __syncthreads();
    float *dst = P.scratch + (size_t)tile * kTileFloats;
    merge_tile<0>(s_reg, s_empty, dst);
    merge_tile<1>(s_reg, s_empty, dst);
    merge_tile<2>(s_reg, s_empty, dst);
}

template <int R, int FMT, bool ADJ, bool AFF = false>
static cudaError_t launch_tiles(const P2GArgs &P, int grid, cudaStream_t s) {
    const int smem = p2g_smem_bytes<R, AFF>();
    static int configured_device = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (configured_device != dev) {
        cudaError_t e = cudaFuncSetAttribute(k_p2g_tiles<R, FMT, ADJ, AFF>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        configured_device = dev;
    }
    k_p2g_tiles<R, FMT, ADJ, AFF><<<grid, kP2GWarps * 32, smem, s>>>(P);
    return cudaGetLastError();
}

// Candidate tiles of a node along one axis: node n (owner tile u, tile size
// S, region width Wd, T tiles) lies in the regions of tiles u + o0 and, when
// `two`, u + o0 + 1, with o0 in {-1, 0}.  For candidate c the tile and
// region offsets are separable: `part[c]` = tile offset x tile stride +
// (n - S (u + o) + 1) x region stride, `live[c]` the neighbour index term.
struct AxisCand {
    int part[2], live[2];
    bool ok[2];
};

__device__ __forceinline__ AxisCand axis_cand(int n, int u, int S, int Wd, int T,
                                              int64_t tile_stride, int reg_stride,
                                              int live_stride) {
    // S is 8 or 4: floor division by a power of two (n + 2 - Wd may be < 0)
    const int sh = S == 8 ? 3 : 2;
    const int lo = max(0, (n + 2 - Wd + S - 1) >> sh), hi = min(T - 1, (n + 1) >> sh);
    AxisCand c;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int t = lo + k;
        c.ok[k] = t <= hi;
        c.part[k] = (int)((t - u) * tile_stride) + (n - S * t + 1) * reg_stride;
        c.live[k] = (t - u + 1) * live_stride;
    }
    return c;
}

// Sum over the (at most 8) tile regions covering node (i, j, k) of face grid
// A, in ascending tile order (z, then y, then x); tiles without particles
// wrote nothing and count as 0.  All candidate values are loaded before the
// ordered sum, so a thread has up to 16 loads in flight.  With gv non-NULL it
// also applies the single-phase grid update (v = mv/m, + dt g, walls).
template <int A>
__device__ __forceinline__ void reduce_node(const GridGeom &g, const uint8_t *s_live, int ux,
                                            int uy, int uz, int i, int j, int k,
                                            const float *__restrict__ tile_base,
                                            float *__restrict__ gm, float *__restrict__ gp,
                                            float *__restrict__ gv, float dt, float ga,
                                            bool accumulate, bool any_live) {
    // +0 starts the sum, so it is never -0 and the zeros of unused slots
    // leave it unchanged: the same bits as summing the used tiles alone
    float sm = 0.0f, sv = 0.0f;
    if (any_live) {  // CTA-uniform: no tile around this one holds particles otherwise
        constexpr int X = tile_x(A), Y = tile_y(A), Z = tile_z(A);
        const int64_t F = kTileFloats;
        const AxisCand cx = axis_cand(i, ux, 8, X, g.tiles[0], F, 1, 1);
        const AxisCand cy = axis_cand(j, uy, 8, Y, g.tiles[1], F * g.tiles[0], X, 3);
        const AxisCand cz = axis_cand(k, uz, 4, Z, g.tiles[2], F * g.tiles[0] * g.tiles[1], X * Y, 9);
        float m[8], v[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int az = c >> 2, ay = (c >> 1) & 1, ax = c & 1;
            m[c] = v[c] = 0.0f;
            if (cz.ok[az] && cy.ok[ay] && cx.ok[ax] &&
                s_live[cz.live[az] + cy.live[ay] + cx.live[ax]]) {
                const float *src = tile_base + (cz.part[az] + cy.part[ay] + cx.part[ax]);
                m[c] = __ldg(src + tile_off(A, 0));
                v[c] = __ldg(src + tile_off(A, 1));
            }
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            sm += m[c];
            sv += v[c];
        }
    }
    const int dX = g.n[0] + (A == 0), dY = g.n[1] + (A == 1);
    const int64_t idx = ((int64_t)k * dY + j) * dX + i;
    if (gm) gm[idx] = sm;
    gp[idx] = accumulate ? gp[idx] + sv : sv;
    if (gv) {
        const int ia = A == 0 ? i : (A == 1 ? j : k);
        float vel = sm > 0.0f ? sv / sm : 0.0f;
        vel = fmaf(dt, ga, vel);
        gv[idx] = (ia == 0 || ia == g.n[A]) ? 0.0f : vel;
    }
}

// One CTA per key tile writes the nodes the tile owns on all three face
// grids: [8tx, 8tx + 8) x [8ty, 8ty + 8) x [4tz, 4tz + 4), the last tile
// along axis A also the wall layer n[A] of face grid A.  Thread (lx, ly, lz)
// takes one owned node per face; the owned nodes only draw on the 27 tiles
// around this one, whose live flags are staged first.
struct ReduceOut {
    float *gm[3], *gp[3], *gv[3];
    float ga[3];
};

__global__ void __launch_bounds__(256) k_p2g_reduce(GridGeom g, const uint8_t *__restrict__ live,
                                                    const float *__restrict__ scratch,
                                                    ReduceOut O, float dt, bool accumulate) {
    __shared__ uint8_t s_live[27];
    const uint32_t tile = blockIdx.x;
    const int ux = (int)(tile % (uint32_t)g.tiles[0]);
    const int uy = (int)((tile / (uint32_t)g.tiles[0]) % (uint32_t)g.tiles[1]);
    const int uz = (int)(tile / ((uint32_t)g.tiles[0] * (uint32_t)g.tiles[1]));
    const int t = threadIdx.x;
    if (t < 27) {
        const int vz = uz + t / 9 - 1, vy = uy + (t / 3) % 3 - 1, vx = ux + t % 3 - 1;
        const bool in = vx >= 0 && vx < g.tiles[0] && vy >= 0 && vy < g.tiles[1] && vz >= 0 &&
                        vz < g.tiles[2];
        s_live[t] = in ? live[((uint32_t)vz * g.tiles[1] + vy) * g.tiles[0] + vx] : 0;
    }
    const bool any_live = __syncthreads_or(t < 27 && s_live[t]);
    const int i = 8 * ux + (t & 7), j = 8 * uy + ((t >> 3) & 7), k = 4 * uz + (t >> 6);
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    // candidate offsets are relative to the owner tile, within +-1 tile of it
    scratch += (size_t)tile * kTileFloats;
    // a tile at the grid's upper edge may extend past the cells (n not a
    // multiple of the tile): nodes beyond the face grid are not written
    if (i < nx + 1 && j < ny && k < nz)
        reduce_node<0>(g, s_live, ux, uy, uz, i, j, k, scratch, O.gm[0], O.gp[0], O.gv[0], dt,
                       O.ga[0], accumulate, any_live);
    if (i < nx && j < ny + 1 && k < nz)
        reduce_node<1>(g, s_live, ux, uy, uz, i, j, k, scratch, O.gm[1], O.gp[1], O.gv[1], dt,
                       O.ga[1], accumulate, any_live);
    if (i < nx && j < ny && k < nz + 1)
        reduce_node<2>(g, s_live, ux, uy, uz, i, j, k, scratch, O.gm[2], O.gp[2], O.gv[2], dt,
                       O.ga[2], accumulate, any_live);
    // the wall layer n[A] lies one past the last tile when the tile size
    // divides n[A]: 8 x 4, 8 x 4 and 8 x 8 more nodes
    const int i8 = 8 * ux + (t & 7), j8 = 8 * uy + (t & 7);   // t < 32: 8 x 4
    const int k4 = 4 * uz + (t >> 3), j64 = 8 * uy + (t >> 3);  // t < 64: 8 x 8
    if (ux == g.tiles[0] - 1 && 8 * g.tiles[0] == nx && t < 32 && j8 < ny && k4 < nz)
        reduce_node<0>(g, s_live, ux, uy, uz, nx, j8, k4, scratch, O.gm[0], O.gp[0], O.gv[0],
                       dt, O.ga[0], accumulate, any_live);
    if (uy == g.tiles[1] - 1 && 8 * g.tiles[1] == ny && t < 32 && i8 < nx && k4 < nz)
        reduce_node<1>(g, s_live, ux, uy, uz, i8, ny, k4, scratch, O.gm[1], O.gp[1], O.gv[1], dt,
                       O.ga[1], accumulate, any_live);
    if (uz == g.tiles[2] - 1 && 4 * g.tiles[2] == nz && t < 64 && i8 < nx && j64 < ny)
        reduce_node<2>(g, s_live, ux, uy, uz, i8, j64, nz, scratch, O.gm[2], O.gp[2], O.gv[2], dt,
                       O.ga[2], accumulate, any_live);
}

// ---------------------------------------------------------------- built-in scratch
// For callers that cannot hand the library a workspace (see
// polypic_p2g_noalloc): the tile regions and live flags live in fixed-size
// device arrays that every GPU loading the library holds until the process
// exits.  Host code must not pass these names to a kernel (on the host they
// are stand-ins, not device addresses); p2g_builtin_scratch() looks the
// device addresses up once per device with cudaGetSymbolAddress.
constexpr int kBuiltinTiles = 2048;
static __device__ __align__(256) float g_builtin_tiles[(size_t)kBuiltinTiles * kTileFloats];
static __device__ __align__(256) uint8_t g_builtin_live[kBuiltinTiles];

int p2g_builtin_max_tiles() { return kBuiltinTiles; }

cudaError_t p2g_builtin_scratch(float **tiles, uint8_t **live) {
    constexpr int kMaxDevices = 64;
    static std::mutex mu;
    static bool ready[kMaxDevices] = {};
    static float *tile_ptr[kMaxDevices] = {};
    static uint8_t *live_ptr[kMaxDevices] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (!ready[dev]) {
        void *t = nullptr, *l = nullptr;
        if ((e = cudaGetSymbolAddress(&t, g_builtin_tiles)) != cudaSuccess) return e;
        if ((e = cudaGetSymbolAddress(&l, g_builtin_live)) != cudaSuccess) return e;
        tile_ptr[dev] = static_cast<float *>(t);
        live_ptr[dev] = static_cast<uint8_t *>(l);
        ready[dev] = true;
    }
    *tiles = tile_ptr[dev];
    *live = live_ptr[dev];
    return cudaSuccess;
}

size_t p2g_scratch_bytes(int64_t num_keys) {
    return (size_t)(num_keys / 256) * (kTileFloats * sizeof(float) + 1) + 512;
}

static cudaError_t reduce_tiles(const P2GArgs &P, float *gm[3], float *gp[3], float *gv[3],
                                float dt, const float gravity[3], bool accumulate, cudaStream_t s) {
    ReduceOut O;
    for (int a = 0; a < 3; ++a) {
        O.gm[a] = gm ? gm[a] : nullptr;
        O.gp[a] = gp[a];
        O.gv[a] = gv ? gv[a] : nullptr;
        O.ga[a] = gravity ? gravity[a] : 0.0f;
    }
    const int ntiles = (int)(P.nblocks / kP2GWarps);
    k_p2g_reduce<<<ntiles, 256, 0, s>>>(P.g, P.tile_live, P.scratch, O, dt, accumulate);
    return cudaGetLastError();
}

cudaError_t p2g_adjoint_scatter(const P2GArgs &P, float *lv[3], bool accumulate, int R,
                                cudaStream_t s) {
    const int grid = (int)(P.nblocks / kP2GWarps);
    cudaError_t e = cudaErrorInvalidValue;
    if (R == 1) e = launch_tiles<1, POLYPIC_COEFF_F32, true>(P, grid, s);
    if (R == 4) e = launch_tiles<4, POLYPIC_COEFF_F32, true>(P, grid, s);
    if (R == 8) e = launch_tiles<8, POLYPIC_COEFF_F32, true>(P, grid, s);
    if (R == 27) e = launch_tiles<27, POLYPIC_COEFF_F32, true>(P, grid, s);
    if (e != cudaSuccess) return e;
    return reduce_tiles(P, nullptr, lv, nullptr, 0.0f, nullptr, accumulate, s);
}

cudaError_t p2g(const P2GArgs &P, float *gm[3], float *gp[3], float *gv[3], float dt,
                const float gravity[3], int R, int fmt, cudaStream_t s, bool ordered) {
    const int grid = (int)(P.nblocks / kP2GWarps);
    if (ordered) {
        const cudaError_t e = launch_p2g_ordered(P, R, fmt, grid, s);
        if (e != cudaSuccess) return e;
        return reduce_tiles(P, gm, gp, gv, dt, gravity, false, s);
    }
    cudaError_t e = cudaErrorInvalidValue;
    if (P.affine) {  // Eq 12's affine map: FP32 coefficients, 4, 8 or 27 modes
        if (fmt != POLYPIC_COEFF_F32) return cudaErrorInvalidValue;
        if (R == 4) e = launch_tiles<4, POLYPIC_COEFF_F32, false, true>(P, grid, s);
        else if (R == 8) e = launch_tiles<8, POLYPIC_COEFF_F32, false, true>(P, grid, s);
        else if (R == 27) e = launch_tiles<27, POLYPIC_COEFF_F32, false, true>(P, grid, s);
        if (e != cudaSuccess) return e;
        return reduce_tiles(P, gm, gp, gv, dt, gravity, false, s);
    }
#define POLYPIC_P2G_CASE(RR, FF) \
    if (R == RR && fmt == FF) e = launch_tiles<RR, FF, false>(P, grid, s);
    POLYPIC_P2G_CASE(1, POLYPIC_COEFF_F32)
    POLYPIC_P2G_CASE(4, POLYPIC_COEFF_F32)
    POLYPIC_P2G_CASE(8, POLYPIC_COEFF_F32)
    POLYPIC_P2G_CASE(27, POLYPIC_COEFF_F32)
    POLYPIC_P2G_CASE(1, POLYPIC_COEFF_BF16)
    POLYPIC_P2G_CASE(4, POLYPIC_COEFF_BF16)
    POLYPIC_P2G_CASE(8, POLYPIC_COEFF_BF16)
    POLYPIC_P2G_CASE(27, POLYPIC_COEFF_BF16)
    POLYPIC_P2G_CASE(1, POLYPIC_COEFF_F16)
    POLYPIC_P2G_CASE(4, POLYPIC_COEFF_F16)
    POLYPIC_P2G_CASE(8, POLYPIC_COEFF_F16)
    POLYPIC_P2G_CASE(27, POLYPIC_COEFF_F16)
#undef POLYPIC_P2G_CASE
    if (e != cudaSuccess) return e;
    return reduce_tiles(P, gm, gp, gv, dt, gravity, false, s);
}

}  // namespace polypic

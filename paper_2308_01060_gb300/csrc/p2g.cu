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
#include <cuda.h>

#include <mutex>

#include "p2g_tiles.cuh"

namespace polypic {

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
    if (gm) gm[idx] = accumulate ? gm[idx] + sm : sm;
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
// device addresses up with cudaGetSymbolAddress.  The address belongs to the
// copy of the module loaded in the current CUDA context, so it is cached per
// context (the driver's cuCtxGetCurrent) and looked up again on every call
// made outside a stream capture, which also covers a context that was torn
// down and recreated (cudaDeviceReset) under the same handle.  During a
// capture only the cached address is used.
constexpr int kBuiltinTiles = 2048;
static __device__ __align__(256) float g_builtin_tiles[(size_t)kBuiltinTiles * kTileFloats];
static __device__ __align__(256) uint8_t g_builtin_live[kBuiltinTiles];

int p2g_builtin_max_tiles() { return kBuiltinTiles; }

namespace {
using CtxGetCurrentFn = CUresult (*)(CUcontext *);

// cuCtxGetCurrent through the runtime's driver entry point (no link-time
// dependency on libcuda); nullptr if the driver does not provide it.
CtxGetCurrentFn ctx_get_current() {
    static CtxGetCurrentFn fn = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return reinterpret_cast<CtxGetCurrentFn>(f);
    }();
    return fn;
}

struct BuiltinEntry {
    CUcontext ctx;
    float *tiles;
    uint8_t *live;
};
}  // namespace

cudaError_t p2g_builtin_scratch(cudaStream_t s, float **tiles, uint8_t **live) {
    constexpr int kEntries = 64;
    static std::mutex mu;
    static BuiltinEntry cache[kEntries] = {};
    static int used = 0, next = 0;
    // the runtime call first: it makes the device's context current
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess) return e;
    CUcontext ctx = nullptr;
    const CtxGetCurrentFn get = ctx_get_current();
    if (get && get(&ctx) != CUDA_SUCCESS) return cudaErrorContextIsDestroyed;
    std::lock_guard<std::mutex> lock(mu);
    int hit = -1;
    for (int i = 0; i < used; ++i)
        if (cache[i].ctx == ctx) hit = i;
    if (cap == cudaStreamCaptureStatusNone || hit < 0 || !get) {
        if (cap != cudaStreamCaptureStatusNone) return cudaErrorStreamCaptureUnsupported;
        void *t = nullptr, *l = nullptr;
        if ((e = cudaGetSymbolAddress(&t, g_builtin_tiles)) != cudaSuccess) return e;
        if ((e = cudaGetSymbolAddress(&l, g_builtin_live)) != cudaSuccess) return e;
        if (hit < 0) {
            hit = used < kEntries ? used++ : next;
            next = (hit + 1) % kEntries;
        }
        cache[hit] = BuiltinEntry{ctx, static_cast<float *>(t), static_cast<uint8_t *>(l)};
    }
    *tiles = cache[hit].tiles;
    *live = cache[hit].live;
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
    const cudaError_t e = launch_tiles_adj(P, R, grid, s);
    if (e != cudaSuccess) return e;
    return reduce_tiles(P, nullptr, lv, nullptr, 0.0f, nullptr, accumulate, s);
}

cudaError_t p2g(const P2GArgs &P, float *gm[3], float *gp[3], float *gv[3], float dt,
                const float gravity[3], int R, int fmt, cudaStream_t s) {
    const int grid = (int)(P.nblocks / kP2GWarps);
    cudaError_t e;
    if (P.affine) {  // Eq 12's affine map: FP32 coefficients, 4, 8 or 27 modes
        if (fmt != POLYPIC_COEFF_F32) return cudaErrorInvalidValue;
        e = launch_tiles_aff(P, R, grid, s);
    } else if (fmt == POLYPIC_COEFF_F32) {
        // a solid phase (a sheet) crosses a block in few of its cells: lane teams
        e = P.mass_abs ? launch_tiles_teams(P, R, grid, s) : launch_tiles_f32(P, R, grid, s);
    } else {
        e = launch_tiles_16(P, R, fmt, grid, s);
    }
    if (e != cudaSuccess) return e;
    return reduce_tiles(P, gm, gp, gv, dt, gravity, false, s);
}

cudaError_t p2g_reduce(const P2GArgs &P, float *gm[3], float *gp[3], bool accumulate,
                       cudaStream_t s) {
    return reduce_tiles(P, gm, gp, nullptr, 0.0f, nullptr, accumulate, s);
}

cudaError_t p2g_accumulate(const P2GArgs &P, float *gm[3], float *gp[3], int R, cudaStream_t s) {
    const int grid = (int)(P.nblocks / kP2GWarps);
    const cudaError_t e = launch_tiles_f32(P, R, grid, s);
    if (e != cudaSuccess) return e;
    return reduce_tiles(P, gm, gp, nullptr, 0.0f, nullptr, true, s);
}

}  // namespace polypic

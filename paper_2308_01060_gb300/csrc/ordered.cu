// ordered.cu -- kernels of ordered phases (Eqs 6-8, Section 3.3): particle
// arrays kept in their own slot order (tile_order.cuh), so that P2G reads
// each round of a warp as one contiguous run and its lanes hold cells of
// similar population.
//
// A step on an ordered phase cannot write G2P's outputs in the order P2G
// will read next unless it knows that order first, so the step advects
// before it fits:
//   k_advect       tile by tile in the current order: the PIC velocity
//                  v_p = c_p0 (the G2P fit restricted to mode 0), the new
//                  position, its key, and a count with arrival rank (the key
//                  producer of the next order);
//   (sort)         finish_order() turns the counts into the next order;
//   k_g2p_ordered  tile by tile in the NEXT order: gathers each particle's
//                  old position, fits all modes there from a footprint staged
//                  with a one-cell halo, advects again with the velocity mode
//                  (bit-identical to k_advect's: same arithmetic, same nodes),
//                  writes every output contiguously;
//   k_g2p_far      the particles that moved more than a cell out of their new
//                  tile, fitted from the grid itself;
//   k_gather       copies a phase into a given order (to order a phase once).
#include "ordered.cuh"

#include "g2p_fit.cuh"

namespace polypic {

// ---------------------------------------------------------------- advection
__global__ void __launch_bounds__(kG2PThreads) k_advect(AdvectArgs A) {
    __shared__ float s_tile[kVelTileFloats];
    const GridGeom &g = A.g;
    const uint32_t tile = blockIdx.x;
    if (tile == 0 && threadIdx.x == 0) {
        *A.num_crowded = 0;
        *A.num_far = 0;
    }
    const uint32_t jb = A.cell_start[tile * 256], je = A.cell_start[tile * 256 + 256];
    if (jb == je) return;  // CTA-uniform
    const int tx = (int)(tile % (uint32_t)g.tiles[0]);
    const int ty = (int)((tile / (uint32_t)g.tiles[0]) % (uint32_t)g.tiles[1]);
    const int tz = (int)(tile / ((uint32_t)g.tiles[0] * (uint32_t)g.tiles[1]));
    const int ox = 8 * tx - 1, oy = 8 * ty - 1, oz = 4 * tz - 1;
    stage_velocity<0>(g, A.vel, tx, ty, tz, s_tile);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    for (uint32_t j0 = jb; j0 < je; j0 += kG2PThreads) {  // CTA-uniform: whole warps below
        const uint32_t j = j0 + threadIdx.x;
        const bool live = j < je;
        float px = 0.0f, py = 0.0f, pz = 0.0f;
        if (live) {
            px = A.x[j];
            py = A.y[j];
            pz = A.z[j];
        }
        const float v0 = cell_coord(px, g.inv_dx), v1 = cell_coord(py, g.inv_dx),
                    v2 = cell_coord(pz, g.inv_dx);
        bool ok = coord_valid(v0, g.n[0]) && coord_valid(v1, g.n[1]) && coord_valid(v2, g.n[2]);
        const int ci = cell_index(v0, g.n[0]) - 8 * tx, cj = cell_index(v1, g.n[1]) - 8 * ty,
                  ck = cell_index(v2, g.n[2]) - 4 * tz;
        ok = live && ok && ci >= 0 && ci < 8 && cj >= 0 && cj < 8 && ck >= 0 && ck < 4;
        float vel[3] = {0.0f, 0.0f, 0.0f};
        if (ok) {
            const Axis ac0 = axis_decide(v0, false), af0 = axis_decide(v0, true);
            const Axis ac1 = axis_decide(v1, false), af1 = axis_decide(v1, true);
            const Axis ac2 = axis_decide(v2, false), af2 = axis_decide(v2, true);
            const Stencil1D sc0 = stencil_1d(ac0.t), sf0 = stencil_1d(af0.t);
            const Stencil1D sc1 = stencil_1d(ac1.t), sf1 = stencil_1d(af1.t);
            const Stencil1D sc2 = stencil_1d(ac2.t), sf2 = stencil_1d(af2.t);
            float c[1];
            g2p_component<1, 0, Tile<0>::X, Tile<0>::Y>(s_tile, af0.base - ox, ac1.base - oy,
                                                        ac2.base - oz, sf0, af0.guard, sc1,
                                                        ac1.guard, sc2, ac2.guard, 1.0f, 1.0f, c);
            vel[0] = c[0];
            g2p_component<1, 1, Tile<1>::X, Tile<1>::Y>(s_tile + kVelTileOff1, ac0.base - ox,
                                                        af1.base - oy, ac2.base - oz, sc0,
                                                        ac0.guard, sf1, af1.guard, sc2,
                                                        ac2.guard, 1.0f, 1.0f, c);
            vel[1] = c[0];
            g2p_component<1, 2, Tile<2>::X, Tile<2>::Y>(s_tile + kVelTileOff2, ac0.base - ox,
                                                        ac1.base - oy, af2.base - oz, sc0,
                                                        ac0.guard, sc1, ac1.guard, sf2,
                                                        af2.guard, 1.0f, 1.0f, c);
            vel[2] = c[0];
        }
        if (live && !ok) atomicOr(A.status, kFlagOutOfDomain);
        const float nx = ok ? fminf(fmaxf(fmaf(A.dt, vel[0], px), g.lo[0]), g.hi[0]) : px;
        const float ny = ok ? fminf(fmaxf(fmaf(A.dt, vel[1], py), g.lo[1]), g.hi[1]) : py;
        const float nz = ok ? fminf(fmaxf(fmaf(A.dt, vel[2], pz), g.lo[2]), g.hi[2]) : pz;
        const float w0 = cell_coord(nx, g.inv_dx), w1 = cell_coord(ny, g.inv_dx),
                    w2 = cell_coord(nz, g.inv_dx);
        const uint32_t k =
            cell_key(g, cell_index(w0, g.n[0]), cell_index(w1, g.n[1]), cell_index(w2, g.n[2]));
        if (live) A.key[j] = k;
        // count with arrival rank, warp-aggregated
        const unsigned active = __ballot_sync(0xffffffffu, live);
        if (live) {
            const unsigned peers = __match_any_sync(active, k);
            const int leader = __ffs(peers) - 1;
            uint32_t old = 0;
            if (lane == leader) old = atomicAdd(&A.counts[k], (uint32_t)__popc(peers));
            old = __shfl_sync(active, old, leader);
            A.rank[j] = old + (uint32_t)__popc(peers & lt);
        }
    }
}

cudaError_t advect(const AdvectArgs &A, int64_t num_tiles, cudaStream_t s) {
    k_advect<<<(unsigned)num_tiles, kG2PThreads, 0, s>>>(A);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- G2P
// Fit of a particle whose footprint is not staged: the 27 nodes of each
// component are read from the grids (nodes outside a grid count as 0).
template <int R>
__device__ __forceinline__ void fit_from_grid(const GridGeom &g, const float *const vel[3],
                                              const Axis *ac, const Axis *af, float inv1,
                                              float inv2, float (&Chat)[3][R]) {
    Stencil1D sc[3], sf[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        sc[b] = stencil_1d(ac[b].t);
        sf[b] = stencil_1d(af[b].t);
    }
    float loc[27];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int dX = g.n[0] + (a == 0), dY = g.n[1] + (a == 1), dZ = g.n[2] + (a == 2);
        const int bx = a == 0 ? af[0].base : ac[0].base;
        const int by = a == 1 ? af[1].base : ac[1].base;
        const int bz = a == 2 ? af[2].base : ac[2].base;
#pragma unroll
        for (int kz = 0; kz < 3; ++kz)
#pragma unroll
            for (int ky = 0; ky < 3; ++ky)
#pragma unroll
                for (int kx = 0; kx < 3; ++kx) {
                    const int gx = bx + kx, gy = by + ky, gz = bz + kz;
                    float v = 0.0f;
                    if (gx >= 0 && gx < dX && gy >= 0 && gy < dY && gz >= 0 && gz < dZ)
                        v = vel[a][((int64_t)gz * dY + gy) * dX + gx];
                    loc[(kz * 3 + ky) * 3 + kx] = v;
                }
        if (a == 0)
            g2p_component<R, 0, 3, 3>(loc, 0, 0, 0, sf[0], af[0].guard, sc[1], ac[1].guard, sc[2],
                                      ac[2].guard, inv1, inv2, Chat[0]);
        else if (a == 1)
            g2p_component<R, 1, 3, 3>(loc, 0, 0, 0, sc[0], ac[0].guard, sf[1], af[1].guard, sc[2],
                                      ac[2].guard, inv1, inv2, Chat[1]);
        else
            g2p_component<R, 2, 3, 3>(loc, 0, 0, 0, sc[0], ac[0].guard, sc[1], ac[1].guard, sf[2],
                                      af[2].guard, inv1, inv2, Chat[2]);
    }
}

// Outputs of slot j of the next order from the fit Chat at the old
// position (px, py, pz) (shared by the two G2P kernels of ordered phases).
template <int R, int FMT>
__device__ __forceinline__ void write_slot(const OrderedG2PArgs &A, uint32_t j, uint32_t p,
                                           bool ok, float px, float py, float pz, float m,
                                           float mabs, const float (&Chat)[3][R]) {
    using T = typename Codec<FMT>::T;
    const int64_t cnt = A.count;
    T *out = reinterpret_cast<T *>(A.ocoeff) + j;  // row (a, r) starts (a R + r) * cnt in
    if constexpr (FMT == POLYPIC_COEFF_F32) {
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int r = 0; r < R; ++r, out += cnt) *out = Chat[a][r];
    } else {
        float sc = 0.0f;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int r = 0; r < R; ++r) sc = fmaxf(sc, fabsf(Chat[a][r]));
        const float inv = sc > 0.0f ? 1.0f / sc : 0.0f;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int r = 0; r < R; ++r, out += cnt) *out = Codec<FMT>::encode(Chat[a][r] * inv);
        A.oscale[j] = sc;
    }
    // advection with the velocity mode, as k_advect did, and its key
    const GridGeom &g = A.g;
    A.ox[j] = ok ? fminf(fmaxf(fmaf(A.dt, Chat[0][0], px), g.lo[0]), g.hi[0]) : px;
    A.oy[j] = ok ? fminf(fmaxf(fmaf(A.dt, Chat[1][0], py), g.lo[1]), g.hi[1]) : py;
    A.oz[j] = ok ? fminf(fmaxf(fmaf(A.dt, Chat[2][0], pz), g.lo[2]), g.hi[2]) : pz;
    A.okey[j] = A.key_new[p];
    A.omass[j] = m;
    if (A.omass_abs) A.omass_abs[j] = mabs;
}

template <int R, int FMT>
__global__ void __launch_bounds__(kG2PThreads) k_g2p_ordered(OrderedG2PArgs A) {
    using S1 = Shape<1>;
    __shared__ float s_tile[S1::kFloats];
    const GridGeom &g = A.g;
    const uint32_t tile = blockIdx.x;  // a tile of the NEXT order
    const uint32_t jb = A.cell_start[tile * 256], je = A.cell_start[tile * 256 + 256];
    if (jb == je) return;  // CTA-uniform
    const int tx = (int)(tile % (uint32_t)g.tiles[0]);
    const int ty = (int)((tile / (uint32_t)g.tiles[0]) % (uint32_t)g.tiles[1]);
    const int tz = (int)(tile / ((uint32_t)g.tiles[0] * (uint32_t)g.tiles[1]));
    const int ox = 8 * tx - 2, oy = 8 * ty - 2, oz = 4 * tz - 2;  // halo of one cell

    // first particle's loads go out before the tile staging and its barrier
    uint32_t j = jb + threadIdx.x;
    uint32_t p = 0;
    float px = 0.0f, py = 0.0f, pz = 0.0f, m = 0.0f, mabs = 0.0f;
    if (j < je) {
        p = A.perm[j];
        px = A.x[p]; py = A.y[p]; pz = A.z[p]; m = A.mass[p];
        if (A.mass_abs) mabs = A.mass_abs[p];
    }
    uint32_t pn = (j + kG2PThreads < je) ? A.perm[j + kG2PThreads] : 0u;
    stage_velocity<1>(g, A.vel, tx, ty, tz, s_tile);
    __syncthreads();

    // FP32 output is physical (c = c dx^L / dx^L); the 16-bit codes take c dx^L
    const float inv1 = FMT == POLYPIC_COEFF_F32 ? A.inv_dxpow[1] : 1.0f;
    const float inv2 = FMT == POLYPIC_COEFF_F32 ? A.inv_dxpow[2] : 1.0f;
    for (; j < je; j += kG2PThreads) {
        // software pipeline: the next particle's data, and the index after it
        const uint32_t jn = j + kG2PThreads;
        float nx = 0.0f, ny = 0.0f, nz = 0.0f, nm = 0.0f, nmabs = 0.0f;
        uint32_t pnn = 0;
        if (jn < je) {
            nx = A.x[pn]; ny = A.y[pn]; nz = A.z[pn]; nm = A.mass[pn];
            if (A.mass_abs) nmabs = A.mass_abs[pn];
            if (jn + kG2PThreads < je) pnn = A.perm[jn + kG2PThreads];
        }
        const float v0 = cell_coord(px, g.inv_dx), v1 = cell_coord(py, g.inv_dx),
                    v2 = cell_coord(pz, g.inv_dx);
        const bool ok =
            coord_valid(v0, g.n[0]) && coord_valid(v1, g.n[1]) && coord_valid(v2, g.n[2]);
        // old cell relative to the halo's lowest cell: staged when in [0,10) x [0,10) x [0,6)
        const int hi = cell_index(v0, g.n[0]) - (8 * tx - 1);
        const int hj = cell_index(v1, g.n[1]) - (8 * ty - 1);
        const int hk = cell_index(v2, g.n[2]) - (4 * tz - 1);
        const bool staged = ok && hi >= 0 && hi < 10 && hj >= 0 && hj < 10 && hk >= 0 && hk < 6;
        // a particle that moved more than a cell out of this tile is fitted
        // from the grid by k_g2p_far
        const bool far = ok && !staged;
        if (far) A.far[atomicAdd(A.num_far, 1u)] = j;
        float Chat[3][R];
        if (staged) {
            const Axis ac0 = axis_decide(v0, false), af0 = axis_decide(v0, true);
            const Axis ac1 = axis_decide(v1, false), af1 = axis_decide(v1, true);
            const Axis ac2 = axis_decide(v2, false), af2 = axis_decide(v2, true);
            const Stencil1D sc0 = stencil_1d(ac0.t), sf0 = stencil_1d(af0.t);
            const Stencil1D sc1 = stencil_1d(ac1.t), sf1 = stencil_1d(af1.t);
            const Stencil1D sc2 = stencil_1d(ac2.t), sf2 = stencil_1d(af2.t);
            g2p_component<R, 0, S1::D<0>::X, S1::D<0>::Y>(
                s_tile, af0.base - ox, ac1.base - oy, ac2.base - oz, sf0, af0.guard, sc1,
                ac1.guard, sc2, ac2.guard, inv1, inv2, Chat[0]);
            g2p_component<R, 1, S1::D<1>::X, S1::D<1>::Y>(
                s_tile + S1::kOff1, ac0.base - ox, af1.base - oy, ac2.base - oz, sc0, ac0.guard,
                sf1, af1.guard, sc2, ac2.guard, inv1, inv2, Chat[1]);
            g2p_component<R, 2, S1::D<2>::X, S1::D<2>::Y>(
                s_tile + S1::kOff2, ac0.base - ox, ac1.base - oy, af2.base - oz, sc0, ac0.guard,
                sc1, ac1.guard, sf2, af2.guard, inv1, inv2, Chat[2]);
        } else {
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int r = 0; r < R; ++r) Chat[a][r] = 0.0f;
        }
        if (!far) {
            if (!ok) atomicOr(A.status, kFlagOutOfDomain);
            const bool finite =
                isfinite(Chat[0][0]) && isfinite(Chat[1][0]) && isfinite(Chat[2][0]);
            if (!finite) atomicOr(A.status, kFlagNonFinite);
            write_slot<R, FMT>(A, j, p, ok, px, py, pz, m, mabs, Chat);
        }
        px = nx; py = ny; pz = nz; m = nm; mabs = nmabs; p = pn; pn = pnn;
    }
}

// Particles listed by k_g2p_ordered: the fit from the grid itself.
// Launched with a fixed grid; it exits at once when the list is empty.
template <int R, int FMT>
__global__ void __launch_bounds__(128) k_g2p_far(OrderedG2PArgs A) {
    const uint32_t nfar = *A.num_far;
    const float inv1 = FMT == POLYPIC_COEFF_F32 ? A.inv_dxpow[1] : 1.0f;
    const float inv2 = FMT == POLYPIC_COEFF_F32 ? A.inv_dxpow[2] : 1.0f;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nfar;
         i += gridDim.x * blockDim.x) {
        const uint32_t j = A.far[i], p = A.perm[j];
        const float px = A.x[p], py = A.y[p], pz = A.z[p];
        const float v0 = cell_coord(px, A.g.inv_dx), v1 = cell_coord(py, A.g.inv_dx),
                    v2 = cell_coord(pz, A.g.inv_dx);
        const Axis ac[3] = {axis_decide(v0, false), axis_decide(v1, false),
                            axis_decide(v2, false)};
        const Axis af[3] = {axis_decide(v0, true), axis_decide(v1, true), axis_decide(v2, true)};
        float Chat[3][R];
        fit_from_grid<R>(A.g, A.vel, ac, af, inv1, inv2, Chat);
        const bool finite = isfinite(Chat[0][0]) && isfinite(Chat[1][0]) && isfinite(Chat[2][0]);
        if (!finite) atomicOr(A.status, kFlagNonFinite);
        write_slot<R, FMT>(A, j, p, true, px, py, pz, A.mass[p],
                           A.mass_abs ? A.mass_abs[p] : 0.0f, Chat);
    }
}

cudaError_t g2p_ordered(const OrderedG2PArgs &A, int64_t num_tiles, int R, int fmt,
                        cudaStream_t s) {
    const unsigned grid = (unsigned)num_tiles;
#define POLYPIC_G2PO_CASE(RR, FF)                               \
    if (R == RR && fmt == FF) {                                \
        k_g2p_ordered<RR, FF><<<grid, kG2PThreads, 0, s>>>(A); \
        k_g2p_far<RR, FF><<<152, 128, 0, s>>>(A);              \
        return cudaGetLastError();                             \
    }
    POLYPIC_G2PO_CASE(1, POLYPIC_COEFF_F32)
    POLYPIC_G2PO_CASE(4, POLYPIC_COEFF_F32)
    POLYPIC_G2PO_CASE(8, POLYPIC_COEFF_F32)
    POLYPIC_G2PO_CASE(27, POLYPIC_COEFF_F32)
    POLYPIC_G2PO_CASE(1, POLYPIC_COEFF_BF16)
    POLYPIC_G2PO_CASE(4, POLYPIC_COEFF_BF16)
    POLYPIC_G2PO_CASE(8, POLYPIC_COEFF_BF16)
    POLYPIC_G2PO_CASE(27, POLYPIC_COEFF_BF16)
    POLYPIC_G2PO_CASE(1, POLYPIC_COEFF_F16)
    POLYPIC_G2PO_CASE(4, POLYPIC_COEFF_F16)
    POLYPIC_G2PO_CASE(8, POLYPIC_COEFF_F16)
    POLYPIC_G2PO_CASE(27, POLYPIC_COEFF_F16)
#undef POLYPIC_G2PO_CASE
    return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------- gather
template <typename E>
__global__ void __launch_bounds__(256) k_gather(GatherArgs A) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= A.count) return;
    const uint32_t p = A.perm[j];
    for (int a = 0; a < 3; ++a) A.ox[a][j] = A.x[a][p];
    A.omass[j] = A.mass[p];
    if (A.omass_abs) A.omass_abs[j] = A.mass_abs ? A.mass_abs[p] : 0.0f;
    if (A.oscale) A.oscale[j] = A.scale ? A.scale[p] : 0.0f;
    if (A.okey) A.okey[j] = A.key[p];
    const E *c = static_cast<const E *>(A.coeff);
    E *o = static_cast<E *>(A.ocoeff);
    for (int r = 0; r < A.rows; ++r) o[(int64_t)r * A.count + j] = c[(int64_t)r * A.count + p];
}

cudaError_t gather_phase(const GatherArgs &A, cudaStream_t s) {
    if (A.count == 0) return cudaSuccess;
    const unsigned grid = (unsigned)((A.count + 255) / 256);
    if (A.elem == 4) k_gather<uint32_t><<<grid, 256, 0, s>>>(A);
    else if (A.elem == 2) k_gather<uint16_t><<<grid, 256, 0, s>>>(A);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace polypic

// g2p.cu -- grid-to-particle transfer and mode fit (Eqs 6-8, Section 3.3),
// with the advection fused in.
//
//   c_pra = sum_i w s_r v~_ia / d_r,  d_r = sum_i w s_r^2   (decoupled LSQ)
//   v_p = c_p0,  x_p <- clamp(x_p + dt v_p, 1.5 dx, (n - 1.5) dx)
//
// One CTA per 8x8x4-cell tile.  The tile's velocity footprint on each face
// grid (at most 11 x 10 x 7 nodes) is staged in shared memory with coalesced
// loads; every thread then fits one particle at a time from the staged tile.
// The fit is the transpose of P2G's sum factorisation with per-axis weights
//   G0_k = W_k,  G1_k = W_k z_k / mu2 = 4 F1_k,  G2_k = W_k g_k / d_2 = (1,-2,1)/2
// (z in cells): the quadratic fit is half the second difference for every t,
// so no denominator is formed; the guard zeroes G2 on a guarded axis.  The
// FP32 output folds 1/dx and 1/dx^2 into the degree-1 and degree-2 factors and
// so comes out in physical units; the 16-bit formats fit c dx^L, divide by the
// per-particle scale s_p = max |c dx^L| and round to nearest even, two codes
// (modes 2k and 2k + 1) per 32-bit word.  Outputs are written in sorted slot
// order (coalesced).  With Eq 10's gradient form
// (4 modes) the linear modes are sum_i dw_ipa/dx_p v~_ia instead of the fit.
#include <type_traits>

#include "g2p.cuh"
#include "g2p_fit.cuh"

namespace polypic {

template <int R, int FMT, bool GRADW>
__global__ void __launch_bounds__(kG2PThreads) k_g2p_tiles(G2PArgs A) {
    __shared__ float s_tile[kVelTileFloats];
    const GridGeom &g = A.g;
    const uint32_t tile = blockIdx.x;
    const uint32_t jb = A.cell_start[tile * 256], je = A.cell_start[tile * 256 + 256];
    if (jb == je) return;  // CTA-uniform
    const int tx = (int)(tile % (uint32_t)g.tiles[0]);
    const int ty = (int)((tile / (uint32_t)g.tiles[0]) % (uint32_t)g.tiles[1]);
    const int tz = (int)(tile / ((uint32_t)g.tiles[0] * (uint32_t)g.tiles[1]));
    const int ox = 8 * tx - 1, oy = 8 * ty - 1, oz = 4 * tz - 1;

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

    // stage the three velocity footprints (nodes outside a grid read as 0)
    stage_velocity<0>(g, A.vel, tx, ty, tz, s_tile);
    __syncthreads();

    using T = typename Codec<FMT>::T;
    T *ocoeff = reinterpret_cast<T *>(A.ocoeff);
    const int64_t cnt = A.count;
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
        bool ok = coord_valid(v0, g.n[0]) && coord_valid(v1, g.n[1]) && coord_valid(v2, g.n[2]);
        const int ci = cell_index(v0, g.n[0]) - 8 * tx, cj = cell_index(v1, g.n[1]) - 8 * ty,
                  ck = cell_index(v2, g.n[2]) - 4 * tz;
        ok = ok && ci >= 0 && ci < 8 && cj >= 0 && cj < 8 && ck >= 0 && ck < 4;

        if (!ok) atomicOr(A.status, kFlagOutOfDomain);
        Axis ac0{}, af0{}, ac1{}, af1{}, ac2{}, af2{};
        Stencil1D sc0{}, sf0{}, sc1{}, sf1{}, sc2{}, sf2{};
        if (ok) {
            ac0 = axis_decide(v0, false); af0 = axis_decide(v0, true);
            ac1 = axis_decide(v1, false); af1 = axis_decide(v1, true);
            ac2 = axis_decide(v2, false); af2 = axis_decide(v2, true);
            sc0 = stencil_1d(ac0.t); sf0 = stencil_1d(af0.t);
            sc1 = stencil_1d(ac1.t); sf1 = stencil_1d(af1.t);
            sc2 = stencil_1d(ac2.t); sf2 = stencil_1d(af2.t);
        }
        // fit of component a (zero for a particle outside its tile)
        auto fit = [&](auto acomp, float (&C)[R]) {
            constexpr int a = decltype(acomp)::value;
            if (ok) {
                if constexpr (a == 0)
                    g2p_component<R, 0, Tile<0>::X, Tile<0>::Y, GRADW,
                                  FMT != POLYPIC_COEFF_F32>(
                        s_tile, af0.base - ox, ac1.base - oy, ac2.base - oz, sf0, af0.guard, sc1,
                        ac1.guard, sc2, ac2.guard, inv1, inv2, C, af0.t, ac1.t, ac2.t);
                else if constexpr (a == 1)
                    g2p_component<R, 1, Tile<1>::X, Tile<1>::Y, GRADW,
                                  FMT != POLYPIC_COEFF_F32>(
                        s_tile + kVelTileOff1, ac0.base - ox, af1.base - oy, ac2.base - oz, sc0,
                        ac0.guard, sf1, af1.guard, sc2, ac2.guard, inv1, inv2, C, ac0.t, af1.t,
                        ac2.t);
                else
                    g2p_component<R, 2, Tile<2>::X, Tile<2>::Y, GRADW,
                                  FMT != POLYPIC_COEFF_F32>(
                        s_tile + kVelTileOff2, ac0.base - ox, ac1.base - oy, af2.base - oz, sc0,
                        ac0.guard, sc1, ac1.guard, sf2, af2.guard, inv1, inv2, C, ac0.t, ac1.t,
                        af2.t);
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) C[r] = 0.0f;
            }
        };
        float vel[3];
        T *out = ocoeff + j;  // FP32: row (a, r) starts (a R + r) * cnt elements in
        if constexpr (FMT == POLYPIC_COEFF_F32) {
            // each component's coefficients leave as soon as they are fitted,
            // spreading the stores over the particle's arithmetic
            auto fit_store = [&](auto acomp) {
                float C[R];
                fit(acomp, C);
#pragma unroll
                for (int r = 0; r < R; ++r, out += cnt) *out = C[r];
                vel[decltype(acomp)::value] = C[0];
            };
            fit_store(std::integral_constant<int, 0>{});
            fit_store(std::integral_constant<int, 1>{});
            fit_store(std::integral_constant<int, 2>{});
        } else {
            float Chat[3][R];
            fit(std::integral_constant<int, 0>{}, Chat[0]);
            fit(std::integral_constant<int, 1>{}, Chat[1]);
            fit(std::integral_constant<int, 2>{}, Chat[2]);
            float s = 0.0f;
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int r = 0; r < R; ++r) s = fmaxf(s, fabsf(Chat[a][r]));
            const float inv = s > 0.0f ? 1.0f / s : 0.0f;
            // word (a H + k, j), H = (R + 1) / 2: modes 2k (low half) and 2k + 1
            constexpr int H = (R + 1) / 2;
            uint32_t *ow = reinterpret_cast<uint32_t *>(A.ocoeff) + j;
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int k = 0; k < H; ++k, ow += cnt) {
                    const uint32_t lo = Codec<FMT>::bits(Codec<FMT>::encode(Chat[a][2 * k] * inv));
                    const uint32_t hi = 2 * k + 1 < R
                        ? Codec<FMT>::bits(Codec<FMT>::encode(Chat[a][2 * k + 1] * inv)) : 0u;
                    *ow = lo | (hi << 16);
                }
            A.oscale[j] = s;
#pragma unroll
            for (int a = 0; a < 3; ++a) vel[a] = Chat[a][0];
        }
        const bool finite = isfinite(vel[0]) && isfinite(vel[1]) && isfinite(vel[2]);
        if (!finite) atomicOr(A.status, kFlagNonFinite);
        // advection with the fitted velocity (unquantised)
        const float vx = ok ? vel[0] : 0.0f, vy = ok ? vel[1] : 0.0f, vz = ok ? vel[2] : 0.0f;
        A.ox[j] = ok ? fminf(fmaxf(fmaf(A.dt, vx, px), g.lo[0]), g.hi[0]) : px;
        A.oy[j] = ok ? fminf(fmaxf(fmaf(A.dt, vy, py), g.lo[1]), g.hi[1]) : py;
        A.oz[j] = ok ? fminf(fmaxf(fmaf(A.dt, vz, pz), g.lo[2]), g.hi[2]) : pz;
        A.omass[j] = m;
        if (A.omass_abs) A.omass_abs[j] = mabs;
        px = nx; py = ny; pz = nz; m = nm; mabs = nmabs; pn = pnn;
    }
}

cudaError_t g2p(const G2PArgs &A, int64_t num_tiles, int R, int fmt, cudaStream_t s) {
    const int grid = (int)num_tiles;
    if (A.grad_w) {  // Eq 10's gradient form: 4 modes only
        if (R != 4) return cudaErrorInvalidValue;
        if (fmt == POLYPIC_COEFF_F32) k_g2p_tiles<4, POLYPIC_COEFF_F32, true><<<grid, kG2PThreads, 0, s>>>(A);
        else if (fmt == POLYPIC_COEFF_BF16) k_g2p_tiles<4, POLYPIC_COEFF_BF16, true><<<grid, kG2PThreads, 0, s>>>(A);
        else if (fmt == POLYPIC_COEFF_F16) k_g2p_tiles<4, POLYPIC_COEFF_F16, true><<<grid, kG2PThreads, 0, s>>>(A);
        else return cudaErrorInvalidValue;
        return cudaGetLastError();
    }
#define POLYPIC_G2P_CASE(RR, FF)                                          \
    if (R == RR && fmt == FF) {                                          \
        k_g2p_tiles<RR, FF, false><<<grid, kG2PThreads, 0, s>>>(A);      \
        return cudaGetLastError();                                       \
    }
    POLYPIC_G2P_CASE(1, POLYPIC_COEFF_F32)
    POLYPIC_G2P_CASE(4, POLYPIC_COEFF_F32)
    POLYPIC_G2P_CASE(8, POLYPIC_COEFF_F32)
    POLYPIC_G2P_CASE(27, POLYPIC_COEFF_F32)
    POLYPIC_G2P_CASE(1, POLYPIC_COEFF_BF16)
    POLYPIC_G2P_CASE(4, POLYPIC_COEFF_BF16)
    POLYPIC_G2P_CASE(8, POLYPIC_COEFF_BF16)
    POLYPIC_G2P_CASE(27, POLYPIC_COEFF_BF16)
    POLYPIC_G2P_CASE(1, POLYPIC_COEFF_F16)
    POLYPIC_G2P_CASE(4, POLYPIC_COEFF_F16)
    POLYPIC_G2P_CASE(8, POLYPIC_COEFF_F16)
    POLYPIC_G2P_CASE(27, POLYPIC_COEFF_F16)
#undef POLYPIC_G2P_CASE
    return cudaErrorInvalidValue;
}

}  // namespace polypic

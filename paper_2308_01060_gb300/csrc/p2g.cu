// p2g.cu -- deterministic particle-to-grid transfer (Eqs 1-5, 13, 15-19).
//
//   m_ia  = sum_p mt_p w_ipa
//   mv_ia = sum_p mt_p w_ipa sum_{r<R} c_pra s_r(x_ia - x_p)
//
// Work decomposition (no float atomics anywhere, so the result is
// bit-identical from run to run):
//   * particles are sorted by cell key; the 32 cells of one 4x4x2 block are
//     one contiguous key range, so a block's particles are one contiguous
//     sorted range;
//   * one warp owns one block.  It walks the block's particles 32 at a time
//     (lane = particle, loads coalesced through the near-identity perm) and
//     each lane evaluates its particle's 27 node contributions per face grid
//     with sum factorisation (81 + 81 + 81 FMA per component instead of the
//     27 x 27 direct sum);
//   * the contributions go to a shared staging array; 27 reducer lanes (one
//     per stencil slot) then sum each cell's run of particles in sorted order
//     (a warp-level segmented reduction through shared memory), keeping two
//     partial sums per slot for the two possible stencil bases along the
//     component's own axis, and add each finished run into the warp's
//     private block region in shared memory;
//   * the warp writes its block region to scratch; k_p2g_reduce sums the up
//     to 8 block regions that cover each face node, in ascending block order.
#include "p2g.cuh"

namespace polypic {

// Per-warp shared layout: staging [m | mv][27 slots][33] + block region.
constexpr int kStageStride = 33;
constexpr int kStageFloats = 2 * 27 * kStageStride;
constexpr int kWarpFloats = kStageFloats + kRegionFloats;
constexpr int kP2GWarps = 8;

template <int A> struct Reg {
    static constexpr int X = reg_x(A), Y = reg_y(A), Z = reg_z(A);
};

// 1-D factor table of one axis: F[a][k] for degree a at node k.
template <int D>
__device__ __forceinline__ void axis_factors(const Stencil1D &s, float (&F)[D][3]) {
#pragma unroll
    for (int k = 0; k < 3; ++k) F[0][k] = s.W[k];
    if constexpr (D > 1) {
#pragma unroll
        for (int k = 0; k < 3; ++k) F[1][k] = s.F1[k];
    }
    if constexpr (D > 2) {
        F[2][0] = s.phi;
        F[2][1] = -2.0f * s.phi;
        F[2][2] = s.phi;
    }
}

template <int R, int FMT, int A>
__device__ __forceinline__ void p2g_component(const P2GArgs &P, uint32_t p, bool live, float mt,
                                              float cscale, const Stencil1D (&sc)[3],
                                              const Stencil1D (&sf)[3], float *st_m,
                                              float *st_v, int lane) {
    constexpr int D = axis_degrees(R);
    using T = typename Codec<FMT>::T;
    const T *coeff = reinterpret_cast<const T *>(P.coeff);
    float Fx[D][3], Fy[D][3], Fz[D][3];
    axis_factors<D>(A == 0 ? sf[0] : sc[0], Fx);
    axis_factors<D>(A == 1 ? sf[1] : sc[1], Fy);
    axis_factors<D>(A == 2 ? sf[2] : sc[2], Fz);

    // coefficients, dimensionless: c_r dx^L_r (FP32) or code_r s_p (16-bit)
    float C[D][D][D];
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b)
#pragma unroll
            for (int c = 0; c < D; ++c) {
                if (has_mode(R, a, b, c)) {
                    const int r = mode_index(a, b, c);
                    float raw = live ? Codec<FMT>::load(coeff + ((int64_t)A * R + r) * P.count + p)
                                     : 0.0f;
                    C[a][b][c] = raw * (FMT == POLYPIC_COEFF_F32 ? P.dxpow[a + b + c] : cscale);
                } else {
                    C[a][b][c] = 0.0f;
                }
            }
    // stage 1: contract z
    float T1[D][D][3];
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b)
#pragma unroll
            for (int kz = 0; kz < 3; ++kz) {
                float s = 0.0f;
#pragma unroll
                for (int c = 0; c < D; ++c)
                    if (has_mode(R, a, b, c)) s = fmaf(C[a][b][c], Fz[c][kz], s);
                T1[a][b][kz] = s;
            }
    // stage 2: contract y
    float T2[D][3][3];
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int ky = 0; ky < 3; ++ky)
#pragma unroll
            for (int kz = 0; kz < 3; ++kz) {
                float s = 0.0f;
#pragma unroll
                for (int b = 0; b < D; ++b) s = fmaf(T1[a][b][kz], Fy[b][ky], s);
                T2[a][ky][kz] = s;
            }
    // stage 3: contract x with the particle mass folded in; mass weights
    float Fxm[D][3];
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int k = 0; k < 3; ++k) Fxm[a][k] = mt * Fx[a][k];
#pragma unroll
    for (int kz = 0; kz < 3; ++kz)
#pragma unroll
        for (int ky = 0; ky < 3; ++ky) {
            const float wyz = Fy[0][ky] * Fz[0][kz];
#pragma unroll
            for (int kx = 0; kx < 3; ++kx) {
                float s = 0.0f;
#pragma unroll
                for (int a = 0; a < D; ++a) s = fmaf(T2[a][ky][kz], Fxm[a][kx], s);
                const int slot = kx + 3 * ky + 9 * kz;
                st_v[slot * kStageStride + lane] = s;
                st_m[slot * kStageStride + lane] = Fxm[0][kx] * wyz;
            }
        }
}

template <int A>
__device__ __forceinline__ void flush_run(float *reg, int cell, int lane, const float (&acc)[2][2]) {
    const int ci = cell & 3, cj = (cell >> 2) & 3, ck = (cell >> 4) & 1;
    const int sk0 = lane % 3, sk1 = (lane / 3) % 3, sk2 = lane / 9;
    const bool red = lane < 27;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        if (red) {
            const int ix = ci + sk0 + (A == 0 ? s : 0);
            const int iy = cj + sk1 + (A == 1 ? s : 0);
            const int iz = ck + sk2 + (A == 2 ? s : 0);
            const int idx = (iz * Reg<A>::Y + iy) * Reg<A>::X + ix;
            reg[reg_off(A, 0) + idx] += acc[s][0];
            reg[reg_off(A, 1) + idx] += acc[s][1];
        }
        __syncwarp();
    }
}

template <int A>
__device__ __forceinline__ void reduce_batch(float *reg, const float *st_m, const float *st_v,
                                             int info, int nb, int lane, int &cur,
                                             float (&acc)[2][2]) {
    const bool red = lane < 27;
    for (int q = 0; q < nb; ++q) {
        const int iq = __shfl_sync(0xffffffffu, info, q);
        const int cq = iq & 31;
        const int sq = (iq >> (5 + A)) & 1;
        if (cq != cur) {  // warp-uniform
            if (cur >= 0) flush_run<A>(reg, cur, lane, acc);
            cur = cq;
            acc[0][0] = acc[0][1] = acc[1][0] = acc[1][1] = 0.0f;
        }
        if (red) {
            const float vm = st_m[lane * kStageStride + q];
            const float vv = st_v[lane * kStageStride + q];
            if (sq) {  // warp-uniform: every lane reads the same particle q
                acc[1][0] += vm;
                acc[1][1] += vv;
            } else {
                acc[0][0] += vm;
                acc[0][1] += vv;
            }
        }
    }
}

template <int R, int FMT>
__global__ void __launch_bounds__(kP2GWarps * 32, 2) k_p2g_blocks(P2GArgs P) {
    extern __shared__ float smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t b = blockIdx.x * kP2GWarps + warp;
    if (b >= P.nblocks) return;  // warp-uniform; the kernel has no CTA barrier
    const uint32_t cs0 = P.cell_start[b * 32], cs1 = P.cell_start[b * 32 + 32];
    if (cs0 == cs1) return;

    float *st_m = smem + warp * kWarpFloats;
    float *st_v = st_m + 27 * kStageStride;
    float *reg = st_m + kStageFloats;
    for (int i = lane; i < kRegionFloats; i += 32) reg[i] = 0.0f;
    __syncwarp();

    int i0, j0, k0;
    block_origin(P.g, b, i0, j0, k0);
    float acc0[2][2] = {{0, 0}, {0, 0}}, acc1[2][2] = {{0, 0}, {0, 0}}, acc2[2][2] = {{0, 0}, {0, 0}};
    int cur0 = -1, cur1 = -1, cur2 = -1;

    for (uint32_t jb = cs0; jb < cs1; jb += 32) {
        const uint32_t j = jb + lane;
        const int nb = (int)min(32u, cs1 - jb);
        const bool live = j < cs1;
        uint32_t p = 0;
        float px = 0.0f, py = 0.0f, pz = 0.0f, mt = 0.0f, cscale = 0.0f;
        if (live) {
            p = P.perm[j];
            px = P.x[p];
            py = P.y[p];
            pz = P.z[p];
            mt = P.mass[p] + (P.mass_abs ? P.mass_abs[p] : 0.0f);
            if (FMT != POLYPIC_COEFF_F32) cscale = P.scale[p];
        }
        const float v0 = cell_coord(px, P.g.inv_dx), v1 = cell_coord(py, P.g.inv_dx),
                    v2 = cell_coord(pz, P.g.inv_dx);
        bool ok = live && coord_valid(v0, P.g.n[0]) && coord_valid(v1, P.g.n[1]) &&
                  coord_valid(v2, P.g.n[2]);
        const int ci = cell_index(v0, P.g.n[0]) - i0, cj = cell_index(v1, P.g.n[1]) - j0,
                  ck = cell_index(v2, P.g.n[2]) - k0;
        ok = ok && ci >= 0 && ci < 4 && cj >= 0 && cj < 4 && ck >= 0 && ck < 2;
        if (__any_sync(0xffffffffu, live && !ok) && lane == 0) atomicOr(P.status, kFlagOutOfDomain);

        Axis ac[3], af[3];
        ac[0] = axis_decide(v0, false); af[0] = axis_decide(v0, true);
        ac[1] = axis_decide(v1, false); af[1] = axis_decide(v1, true);
        ac[2] = axis_decide(v2, false); af[2] = axis_decide(v2, true);
        Stencil1D sc[3], sf[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            sc[a] = stencil_1d(ac[a].t);
            sf[a] = stencil_1d(af[a].t);
        }
        int info = 0;
        if (ok) {
            const int s0 = af[0].base - (ci + i0 - 1), s1 = af[1].base - (cj + j0 - 1),
                      s2 = af[2].base - (ck + k0 - 1);
            info = ci | (cj << 2) | (ck << 4) | (s0 << 5) | (s1 << 6) | (s2 << 7);
        } else {
            mt = 0.0f;
        }
        const bool use = live && ok;

        p2g_component<R, FMT, 0>(P, p, use, mt, cscale, sc, sf, st_m, st_v, lane);
        __syncwarp();
        reduce_batch<0>(reg, st_m, st_v, info, nb, lane, cur0, acc0);
        __syncwarp();
        p2g_component<R, FMT, 1>(P, p, use, mt, cscale, sc, sf, st_m, st_v, lane);
        __syncwarp();
        reduce_batch<1>(reg, st_m, st_v, info, nb, lane, cur1, acc1);
        __syncwarp();
        p2g_component<R, FMT, 2>(P, p, use, mt, cscale, sc, sf, st_m, st_v, lane);
        __syncwarp();
        reduce_batch<2>(reg, st_m, st_v, info, nb, lane, cur2, acc2);
        __syncwarp();
    }
    if (cur0 >= 0) flush_run<0>(reg, cur0, lane, acc0);
    if (cur1 >= 0) flush_run<1>(reg, cur1, lane, acc1);
    if (cur2 >= 0) flush_run<2>(reg, cur2, lane, acc2);
    __syncwarp();
    float *dst = P.scratch + (size_t)b * kRegionFloats;
    for (int i = lane; i < kRegionFloats; i += 32) dst[i] = reg[i];
}

// Sum of the block regions covering each node of face grid A, in ascending
// block order (bz, by, bx); empty blocks wrote nothing and are skipped.
template <int A>
__global__ void __launch_bounds__(256) k_p2g_reduce(GridGeom g, const uint32_t *__restrict__ cs,
                                                    const float *__restrict__ scratch,
                                                    float *__restrict__ gm,
                                                    float *__restrict__ gp) {
    const int dX = g.n[0] + (A == 0), dY = g.n[1] + (A == 1), dZ = g.n[2] + (A == 2);
    const int64_t total = (int64_t)dX * dY * dZ;
    const int nbx = 2 * g.tiles[0], nby = 2 * g.tiles[1], nbz = 2 * g.tiles[2];
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx % dX);
        const int j = (int)((idx / dX) % dY);
        const int k = (int)(idx / ((int64_t)dX * dY));
        // block b covers nodes [4b - 1, 4b - 1 + RX) along x (same for y; 2b along z)
        const int bx0 = max(0, (i + 2 - Reg<A>::X + 3) >> 2), bx1 = min(nbx - 1, (i + 1) >> 2);
        const int by0 = max(0, (j + 2 - Reg<A>::Y + 3) >> 2), by1 = min(nby - 1, (j + 1) >> 2);
        const int bz0 = max(0, (k + 2 - Reg<A>::Z + 1) >> 1), bz1 = min(nbz - 1, (k + 1) >> 1);
        float sm = 0.0f, sv = 0.0f;
        for (int bz = bz0; bz <= bz1; ++bz)
            for (int by = by0; by <= by1; ++by)
                for (int bx = bx0; bx <= bx1; ++bx) {
                    const uint32_t blk = block_of(g, bx, by, bz);
                    if (cs[blk * 32] == cs[blk * 32 + 32]) continue;
                    const int lx = i - (4 * bx - 1), ly = j - (4 * by - 1), lz = k - (2 * bz - 1);
                    const int r = (lz * Reg<A>::Y + ly) * Reg<A>::X + lx;
                    const float *src = scratch + (size_t)blk * kRegionFloats;
                    sm += src[reg_off(A, 0) + r];
                    sv += src[reg_off(A, 1) + r];
                }
        gm[idx] = sm;
        gp[idx] = sv;
    }
}

template <int R, int FMT>
static cudaError_t launch_blocks(const P2GArgs &P, cudaStream_t s) {
    static bool attr_set = false;
    const int smem = kP2GWarps * kWarpFloats * (int)sizeof(float);
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_p2g_blocks<R, FMT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const int grid = (int)((P.nblocks + kP2GWarps - 1) / kP2GWarps);
    k_p2g_blocks<R, FMT><<<grid, kP2GWarps * 32, smem, s>>>(P);
    return cudaGetLastError();
}

size_t p2g_scratch_bytes(int64_t num_keys) {
    return (size_t)(num_keys / 32) * kRegionFloats * sizeof(float) + 256;
}

cudaError_t p2g(const P2GArgs &P, float *gm[3], float *gp[3], int R, int fmt, cudaStream_t s) {
    cudaError_t e = cudaErrorInvalidValue;
#define POLYPIC_P2G_CASE(RR, FF) \
    if (R == RR && fmt == FF) e = launch_blocks<RR, FF>(P, s);
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
    const GridGeom &g = P.g;
    auto blocks_for = [&](int a) {
        int64_t tot = (int64_t)(g.n[0] + (a == 0)) * (g.n[1] + (a == 1)) * (g.n[2] + (a == 2));
        int64_t nb = (tot + 255) / 256;
        return (int)(nb < 152 * 64 ? nb : 152 * 64);
    };
    k_p2g_reduce<0><<<blocks_for(0), 256, 0, s>>>(g, P.cell_start, P.scratch, gm[0], gp[0]);
    k_p2g_reduce<1><<<blocks_for(1), 256, 0, s>>>(g, P.cell_start, P.scratch, gm[1], gp[1]);
    k_p2g_reduce<2><<<blocks_for(2), 256, 0, s>>>(g, P.cell_start, P.scratch, gm[2], gp[2]);
    return cudaGetLastError();
}

}  // namespace polypic

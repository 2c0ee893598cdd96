// pcg.cu -- pressure projection of the fluid grid velocity.
//
// The paper delegates the pressure solve to the host simulator (Section 3);
// this is the stated minimal form.  Cells holding fluid particles are fluid;
// other cells have p = 0; walls have zero normal velocity.  For a fluid cell c
//   sum_{non-wall neighbours n} (p_c - p_n) = -(rho dx^2 / dt) div_c,
//   div_c = sum_a (v_a(c + e_a) - v_a(c)) / dx,
// solved by conjugate gradients with FP32 vectors and FP64 dot products and
// norms (two-stage deterministic reductions), preconditioned by one
// multigrid V-cycle; then v_a -= dt / (rho dx) (p_hi - p_lo) on every non-wall
// face next to a fluid cell.  alpha and beta are formed on the device; the
// host reads the residual norm every kCheckEvery iterations.
//
// The V-cycle (an aggregation multigrid): a coarse cell is the 2x2x2 block of
// fine cells, fluid if any child is; the coarse operator is the Galerkin
// product P^T A P with P the injection of a coarse value into its fluid
// children, so every level is again a 7-point operator (diagonal and one
// coupling per +x/+y/+z face).  Two damped-Jacobi sweeps (omega 2/3) from zero
// before the coarse correction and two after it, the residual restricted by
// P^T, the coarsest level (at most 512 cells) swept 32 times in one CTA.  The
// cycle is a fixed symmetric linear operator, positive definite because the
// sweeps converge and the Galerkin correction is an A-orthogonal projection,
// so CG keeps its guarantees.
#include <cmath>

#include <new>

#include "pcg.cuh"

namespace polypic {

constexpr int kPcgThreads = 256;
constexpr int kPcgMaxBlocks = 1024;
constexpr int kCheckEvery = 8;

struct PcgBuffers {
    float *x, *r, *z, *d, *d2, *Ap, *diag, *wd;  // d / d2: directions (ping-pong), wd = omega / diag
    uint8_t *fluid;
    double *partial;  // [2][kPcgMaxBlocks]
    double *scal;     // the scalars named by the enum below
};

// scal[]: rz of the current and the previous direction, pAp, |r|^2, |b|^2, rz
// of the newest preconditioned residual
enum { kRz = 0, kRzPrev = 1, kPAp = 2, kRr = 3, kBb = 4, kRzNext = 5 };

__device__ __forceinline__ int64_t cidx(const GridGeom &g, int i, int j, int k) {
    return ((int64_t)k * g.n[1] + j) * g.n[0] + i;
}

// Block sums of two doubles -> partial[blockIdx], partial[kPcgMaxBlocks + blockIdx].
__device__ __forceinline__ void block_sum2(double a, double b, double *partial) {
    __shared__ double sa[kPcgThreads / 32], sb[kPcgThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        sa[w] = a;
        sb[w] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0.0, tb = 0.0;
        for (int i = 0; i < kPcgThreads / 32; ++i) {
            ta += sa[i];
            tb += sb[i];
        }
        partial[blockIdx.x] = ta;
        partial[kPcgMaxBlocks + blockIdx.x] = tb;
    }
}

// Final sums of the partials into scal[ia], scal[ib] (ib < 0: ignore the second).
__global__ void __launch_bounds__(kPcgThreads) k_final(const double *partial, int nblocks,
                                                       double *scal, int ia, int ib) {
    __shared__ double sa[kPcgThreads], sb[kPcgThreads];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nblocks; i += kPcgThreads) {
        a += partial[i];
        b += partial[kPcgMaxBlocks + i];
    }
    sa[threadIdx.x] = a;
    sb[threadIdx.x] = b;
    __syncthreads();
    for (int s = kPcgThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sa[threadIdx.x] += sa[threadIdx.x + s];
            sb[threadIdx.x] += sb[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        scal[ia] = sa[0];
        if (ib >= 0) scal[ib] = sb[0];
    }
}

// ---------------------------------------------------------------- multigrid levels
constexpr int kMgMaxLevels = 12;
constexpr int kMgCoarsest = 512;      // cells of the level swept in one CTA
constexpr int kMgCoarseSweeps = 32;
constexpr float kMgOmega = 2.0f / 3.0f;

// One level of the hierarchy.  Level 0 is the fine system: couplings are -1
// between fluid neighbours (ox == nullptr).  Coarse levels store the Galerkin
// diagonal and the coupling of each cell to its +x, +y, +z neighbour.
struct MgLevel {
    int n[3];
    int64_t cells;
    uint8_t *fluid;
    float *diag, *wd, *ox, *oy, *oz;  // wd = omega / diag, the damped Jacobi scale
    float *x, *b, *t;
};

__host__ __device__ inline int mg_coarse_dim(int n) { return (n + 1) / 2; }

// Coupling of fluid cell c to neighbour m across face (axis a, side +1/-1).
__device__ __forceinline__ float mg_off(const MgLevel &L, int64_t c, int64_t m, int a, int side) {
    if (!L.ox) return L.fluid[m] ? -1.0f : 0.0f;
    const float *o = a == 0 ? L.ox : (a == 1 ? L.oy : L.oz);
    return side > 0 ? o[c] : o[m];
}

// (A v)(c) for fluid cell c at (i, j, k); v(m, i, j, k) gives the vector at
// cell m with coordinates (i, j, k) (called for c and its in-domain
// neighbours, so no functor divides an index).
template <class V>
__device__ __forceinline__ float mg_apply(const MgLevel &L, int64_t c, int i, int j, int k,
                                          const V &v) {
    float s = L.diag[c] * v(c, i, j, k);
    const int64_t sx = 1, sy = L.n[0], sz = (int64_t)L.n[0] * L.n[1];
    if (i > 0) s = fmaf(mg_off(L, c, c - sx, 0, -1), v(c - sx, i - 1, j, k), s);
    if (i < L.n[0] - 1) s = fmaf(mg_off(L, c, c + sx, 0, +1), v(c + sx, i + 1, j, k), s);
    if (j > 0) s = fmaf(mg_off(L, c, c - sy, 1, -1), v(c - sy, i, j - 1, k), s);
    if (j < L.n[1] - 1) s = fmaf(mg_off(L, c, c + sy, 1, +1), v(c + sy, i, j + 1, k), s);
    if (k > 0) s = fmaf(mg_off(L, c, c - sz, 2, -1), v(c - sz, i, j, k - 1), s);
    if (k < L.n[2] - 1) s = fmaf(mg_off(L, c, c + sz, 2, +1), v(c + sz, i, j, k + 1), s);
    return s;
}

// Cell coordinates of a linear index (32-bit division where the index fits).
__device__ __forceinline__ void cell_ijk(int64_t c, int n0, int n1, int &i, int &j, int &k) {
    if (c < 0x7fffffffLL) {
        const uint32_t u = (uint32_t)c, q = u / (uint32_t)n0;
        i = (int)(u - q * (uint32_t)n0);
        j = (int)(q % (uint32_t)n1);
        k = (int)(q / (uint32_t)n1);
    } else {
        const int64_t q = c / n0;
        i = (int)(c - q * n0);
        j = (int)(q % n1);
        k = (int)(q / n1);
    }
}

__device__ __forceinline__ void mg_ijk(const MgLevel &L, int64_t c, int &i, int &j, int &k) {
    cell_ijk(c, L.n[0], L.n[1], i, j, k);
}

#define MG_CELLS(L, c) \
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < (L).cells; \
         c += (int64_t)gridDim.x * blockDim.x)

// Coarse level from fine: fluid flags, Galerkin diagonal and couplings.
__global__ void __launch_bounds__(kPcgThreads) k_mg_coarsen(MgLevel F, MgLevel C) {
    MG_CELLS(C, cc) {
        int I, J, K;
        mg_ijk(C, cc, I, J, K);
        bool fl = false;
        float d = 0.0f, ox = 0.0f, oy = 0.0f, oz = 0.0f;
        for (int q = 0; q < 8; ++q) {
            const int a = q & 1, b = (q >> 1) & 1, e = q >> 2;
            const int i = 2 * I + a, j = 2 * J + b, k = 2 * K + e;
            if (i >= F.n[0] || j >= F.n[1] || k >= F.n[2]) continue;
            const int64_t c = ((int64_t)k * F.n[1] + j) * F.n[0] + i;
            if (!F.fluid[c]) continue;
            fl = true;
            d += F.diag[c];
            // the child's +x / +y / +z couplings: inside the block they fold
            // into the diagonal (both orderings), across it they couple blocks
            if (i + 1 < F.n[0]) {
                const float o = mg_off(F, c, c + 1, 0, +1);
                if (a == 0) d += 2.0f * o; else ox += o;
            }
            if (j + 1 < F.n[1]) {
                const float o = mg_off(F, c, c + F.n[0], 1, +1);
                if (b == 0) d += 2.0f * o; else oy += o;
            }
            if (k + 1 < F.n[2]) {
                const float o = mg_off(F, c, c + (int64_t)F.n[0] * F.n[1], 2, +1);
                if (e == 0) d += 2.0f * o; else oz += o;
            }
        }
        C.fluid[cc] = fl ? 1 : 0;
        C.diag[cc] = fl ? d : 1.0f;
        C.wd[cc] = fl ? kMgOmega / d : 0.0f;
        C.ox[cc] = ox;
        C.oy[cc] = oy;
        C.oz[cc] = oz;
    }
}

// Two damped-Jacobi sweeps from x = 0: x1 = w b / D (formed on the fly for
// the neighbours), x = x1 + w (b - A x1) / D.
__global__ void __launch_bounds__(kPcgThreads) k_mg_pre(MgLevel L) {
    auto x1 = [&](int64_t m, int, int, int) {
        return L.fluid[m] ? L.wd[m] * L.b[m] : 0.0f;
    };
    MG_CELLS(L, c) {
        float out = 0.0f;
        if (L.fluid[c]) {
            int i, j, k;
            mg_ijk(L, c, i, j, k);
            const float ax = mg_apply(L, c, i, j, k, x1);
            out = fmaf(L.wd[c], L.b[c] - ax, x1(c, i, j, k));
        }
        L.x[c] = out;
    }
}

// Coarse right-hand side: the fine residual b - A x summed over each block's
// fluid children (P^T r).
__global__ void __launch_bounds__(kPcgThreads) k_mg_restrict(MgLevel F, MgLevel C) {
    auto xf = [&](int64_t m, int, int, int) { return F.x[m]; };
    MG_CELLS(C, cc) {
        float s = 0.0f;
        if (C.fluid[cc]) {
            int I, J, K;
            mg_ijk(C, cc, I, J, K);
            for (int q = 0; q < 8; ++q) {
                const int i = 2 * I + (q & 1), j = 2 * J + ((q >> 1) & 1), k = 2 * K + (q >> 2);
                if (i >= F.n[0] || j >= F.n[1] || k >= F.n[2]) continue;
                const int64_t c = ((int64_t)k * F.n[1] + j) * F.n[0] + i;
                if (!F.fluid[c]) continue;
                s += F.b[c] - mg_apply(F, c, i, j, k, xf);
            }
        }
        C.b[cc] = s;
    }
}

// Coarse correction and the first post-sweep: x' = x + P x_c (formed on the
// fly), t = x' + w (b - A x') / D.
__global__ void __launch_bounds__(kPcgThreads) k_mg_post(MgLevel F, MgLevel C) {
    auto xp = [&](int64_t m, int i, int j, int k) {
        if (!F.fluid[m]) return 0.0f;
        return F.x[m] + C.x[((int64_t)(k >> 1) * C.n[1] + (j >> 1)) * C.n[0] + (i >> 1)];
    };
    MG_CELLS(F, c) {
        float out = 0.0f;
        if (F.fluid[c]) {
            int i, j, k;
            mg_ijk(F, c, i, j, k);
            const float ax = mg_apply(F, c, i, j, k, xp);
            out = fmaf(F.wd[c], F.b[c] - ax, xp(c, i, j, k));
        }
        F.t[c] = out;
    }
}

// The second post-sweep: x = t + w (b - A t) / D.  On level 0 (DOT) it also
// forms the block sums of b . x = r . z for CG.
template <bool DOT>
__global__ void __launch_bounds__(kPcgThreads) k_mg_sweep(MgLevel L, double *partial) {
    auto tv = [&](int64_t m, int, int, int) { return L.t[m]; };
    double rz = 0.0;
    MG_CELLS(L, c) {
        float out = 0.0f;
        if (L.fluid[c]) {
            int i, j, k;
            mg_ijk(L, c, i, j, k);
            out = fmaf(L.wd[c], L.b[c] - mg_apply(L, c, i, j, k, tv), L.t[c]);
            if (DOT) rz += (double)L.b[c] * (double)out;
        }
        L.x[c] = out;
    }
    if (DOT) block_sum2(rz, 0.0, partial);
}

// The coarsest level: kMgCoarseSweeps damped-Jacobi sweeps from x = 0 in one
// CTA (one thread per cell, the iterate in shared memory).
__global__ void __launch_bounds__(kMgCoarsest) k_mg_coarsest(MgLevel L) {
    __shared__ float s_x[2][kMgCoarsest];
    const int64_t c = threadIdx.x;
    const bool live = c < L.cells && L.fluid[c];
    int i = 0, j = 0, k = 0;
    if (c < L.cells) mg_ijk(L, c, i, j, k);
    s_x[0][c] = 0.0f;
    __syncthreads();
    int cur = 0;
    for (int it = 0; it < kMgCoarseSweeps; ++it) {
        float out = 0.0f;
        if (live) {
            const float *xs = s_x[cur];
            auto v = [&](int64_t m, int, int, int) { return xs[m]; };
            out = fmaf(L.wd[c], L.b[c] - mg_apply(L, c, i, j, k, v), xs[c]);
        }
        s_x[cur ^ 1][c] = out;
        __syncthreads();
        cur ^= 1;
    }
    if (c < L.cells) L.x[c] = s_x[cur][c];
}

// Block sums of b . x (r . z) over the fluid cells, for a one-level cycle.
__global__ void __launch_bounds__(kPcgThreads) k_mg_dot(MgLevel L, double *partial) {
    double rz = 0.0;
    MG_CELLS(L, c) {
        if (L.fluid[c]) rz += (double)L.b[c] * (double)L.x[c];
    }
    block_sum2(rz, 0.0, partial);
}

struct Multigrid {
    int levels;  // the coarsest is levels - 1
    MgLevel L[kMgMaxLevels];
};

// Level dimensions: halve (rounding up) until at most kMgCoarsest cells.
static int mg_dims(const GridGeom &g, int dims[kMgMaxLevels][3]) {
    int n[3] = {g.n[0], g.n[1], g.n[2]};
    int lv = 0;
    for (;;) {
        for (int a = 0; a < 3; ++a) dims[lv][a] = n[a];
        ++lv;
        if ((int64_t)n[0] * n[1] * n[2] <= kMgCoarsest || lv == kMgMaxLevels) break;
        for (int a = 0; a < 3; ++a) n[a] = mg_coarse_dim(n[a]);
    }
    return lv;
}

static size_t mg_scratch_bytes(const GridGeom &g) {
    int dims[kMgMaxLevels][3];
    const int lv = mg_dims(g, dims);
    size_t bytes = 0;
    for (int l = 1; l < lv; ++l) {
        const size_t cells = (size_t)dims[l][0] * dims[l][1] * dims[l][2];
        bytes += cells * (8 * sizeof(float) + 1) + 9 * 256;
    }
    return bytes;
}
__global__ void __launch_bounds__(kPcgThreads) k_setup(GridGeom g, int64_t num_keys,
                                                       const uint32_t *__restrict__ cs,
                                                       const float *__restrict__ v0,
                                                       const float *__restrict__ v1,
                                                       const float *__restrict__ v2, float scale,
                                                       PcgBuffers B) {
    const int64_t nc = (int64_t)g.n[0] * g.n[1] * g.n[2];
    double bb = 0.0;
    for (int64_t c = (int64_t)blockIdx.x * kPcgThreads + threadIdx.x; c < nc;
         c += (int64_t)gridDim.x * kPcgThreads) {
        int i, j, k;
        cell_ijk(c, g.n[0], g.n[1], i, j, k);
        const uint32_t key = cell_key(g, i, j, k);
        const bool fl = cs[key + 1] > cs[key];
        B.fluid[c] = fl ? 1 : 0;
        float b = 0.0f, dg = 1.0f;
        if (fl) {
            const int d0 = g.n[0] + 1, d1 = g.n[1] + 1;
            const float div = (v0[((int64_t)k * g.n[1] + j) * d0 + i + 1] - v0[((int64_t)k * g.n[1] + j) * d0 + i]) +
                              (v1[((int64_t)k * d1 + j + 1) * g.n[0] + i] - v1[((int64_t)k * d1 + j) * g.n[0] + i]) +
                              (v2[((int64_t)(k + 1) * g.n[1] + j) * g.n[0] + i] - v2[((int64_t)k * g.n[1] + j) * g.n[0] + i]);
            b = -scale * div;
            int nn = 0;
            nn += (i > 0) + (i < g.n[0] - 1) + (j > 0) + (j < g.n[1] - 1) + (k > 0) + (k < g.n[2] - 1);
            dg = (float)nn;
        }
        B.diag[c] = dg;
        B.wd[c] = fl ? kMgOmega / dg : 0.0f;
        B.x[c] = 0.0f;
        B.r[c] = b;
        B.d[c] = 0.0f;
        B.d2[c] = 0.0f;
        bb += (double)b * (double)b;
    }
    block_sum2(0.0, bb, B.partial);
}

// The new direction and its product with A in one pass: d_out = z + beta d_in
// (beta = rz / rz_prev, 0 for the first direction), formed on the fly for
// the neighbours, Ap = A d_out, and the block sums of d_out . Ap.
__global__ void __launch_bounds__(kPcgThreads) k_apply(GridGeom g, PcgBuffers B,
                                                       const float *__restrict__ d_in,
                                                       float *__restrict__ d_out, bool first) {
    const int64_t nc = (int64_t)g.n[0] * g.n[1] * g.n[2];
    const double rz = B.scal[kRz], rz_prev = B.scal[kRzPrev];
    const float beta = first || rz_prev == 0.0 ? 0.0f : (float)(rz / rz_prev);
    auto dn = [&](int64_t m) { return B.fluid[m] ? fmaf(beta, d_in[m], B.z[m]) : 0.0f; };
    double pap = 0.0;
    for (int64_t c = (int64_t)blockIdx.x * kPcgThreads + threadIdx.x; c < nc;
         c += (int64_t)gridDim.x * kPcgThreads) {
        float s = 0.0f, dc = 0.0f;
        if (B.fluid[c]) {
            int i, j, k;
            cell_ijk(c, g.n[0], g.n[1], i, j, k);
            dc = dn(c);
            s = B.diag[c] * dc;
            const int64_t sl = (int64_t)g.n[0] * g.n[1];
            if (i > 0) s -= dn(c - 1);
            if (i < g.n[0] - 1) s -= dn(c + 1);
            if (j > 0) s -= dn(c - g.n[0]);
            if (j < g.n[1] - 1) s -= dn(c + g.n[0]);
            if (k > 0) s -= dn(c - sl);
            if (k < g.n[2] - 1) s -= dn(c + sl);
        }
        d_out[c] = dc;
        B.Ap[c] = s;
        pap += (double)dc * (double)s;
    }
    block_sum2(pap, 0.0, B.partial);
}

__global__ void __launch_bounds__(kPcgThreads) k_update(GridGeom g, PcgBuffers B,
                                                        const float *__restrict__ d) {
    const int64_t nc = (int64_t)g.n[0] * g.n[1] * g.n[2];
    const double pap = B.scal[kPAp];
    const float alpha = pap != 0.0 ? (float)(B.scal[kRz] / pap) : 0.0f;
    double rr = 0.0;
    for (int64_t c = (int64_t)blockIdx.x * kPcgThreads + threadIdx.x; c < nc;
         c += (int64_t)gridDim.x * kPcgThreads) {
        if (!B.fluid[c]) continue;
        B.x[c] = fmaf(alpha, d[c], B.x[c]);
        const float r = fmaf(-alpha, B.Ap[c], B.r[c]);
        B.r[c] = r;
        rr += (double)r * (double)r;
    }
    block_sum2(rr, 0.0, B.partial);
}

// rz of the newest preconditioned residual becomes the current one.
__global__ void k_rotate(double *scal) {
    scal[kRzPrev] = scal[kRz];
    scal[kRz] = scal[kRzNext];
}

__global__ void k_latch(uint32_t *status, uint32_t flag) { atomicOr(status, flag); }

// v_a -= dt/(rho dx) (p_hi - p_lo) on non-wall faces next to a fluid cell.
__global__ void __launch_bounds__(kPcgThreads) k_velocity(GridGeom g, int a, float coef,
                                                          const float *__restrict__ p,
                                                          const uint8_t *__restrict__ fluid,
                                                          float *__restrict__ v) {
    const int dX = g.n[0] + (a == 0), dY = g.n[1] + (a == 1), dZ = g.n[2] + (a == 2);
    const int64_t total = (int64_t)dX * dY * dZ;
    for (int64_t f = (int64_t)blockIdx.x * kPcgThreads + threadIdx.x; f < total;
         f += (int64_t)gridDim.x * kPcgThreads) {
        int i, j, k;
        cell_ijk(f, dX, dY, i, j, k);
        const int ia = a == 0 ? i : (a == 1 ? j : k);
        if (ia == 0 || ia == g.n[a]) continue;
        const int64_t hi = cidx(g, i, j, k);
        const int64_t lo = cidx(g, i - (a == 0), j - (a == 1), k - (a == 2));
        if (!fluid[hi] && !fluid[lo]) continue;
        v[f] -= coef * (p[hi] - p[lo]);
    }
}

size_t pcg_scratch_bytes(const GridGeom &g) {
    const size_t nc = (size_t)g.n[0] * g.n[1] * g.n[2];
    return nc * (8 * sizeof(float) + 1) + (2 * kPcgMaxBlocks + 16) * sizeof(double) + 10 * 256 +
           mg_scratch_bytes(g);
}

// z = V-cycle(r): level 0 reads B.r, writes B.z, sweeps through B.Ap; its
// last sweep also leaves the block sums of r . z in `partial` (nb blocks).
static cudaError_t mg_vcycle(const Multigrid &M, double *partial, int nb, cudaStream_t s) {
    auto blocks = [](int64_t cells) {
        return (int)std::min<int64_t>(152 * 8, (cells + kPcgThreads - 1) / kPcgThreads);
    };
    const int top = M.levels - 1;
    for (int l = 0; l < top; ++l) {
        k_mg_pre<<<blocks(M.L[l].cells), kPcgThreads, 0, s>>>(M.L[l]);
        k_mg_restrict<<<blocks(M.L[l + 1].cells), kPcgThreads, 0, s>>>(M.L[l], M.L[l + 1]);
    }
    k_mg_coarsest<<<1, kMgCoarsest, 0, s>>>(M.L[top]);
    for (int l = top - 1; l >= 0; --l) {
        k_mg_post<<<blocks(M.L[l].cells), kPcgThreads, 0, s>>>(M.L[l], M.L[l + 1]);
        if (l > 0)
            k_mg_sweep<false><<<blocks(M.L[l].cells), kPcgThreads, 0, s>>>(M.L[l], nullptr);
        else
            k_mg_sweep<true><<<nb, kPcgThreads, 0, s>>>(M.L[l], partial);
    }
    if (top == 0) {  // one level: the coarsest sweeps are the whole cycle
        k_mg_dot<<<nb, kPcgThreads, 0, s>>>(M.L[0], partial);
    }
    return cudaGetLastError();
}

// Iterations it0 .. it0 + batch - 1 of the CG loop: the new direction and
// its product with A, the step, the residual norm, the V-cycle, r . z.
static void launch_batch(const GridGeom &g, PcgBuffers &B, const Multigrid &M, int nb, int it0,
                         int batch, cudaStream_t s) {
    for (int b = 0; b < batch; ++b) {
        // directions alternate between d and d2
        const bool odd = (it0 + b) & 1;
        float *d_in = odd ? B.d2 : B.d, *d_out = odd ? B.d : B.d2;
        k_apply<<<nb, kPcgThreads, 0, s>>>(g, B, d_in, d_out, it0 + b == 0);
        k_final<<<1, kPcgThreads, 0, s>>>(B.partial, nb, B.scal, kPAp, -1);
        k_update<<<nb, kPcgThreads, 0, s>>>(g, B, d_out);
        k_final<<<1, kPcgThreads, 0, s>>>(B.partial, nb, B.scal, kRr, -1);
        mg_vcycle(M, B.partial, nb, s);
        k_final<<<1, kPcgThreads, 0, s>>>(B.partial, nb, B.scal, kRzNext, -1);
        k_rotate<<<1, 1, 0, s>>>(B.scal);
    }
}

// Two workspace layouts are kept (the forward projection and the adjoint's,
// whose vectors sit behind three face arrays), the older one replaced.
struct PcgGraphs {
    cudaStream_t side = nullptr;   // capture stream (the caller's may be the legacy one)
    struct Entry {
        const float *key = nullptr;                    // B.x of the captured layout
        cudaGraphExec_t exec[2] = {nullptr, nullptr};  // [1]: the batch from iteration 0
        uint64_t used = 0;
    } entry[2];
    uint64_t clock = 0;
};

static void drop(PcgGraphs::Entry &E) {
    for (auto &e : E.exec)
        if (e) {
            cudaGraphExecDestroy(e);
            e = nullptr;
        }
    E.key = nullptr;
}

void pcg_graphs_free(PcgGraphs *G) {
    if (!G) return;
    for (auto &E : G->entry) drop(E);
    if (G->side) cudaStreamDestroy(G->side);
    delete G;
}

// The captured graph of a full batch (kCheckEvery iterations from an even
// iteration count), captured on first use for this workspace; nullptr if the
// capture is not possible here (the batch is then launched directly).
static cudaGraphExec_t batch_graph(PcgGraphs *&G, const GridGeom &g, PcgBuffers &B,
                                   const Multigrid &M, int nb, bool first) {
    if (!G) G = new (std::nothrow) PcgGraphs;
    if (!G) return nullptr;
    PcgGraphs::Entry *E = G->entry[0].key == B.x ? &G->entry[0]
                          : G->entry[1].key == B.x ? &G->entry[1] : nullptr;
    if (!E) {
        E = G->entry[0].used <= G->entry[1].used ? &G->entry[0] : &G->entry[1];
        drop(*E);
        E->key = B.x;
    }
    E->used = ++G->clock;
    cudaGraphExec_t &ex = E->exec[first ? 1 : 0];
    if (ex) return ex;
    if (!G->side && cudaStreamCreateWithFlags(&G->side, cudaStreamNonBlocking) != cudaSuccess) {
        G->side = nullptr;
        (void)cudaGetLastError();
        return nullptr;
    }
    if (cudaStreamBeginCapture(G->side, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    // a later batch is the loop from any even iteration count but 0: the same
    // kernels with k_apply's `first` off
    launch_batch(g, B, M, nb, first ? 0 : kCheckEvery, kCheckEvery, G->side);
    cudaGraph_t graph = nullptr;
    const cudaError_t e1 = cudaStreamEndCapture(G->side, &graph);
    if (e1 != cudaSuccess || !graph) {
        (void)cudaGetLastError();
        return nullptr;
    }
    const cudaError_t e2 = cudaGraphInstantiate(&ex, graph, 0);
    cudaGraphDestroy(graph);
    if (e2 != cudaSuccess) {
        ex = nullptr;
        (void)cudaGetLastError();
        return nullptr;
    }
    return ex;
}

polypic_status pcg_project(const GridGeom &g, int64_t num_keys, const uint32_t *cell_start,
                           float *vel[3], float dt, float rho, int maxiter, double rtol,
                           uint32_t *status, Workspace &ws, cudaStream_t s, PcgGraphs **graphs) {
    (void)num_keys;
    const int64_t nc = (int64_t)g.n[0] * g.n[1] * g.n[2];
    PcgBuffers B;
    B.x = ws.take<float>(nc);
    B.r = ws.take<float>(nc);
    B.z = ws.take<float>(nc);
    B.d = ws.take<float>(nc);
    B.d2 = ws.take<float>(nc);
    B.Ap = ws.take<float>(nc);
    B.diag = ws.take<float>(nc);
    B.wd = ws.take<float>(nc);
    B.fluid = ws.take<uint8_t>(nc);
    B.partial = ws.take<double>(2 * kPcgMaxBlocks);
    B.scal = ws.take<double>(16);
    // the multigrid hierarchy: level 0 reads r, writes z, sweeps through Ap
    Multigrid M;
    {
        int dims[kMgMaxLevels][3];
        M.levels = mg_dims(g, dims);
        for (int l = 0; l < M.levels; ++l) {
            MgLevel &L = M.L[l];
            for (int a = 0; a < 3; ++a) L.n[a] = dims[l][a];
            L.cells = (int64_t)L.n[0] * L.n[1] * L.n[2];
            if (l == 0) {
                L.fluid = B.fluid;
                L.diag = B.diag;
                L.wd = B.wd;
                L.ox = L.oy = L.oz = nullptr;
                L.x = B.z;
                L.b = B.r;
                L.t = B.Ap;
            } else {
                L.fluid = ws.take<uint8_t>(L.cells);
                L.diag = ws.take<float>(L.cells);
                L.wd = ws.take<float>(L.cells);
                L.ox = ws.take<float>(L.cells);
                L.oy = ws.take<float>(L.cells);
                L.oz = ws.take<float>(L.cells);
                L.x = ws.take<float>(L.cells);
                L.b = ws.take<float>(L.cells);
                L.t = ws.take<float>(L.cells);
            }
        }
    }
    if (ws.overflow) return POLYPIC_ERR_WORKSPACE;
    // the coarsest level is swept by one CTA of kMgCoarsest threads
    if (M.L[M.levels - 1].cells > kMgCoarsest) return POLYPIC_ERR_UNSUPPORTED;
    const int nb = (int)std::min<int64_t>(kPcgMaxBlocks, (nc + kPcgThreads - 1) / kPcgThreads);
    const double gdx = (double)g.dx;
    // rhs = -(rho dx^2 / dt) div with div = (sum of face differences) / dx
    const float scale = (float)((double)rho * gdx / (double)dt);

    auto ok = [&]() { return cudaGetLastError() == cudaSuccess; };
    k_setup<<<nb, kPcgThreads, 0, s>>>(g, num_keys, cell_start, vel[0], vel[1], vel[2], scale, B);
    k_final<<<1, kPcgThreads, 0, s>>>(B.partial, nb, B.scal, kRr, kBb);
    for (int l = 1; l < M.levels; ++l) {
        const int blocks = (int)std::min<int64_t>(152 * 8, (M.L[l].cells + kPcgThreads - 1) / kPcgThreads);
        k_mg_coarsen<<<blocks, kPcgThreads, 0, s>>>(M.L[l - 1], M.L[l]);
    }
    // z = M^-1 r and rz = r . z (the first direction is z: k_apply's `first`)
    if (mg_vcycle(M, B.partial, nb, s) != cudaSuccess) return POLYPIC_ERR_CUDA;
    k_final<<<1, kPcgThreads, 0, s>>>(B.partial, nb, B.scal, kRzNext, -1);
    k_rotate<<<1, 1, 0, s>>>(B.scal);
    if (!ok()) return POLYPIC_ERR_CUDA;
    double host[5];
    if (cudaMemcpyAsync(host, B.scal, 5 * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return POLYPIC_ERR_CUDA;
    const double bnorm = std::sqrt(host[kBb]);
    bool converged = bnorm == 0.0;
    int it = 0;
    while (!converged && it < maxiter) {
        const int batch = std::min(kCheckEvery, maxiter - it);
        // a full batch replays its captured graph (its kernels and arguments
        // depend only on the workspace and on whether it is the first)
        cudaGraphExec_t ex = batch == kCheckEvery && graphs
                                 ? batch_graph(*graphs, g, B, M, nb, it == 0)
                                 : nullptr;
        if (ex) {
            if (cudaGraphLaunch(ex, s) != cudaSuccess) return POLYPIC_ERR_CUDA;
        } else {
            launch_batch(g, B, M, nb, it, batch, s);
        }
        if (!ok()) return POLYPIC_ERR_CUDA;
        it += batch;
        if (cudaMemcpyAsync(host, B.scal, 5 * sizeof(double), cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return POLYPIC_ERR_CUDA;
        converged = std::sqrt(host[kRr]) <= rtol * bnorm;
    }
    const float coef = (float)((double)dt / ((double)rho * gdx));
    for (int a = 0; a < 3; ++a) {
        const int64_t tot = (int64_t)(g.n[0] + (a == 0)) * (g.n[1] + (a == 1)) * (g.n[2] + (a == 2));
        const int blocks = (int)std::min<int64_t>(152 * 16, (tot + kPcgThreads - 1) / kPcgThreads);
        k_velocity<<<blocks, kPcgThreads, 0, s>>>(g, a, coef, B.x, B.fluid, vel[a]);
    }
    if (!ok()) return POLYPIC_ERR_CUDA;
    if (!converged) {
        k_latch<<<1, 1, 0, s>>>(status, kFlagNotConverged);
        return POLYPIC_ERR_NOT_CONVERGED;
    }
    return POLYPIC_OK;
}

}  // namespace polypic

// pcg.cu -- pressure projection of the fluid grid velocity.
//
// The paper delegates the pressure solve to the host simulator (Section 3);
// this is the stated minimal form.  Cells holding fluid particles are fluid;
// other cells have p = 0; walls have zero normal velocity.  For a fluid cell c
//   sum_{non-wall neighbours n} (p_c - p_n) = -(rho dx^2 / dt) div_c,
//   div_c = sum_a (v_a(c + e_a) - v_a(c)) / dx,
// solved by Jacobi-preconditioned conjugate gradients with FP32 vectors and
// FP64 dot products and norms (two-stage deterministic reductions); then
// v_a -= dt / (rho dx) (p_hi - p_lo) on every non-wall face next to a fluid
// cell.  alpha and beta are formed on the device; the host reads the
// residual norm every kCheckEvery iterations.
#include <cmath>

#include "pcg.cuh"

namespace polypic {

constexpr int kPcgThreads = 256;
constexpr int kPcgMaxBlocks = 1024;
constexpr int kCheckEvery = 8;

struct PcgBuffers {
    float *x, *r, *z, *d, *Ap, *diag;
    uint8_t *fluid;
    double *partial;  // [2][kPcgMaxBlocks]
    double *scal;     // rz, rz_new, pAp, rr, bb, alpha, beta
};
enum { kRz = 0, kRzNew = 1, kPAp = 2, kRr = 3, kBb = 4 };

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

__global__ void __launch_bounds__(kPcgThreads) k_setup(GridGeom g, int64_t num_keys,
                                                       const uint32_t *__restrict__ cs,
                                                       const float *__restrict__ v0,
                                                       const float *__restrict__ v1,
                                                       const float *__restrict__ v2, float scale,
                                                       PcgBuffers B) {
    const int64_t nc = (int64_t)g.n[0] * g.n[1] * g.n[2];
    double rz = 0.0, bb = 0.0;
    for (int64_t c = (int64_t)blockIdx.x * kPcgThreads + threadIdx.x; c < nc;
         c += (int64_t)gridDim.x * kPcgThreads) {
        const int i = (int)(c % g.n[0]), j = (int)((c / g.n[0]) % g.n[1]),
                  k = (int)(c / ((int64_t)g.n[0] * g.n[1]));
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
        B.x[c] = 0.0f;
        B.r[c] = b;
        const float z = fl ? b / dg : 0.0f;
        B.z[c] = z;
        B.d[c] = z;
        rz += (double)b * (double)z;
        bb += (double)b * (double)b;
    }
    block_sum2(rz, bb, B.partial);
}

__global__ void __launch_bounds__(kPcgThreads) k_apply(GridGeom g, PcgBuffers B) {
    const int64_t nc = (int64_t)g.n[0] * g.n[1] * g.n[2];
    double pap = 0.0;
    for (int64_t c = (int64_t)blockIdx.x * kPcgThreads + threadIdx.x; c < nc;
         c += (int64_t)gridDim.x * kPcgThreads) {
        float s = 0.0f;
        if (B.fluid[c]) {
            const int i = (int)(c % g.n[0]), j = (int)((c / g.n[0]) % g.n[1]),
                      k = (int)(c / ((int64_t)g.n[0] * g.n[1]));
            s = B.diag[c] * B.d[c];
            if (i > 0 && B.fluid[c - 1]) s -= B.d[c - 1];
            if (i < g.n[0] - 1 && B.fluid[c + 1]) s -= B.d[c + 1];
            if (j > 0 && B.fluid[c - g.n[0]]) s -= B.d[c - g.n[0]];
            if (j < g.n[1] - 1 && B.fluid[c + g.n[0]]) s -= B.d[c + g.n[0]];
            const int64_t sl = (int64_t)g.n[0] * g.n[1];
            if (k > 0 && B.fluid[c - sl]) s -= B.d[c - sl];
            if (k < g.n[2] - 1 && B.fluid[c + sl]) s -= B.d[c + sl];
        }
        B.Ap[c] = s;
        pap += (double)B.d[c] * (double)s;
    }
    block_sum2(pap, 0.0, B.partial);
}

__global__ void __launch_bounds__(kPcgThreads) k_update(GridGeom g, PcgBuffers B) {
    const int64_t nc = (int64_t)g.n[0] * g.n[1] * g.n[2];
    const double pap = B.scal[kPAp];
    const float alpha = pap != 0.0 ? (float)(B.scal[kRz] / pap) : 0.0f;
    double rz = 0.0, rr = 0.0;
    for (int64_t c = (int64_t)blockIdx.x * kPcgThreads + threadIdx.x; c < nc;
         c += (int64_t)gridDim.x * kPcgThreads) {
        if (!B.fluid[c]) continue;
        B.x[c] = fmaf(alpha, B.d[c], B.x[c]);
        const float r = fmaf(-alpha, B.Ap[c], B.r[c]);
        B.r[c] = r;
        const float z = r / B.diag[c];
        B.z[c] = z;
        rz += (double)r * (double)z;
        rr += (double)r * (double)r;
    }
    block_sum2(rz, rr, B.partial);
}

__global__ void __launch_bounds__(kPcgThreads) k_direction(GridGeom g, PcgBuffers B) {
    const int64_t nc = (int64_t)g.n[0] * g.n[1] * g.n[2];
    const double rz_old = B.scal[kRz], rz_new = B.scal[kRzNew];
    const float beta = rz_old != 0.0 ? (float)(rz_new / rz_old) : 0.0f;
    for (int64_t c = (int64_t)blockIdx.x * kPcgThreads + threadIdx.x; c < nc;
         c += (int64_t)gridDim.x * kPcgThreads)
        if (B.fluid[c]) B.d[c] = fmaf(beta, B.d[c], B.z[c]);
}

__global__ void k_rotate(double *scal) { scal[kRz] = scal[kRzNew]; }

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
        const int i = (int)(f % dX), j = (int)((f / dX) % dY), k = (int)(f / ((int64_t)dX * dY));
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
    return nc * (6 * sizeof(float) + 1) + (2 * kPcgMaxBlocks + 16) * sizeof(double) + 8 * 256;
}

polypic_status pcg_project(const GridGeom &g, int64_t num_keys, const uint32_t *cell_start,
                           float *vel[3], float dt, float rho, int maxiter, double rtol,
                           uint32_t *status, Workspace &ws, cudaStream_t s) {
    (void)num_keys;
    const int64_t nc = (int64_t)g.n[0] * g.n[1] * g.n[2];
    PcgBuffers B;
    B.x = ws.take<float>(nc);
    B.r = ws.take<float>(nc);
    B.z = ws.take<float>(nc);
    B.d = ws.take<float>(nc);
    B.Ap = ws.take<float>(nc);
    B.diag = ws.take<float>(nc);
    B.fluid = ws.take<uint8_t>(nc);
    B.partial = ws.take<double>(2 * kPcgMaxBlocks);
    B.scal = ws.take<double>(16);
    if (ws.overflow) return POLYPIC_ERR_WORKSPACE;
    const int nb = (int)std::min<int64_t>(kPcgMaxBlocks, (nc + kPcgThreads - 1) / kPcgThreads);
    const double gdx = (double)g.dx;
    // rhs = -(rho dx^2 / dt) div with div = (sum of face differences) / dx
    const float scale = (float)((double)rho * gdx / (double)dt);

    auto ok = [&]() { return cudaGetLastError() == cudaSuccess; };
    k_setup<<<nb, kPcgThreads, 0, s>>>(g, num_keys, cell_start, vel[0], vel[1], vel[2], scale, B);
    k_final<<<1, kPcgThreads, 0, s>>>(B.partial, nb, B.scal, kRz, kBb);
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
        for (int b = 0; b < batch; ++b) {
            k_apply<<<nb, kPcgThreads, 0, s>>>(g, B);
            k_final<<<1, kPcgThreads, 0, s>>>(B.partial, nb, B.scal, kPAp, -1);
            k_update<<<nb, kPcgThreads, 0, s>>>(g, B);
            k_final<<<1, kPcgThreads, 0, s>>>(B.partial, nb, B.scal, kRzNew, kRr);
            k_direction<<<nb, kPcgThreads, 0, s>>>(g, B);
            k_rotate<<<1, 1, 0, s>>>(B.scal);
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

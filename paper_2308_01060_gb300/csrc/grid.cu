// grid.cu -- grid velocity update and its adjoint (face-parallel, HBM bound).
//
// The paper leaves the grid update to the host simulator (Section 3); this is
// the minimal documented form:  v = mv/m where m > 0 else 0 (Eqs 5, 20),
// v~ = v + dt g, optional implicit two-phase drag between the fluid and solid
// grids, and zero normal velocity on the wall faces.
#include "grid.cuh"

namespace polypic {

__global__ void __launch_bounds__(256) k_grid_update(GridUpdateArgs U) {
    const int a = blockIdx.y;
    const GridGeom &g = U.g;
    const int dX = g.n[0] + (a == 0), dY = g.n[1] + (a == 1), dZ = g.n[2] + (a == 2);
    const int64_t total = (int64_t)dX * dY * dZ;
    const float ga = U.gravity[a];
    const float *fm = U.fm[a], *fp = U.fp[a];
    float *fv = U.fv[a];
    const float *sm = U.sm[a], *sp = U.sp[a];
    float *sv = U.sv[a];
    const int na = g.n[a];
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int ia = a == 0 ? (int)(idx % dX) : a == 1 ? (int)((idx / dX) % dY)
                                                         : (int)(idx / ((int64_t)dX * dY));
        const bool wall = ia == 0 || ia == na;
        const float m = fm[idx];
        float v = m > 0.0f ? fp[idx] / m : 0.0f;
        v = fmaf(U.dt, ga, v);
        if (sm) {
            const float ms = sm[idx];
            float vs = ms > 0.0f ? sp[idx] / ms : 0.0f;
            vs = fmaf(U.dt, ga, vs);
            if (m > 0.0f && ms > 0.0f && U.drag_k > 0.0f) {
                const float mtot = m + ms;
                const float mean = (m * v + ms * vs) / mtot;
                const float u = (v - vs) / (1.0f + U.dt * U.drag_k * (1.0f / m + 1.0f / ms));
                v = mean + (ms / mtot) * u;
                vs = mean - (m / mtot) * u;
            }
            sv[idx] = wall ? 0.0f : vs;
        }
        fv[idx] = wall ? 0.0f : v;
    }
}

// Adjoint of the single-phase update: lp = lv / m, lm = -lv mv / m^2 on
// non-wall faces with m > 0, else 0.
__global__ void __launch_bounds__(256) k_grid_update_adjoint(GridAdjointArgs U) {
    const int a = blockIdx.y;
    const GridGeom &g = U.g;
    const int dX = g.n[0] + (a == 0), dY = g.n[1] + (a == 1), dZ = g.n[2] + (a == 2);
    const int64_t total = (int64_t)dX * dY * dZ;
    const int na = g.n[a];
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int ia = a == 0 ? (int)(idx % dX) : a == 1 ? (int)((idx / dX) % dY)
                                                         : (int)(idx / ((int64_t)dX * dY));
        const bool wall = ia == 0 || ia == na;
        const float m = U.fm[a][idx];
        float lm = 0.0f, lp = 0.0f;
        if (!wall && m > 0.0f) {
            const float lv = U.lv[a][idx];
            lp = lv / m;
            lm = -lp * (U.fp[a][idx] / m);
        }
        U.lm[a][idx] = lm;
        U.lp[a][idx] = lp;
    }
}

static dim3 face_grid(const GridGeom &g) {
    int64_t tot = (int64_t)(g.n[0] + 1) * (g.n[1] + 1) * (g.n[2] + 1);
    int64_t nb = (tot + 255) / 256;
    return dim3((unsigned)(nb < 152 * 32 ? nb : 152 * 32), 3, 1);
}

cudaError_t grid_update(const GridUpdateArgs &U, cudaStream_t s) {
    k_grid_update<<<face_grid(U.g), 256, 0, s>>>(U);
    return cudaGetLastError();
}

cudaError_t grid_update_adjoint(const GridAdjointArgs &U, cudaStream_t s) {
    k_grid_update_adjoint<<<face_grid(U.g), 256, 0, s>>>(U);
    return cudaGetLastError();
}

}  // namespace polypic

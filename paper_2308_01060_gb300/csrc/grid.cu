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

// Adjoint of the update, per face, last step first: walls (no gradient on
// wall faces); with a solid grid and drag_k > 0 on faces holding both masses,
// the transposed Jacobian of (v_f, v_s) -> (v_f', v_s') and the drag's
// derivatives in m_f and m_s; gravity (identity); v = mv/m: lp = lv / m,
// lm += -lv mv / m^2 where m > 0, else 0.  The projection's transpose has
// been applied to lv beforehand.
__global__ void __launch_bounds__(256) k_grid_update_adjoint(GridAdjointArgs U) {
    const int a = blockIdx.y;
    const GridGeom &g = U.g;
    const int dX = g.n[0] + (a == 0), dY = g.n[1] + (a == 1), dZ = g.n[2] + (a == 2);
    const int64_t total = (int64_t)dX * dY * dZ;
    const int na = g.n[a];
    const bool solid = U.sm[a] != nullptr;
    const float ga = U.gravity[a];
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int ia = a == 0 ? (int)(idx % dX) : a == 1 ? (int)((idx / dX) % dY)
                                                         : (int)(idx / ((int64_t)dX * dY));
        const bool wall = ia == 0 || ia == na;
        const float mf = U.fm[a][idx];
        const float ms = solid ? U.sm[a][idx] : 0.0f;
        float lvf = wall ? 0.0f : U.lv[a][idx];
        float lvs = (solid && !wall) ? U.lsv[a][idx] : 0.0f;
        float dmf = 0.0f, dms = 0.0f;
        if (solid && U.drag_k > 0.0f && mf > 0.0f && ms > 0.0f) {
            const float vf = fmaf(U.dt, ga, U.fp[a][idx] / mf);
            const float vs = fmaf(U.dt, ga, U.sp[a][idx] / ms);
            const float M = mf + ms, wa = ms / M, wb = mf / M;
            const float Dd = 1.0f + U.dt * U.drag_k * (1.0f / mf + 1.0f / ms);
            const float u = (vf - vs) / Dd, mean = wb * vf + wa * vs;
            const float iM2 = 1.0f / (M * M);
            const float mean_f = (vf - mean) / M, mean_s = (vs - mean) / M;
            const float wa_f = -ms * iM2, wa_s = mf * iM2;
            const float wb_f = ms * iM2, wb_s = -mf * iM2;
            const float c = u * U.dt * U.drag_k / Dd;
            const float u_f = c / (mf * mf), u_s = c / (ms * ms);
            dmf = lvf * (mean_f + wa_f * u + wa * u_f) + lvs * (mean_f - wb_f * u - wb * u_f);
            dms = lvf * (mean_s + wa_s * u + wa * u_s) + lvs * (mean_s - wb_s * u - wb * u_s);
            const float nf = lvf * (wb + wa / Dd) + lvs * (wb - wb / Dd);
            const float ns = lvf * (wa - wa / Dd) + lvs * (wa + wb / Dd);
            lvf = nf;
            lvs = ns;
        }
        float lm = 0.0f, lp = 0.0f;
        if (mf > 0.0f) {
            lp = lvf / mf;
            lm = dmf - lp * (U.fp[a][idx] / mf);
        }
        U.lm[a][idx] = lm;
        U.lp[a][idx] = lp;
        if (solid) {
            float sm_ = 0.0f, sp_ = 0.0f;
            if (ms > 0.0f) {
                sp_ = lvs / ms;
                sm_ = dms - sp_ * (U.sp[a][idx] / ms);
            }
            U.lsm[a][idx] = sm_;
            U.lsp[a][idx] = sp_;
        }
    }
}

struct WallCopyArgs {
    GridGeom g;
    const float *src[3];
    float *dst[3];
};

__global__ void __launch_bounds__(256) k_wall_zeroed_copy(WallCopyArgs W) {
    const int a = blockIdx.y;
    const GridGeom &g = W.g;
    const int dX = g.n[0] + (a == 0), dY = g.n[1] + (a == 1), dZ = g.n[2] + (a == 2);
    const int64_t total = (int64_t)dX * dY * dZ;
    const int na = g.n[a];
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int ia = a == 0 ? (int)(idx % dX) : a == 1 ? (int)((idx / dX) % dY)
                                                         : (int)(idx / ((int64_t)dX * dY));
        W.dst[a][idx] = (ia == 0 || ia == na) ? 0.0f : W.src[a][idx];
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

cudaError_t wall_zeroed_copy(const GridGeom &g, const float *const src[3], float *const dst[3],
                             cudaStream_t s) {
    WallCopyArgs W{};
    W.g = g;
    for (int a = 0; a < 3; ++a) {
        W.src[a] = src[a];
        W.dst[a] = dst[a];
    }
    k_wall_zeroed_copy<<<face_grid(g), 256, 0, s>>>(W);
    return cudaGetLastError();
}

}  // namespace polypic

// fabric.cu -- stand-ins for what the paper takes from Fei et al.: the sheet's
// mechanics (a mass-spring lattice on the vertex particles) and the absorption
// of fluid mass into the solid's m_abs (Eqs 18-20 take m_abs as given).
//
// Forces: vertex (i, k) of the m x m lattice has id k m + i (ids >= m^2 are
// element particles, no springs).  Springs to the neighbours at (+-1, 0),
// (0, +-1) [stretch, rest h], (+-1, +-1) [shear, rest h sqrt 2], (+-2, 0),
// (0, +-2) [bend, rest 2h]; with d = x_j - x_i, L = |d|, e = d / L the force
// on i is k (L - L0) e + c ((v_j - v_i) . e) e, and v_i = c_i0 takes the step
// v_i += dt f / (m_i + m_abs,i).  The particle arrays are in slot order, so a
// scatter first maps each lattice id to its slot; all velocities are read
// before any is written (the new ones go to scratch).
//
// Absorption: warp per block of 32 keys, lane per cell, walking both phases'
// block-interleaved slots round by round (round r holds the r-th particle of
// every key with more than r particles).  Per cell: M_f = sum of the fluid
// masses, solid demand d_p = min(rate dt m_s, max(0, capacity m_s - m_abs)),
// D = min(sum d, max_fraction M_f); the solid gains d_p D / sum d, each fluid
// particle loses m_q D / M_f.  Sums run in slot order: deterministic.
#include "fabric.cuh"

namespace polypic {

namespace {

constexpr int kThreads = 256;
constexpr uint32_t kNoSlot = 0xffffffffu;

__global__ void __launch_bounds__(kThreads) k_fill_u32(uint32_t *p, int64_t n, uint32_t v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

__global__ void __launch_bounds__(kThreads) k_slot_of(const uint32_t *id, int64_t count,
                                                      uint32_t nv, uint32_t *slot_of) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < count;
         j += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t v = id[j];
        if (v < nv) slot_of[v] = (uint32_t)j;
    }
}

struct ForceArgs {
    int64_t count;
    const float *x[3];
    const float *mass, *mass_abs;
    float *vel[3];         // mode 0 of each component: coeff + a R count
    const uint32_t *id, *slot_of;
    float *vnew[3];
    int m;
    float h, k_stretch, k_shear, k_bend, damping, dt;
};

__global__ void __launch_bounds__(kThreads) k_fabric_forces(ForceArgs F) {
    const int oi[12] = {1, -1, 0, 0, 1, 1, -1, -1, 2, -2, 0, 0};
    const int ok[12] = {0, 0, 1, -1, 1, -1, 1, -1, 0, 0, 2, -2};
    const uint32_t nv = (uint32_t)F.m * (uint32_t)F.m;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < F.count;
         j += (int64_t)gridDim.x * blockDim.x) {
        const float vx = F.vel[0][j], vy = F.vel[1][j], vz = F.vel[2][j];
        const uint32_t v = F.id[j];
        if (v >= nv) {
            F.vnew[0][j] = vx;
            F.vnew[1][j] = vy;
            F.vnew[2][j] = vz;
            continue;
        }
        const int i = (int)(v % (uint32_t)F.m), k = (int)(v / (uint32_t)F.m);
        const float px = F.x[0][j], py = F.x[1][j], pz = F.x[2][j];
        float fx = 0.0f, fy = 0.0f, fz = 0.0f;
#pragma unroll
        for (int s = 0; s < 12; ++s) {
            const int i2 = i + oi[s], k2 = k + ok[s];
            if (i2 < 0 || i2 >= F.m || k2 < 0 || k2 >= F.m) continue;
            const uint32_t q = F.slot_of[(uint32_t)k2 * (uint32_t)F.m + (uint32_t)i2];
            if (q == kNoSlot) continue;
            const float kk = s < 4 ? F.k_stretch : s < 8 ? F.k_shear : F.k_bend;
            const float L0 = s < 4 ? F.h : s < 8 ? F.h * 1.41421356f : 2.0f * F.h;
            const float dx = F.x[0][q] - px, dy = F.x[1][q] - py, dz = F.x[2][q] - pz;
            const float L = sqrtf(dx * dx + dy * dy + dz * dz);
            if (!(L > 0.0f)) continue;
            const float iL = 1.0f / L;
            const float ex = dx * iL, ey = dy * iL, ez = dz * iL;
            const float rv = (F.vel[0][q] - vx) * ex + (F.vel[1][q] - vy) * ey +
                             (F.vel[2][q] - vz) * ez;
            const float mag = kk * (L - L0) + F.damping * rv;
            fx += mag * ex;
            fy += mag * ey;
            fz += mag * ez;
        }
        const float mt = F.mass[j] + (F.mass_abs ? F.mass_abs[j] : 0.0f);
        const float s = F.dt / mt;
        F.vnew[0][j] = vx + s * fx;
        F.vnew[1][j] = vy + s * fy;
        F.vnew[2][j] = vz + s * fz;
    }
}

__global__ void __launch_bounds__(kThreads) k_store_velocity(ForceArgs F) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < F.count;
         j += (int64_t)gridDim.x * blockDim.x) {
        F.vel[0][j] = F.vnew[0][j];
        F.vel[1][j] = F.vnew[1][j];
        F.vel[2][j] = F.vnew[2][j];
    }
}

struct AbsorbArgs {
    int64_t num_blocks;               // key blocks of 32
    const uint32_t *fcs, *fperm;      // fluid cell_start, perm
    const uint32_t *scs, *sperm;      // solid cell_start, perm
    float *fmass;
    const float *smass;
    float *mass_abs;
    float want_per_mass;              // rate dt
    float capacity, max_fraction;
};

__device__ __forceinline__ float demand(float ms, float mabs, float want_per_mass, float cap) {
    const float room = cap * ms - mabs;
    const float want = want_per_mass * ms;
    return room > 0.0f ? fminf(want, room) : 0.0f;
}

// One warp per block of 32 keys, lane = key.  `walk` visits the lane's
// particles of one phase in slot order (round by round) and calls f(index).
template <class F>
__device__ __forceinline__ void walk(const uint32_t *cs, const uint32_t *perm, uint32_t key0,
                                     uint32_t lane, F &&f) {
    const uint32_t lo = cs[key0 + lane], hi = cs[key0 + lane + 1];
    const uint32_t cnt = hi - lo;
    const uint32_t rounds = __reduce_max_sync(0xffffffffu, cnt);
    uint32_t base = cs[key0];
    const uint32_t below = (1u << lane) - 1u;
    for (uint32_t r = 0; r < rounds; ++r) {
        const uint32_t live = __ballot_sync(0xffffffffu, cnt > r);
        if (cnt > r) f(perm[base + __popc(live & below)]);
        base += __popc(live);
    }
}

__global__ void __launch_bounds__(kThreads) k_absorb(AbsorbArgs A) {
    const uint32_t lane = threadIdx.x & 31u;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
    for (int64_t b = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32; b < A.num_blocks;
         b += warps) {
        const uint32_t key0 = (uint32_t)b * 32u;
        // blocks without both phases do nothing (warp-uniform tests)
        if (A.scs[key0] == A.scs[key0 + 32] || A.fcs[key0] == A.fcs[key0 + 32]) continue;
        float Mf = 0.0f, Dd = 0.0f;
        walk(A.fcs, A.fperm, key0, lane, [&](uint32_t q) { Mf += A.fmass[q]; });
        walk(A.scs, A.sperm, key0, lane, [&](uint32_t p) {
            Dd += demand(A.smass[p], A.mass_abs[p], A.want_per_mass, A.capacity);
        });
        const float D = fminf(Dd, A.max_fraction * Mf);
        const bool act = D > 0.0f;
        if (!__any_sync(0xffffffffu, act)) continue;
        const float gain = act ? D / Dd : 0.0f, loss = act ? D / Mf : 0.0f;
        walk(A.scs, A.sperm, key0, lane, [&](uint32_t p) {
            if (act) A.mass_abs[p] += demand(A.smass[p], A.mass_abs[p], A.want_per_mass,
                                             A.capacity) * gain;
        });
        walk(A.fcs, A.fperm, key0, lane, [&](uint32_t q) {
            if (act) A.fmass[q] -= A.fmass[q] * loss;
        });
    }
}

__global__ void __launch_bounds__(kThreads) k_gather_ids(const uint32_t *in, const uint32_t *perm,
                                                         int64_t count, uint32_t *out) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < count;
         j += (int64_t)gridDim.x * blockDim.x)
        out[j] = in[perm[j]];
}

unsigned blocks_for(int64_t n) {
    int64_t b = (n + kThreads - 1) / kThreads;
    if (b < 1) b = 1;
    return (unsigned)(b < 152 * 16 ? b : 152 * 16);
}

}  // namespace

size_t fabric_scratch_bytes(int64_t count, int m) {
    return (size_t)count * 3 * sizeof(float) + (size_t)m * m * sizeof(uint32_t) + 3 * 256;
}

cudaError_t fabric_forces(const FabricForceArgs &a, Workspace &ws, cudaStream_t s) {
    const int64_t nv = (int64_t)a.m * a.m;
    uint32_t *slot_of = ws.take<uint32_t>((size_t)nv);
    ForceArgs F{};
    F.count = a.count;
    for (int c = 0; c < 3; ++c) {
        F.x[c] = a.x[c];
        F.vel[c] = a.vel[c];
        F.vnew[c] = ws.take<float>((size_t)a.count);
    }
    if (ws.overflow) return cudaErrorInvalidValue;
    F.mass = a.mass;
    F.mass_abs = a.mass_abs;
    F.id = a.id;
    F.slot_of = slot_of;
    F.m = a.m;
    F.h = a.h;
    F.k_stretch = a.k_stretch;
    F.k_shear = a.k_shear;
    F.k_bend = a.k_bend;
    F.damping = a.damping;
    F.dt = a.dt;
    k_fill_u32<<<blocks_for(nv), kThreads, 0, s>>>(slot_of, nv, kNoSlot);
    k_slot_of<<<blocks_for(a.count), kThreads, 0, s>>>(a.id, a.count, (uint32_t)nv, slot_of);
    k_fabric_forces<<<blocks_for(a.count), kThreads, 0, s>>>(F);
    k_store_velocity<<<blocks_for(a.count), kThreads, 0, s>>>(F);
    return cudaGetLastError();
}

cudaError_t absorb(const AbsorbCall &a, cudaStream_t s) {
    AbsorbArgs A{};
    A.num_blocks = a.num_keys / 32;
    A.fcs = a.fluid_cell_start;
    A.fperm = a.fluid_perm;
    A.scs = a.solid_cell_start;
    A.sperm = a.solid_perm;
    A.fmass = a.fluid_mass;
    A.smass = a.solid_mass;
    A.mass_abs = a.mass_abs;
    A.want_per_mass = a.rate * a.dt;
    A.capacity = a.capacity;
    A.max_fraction = a.max_fraction;
    const int64_t ctas = (A.num_blocks + 7) / 8;
    k_absorb<<<(unsigned)(ctas < 152 * 16 ? (ctas > 0 ? ctas : 1) : 152 * 16), kThreads, 0, s>>>(A);
    return cudaGetLastError();
}

cudaError_t gather_ids(const uint32_t *in, const uint32_t *perm, int64_t count, uint32_t *out,
                       cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    k_gather_ids<<<blocks_for(count), kThreads, 0, s>>>(in, perm, count, out);
    return cudaGetLastError();
}

}  // namespace polypic

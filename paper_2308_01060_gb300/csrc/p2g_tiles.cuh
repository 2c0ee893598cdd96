// p2g_tiles.cuh -- the P2G tile kernel of block-interleaved phases (its
// per-particle pieces are in p2g_kernel.cuh) and its launcher.  Each
// instantiation is compiled in one of the p2g_tiles_*.cu translation units,
// so that the heavy 27-mode variants build in parallel.
//
// Work decomposition (no float atomics, bit-identical from run to run): one
// CTA per 8x8x4-cell tile, one warp per 4x4x2-cell block, one lane per cell;
// a lane accumulates its cell's 4 x 3 x 3 footprint of face grid A in
// registers over the rounds of the three component passes, the warp adds the
// 32 footprints into its block region in 36 node-offset phases, and the CTA
// adds the 8 block regions into the tile region in ascending block order.
#pragma once
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

template <int R, bool AFF = false, int FMT = POLYPIC_COEFF_F32> constexpr int p2g_smem_bytes() {
    return (kP2GWarps * kRegionFloats + kP2GWarps * kStages * Stage<R, AFF, FMT>::NV * 32) * 4;
}
static_assert(p2g_smem_bytes<27, true>() <= 227 * 1024,
              "P2G staging exceeds the shared memory of a CTA");

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
    using S = Stage<R, AFF, FMT>;
    const bool interior = gi >= 1 && gi <= P.g.n[0] - 2 && gj >= 1 && gj <= P.g.n[1] - 2 &&
                          gk >= 1 && gk <= P.g.n[2] - 2;
    Foot F;
    F.zero();
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
                                           av_.guard, aw.guard, F, au.t, av_.t, aw.t);
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
                rm[idx] += F.m(d, kv, kw);
                rv[idx] += F.v(d, kv, kw);
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
        pipe_issue<R, FMT, ADJ, AFF>(P, q, bs, n_c, maxn, lt, stage + k * Stage<R, AFF, FMT>::NV * 32,
                                     lane);
    p2g_pass<R, FMT, 0, ADJ, AFF>(P, q, bs, n_c, maxn, ci, cj, ck, gi, gj, gk, lane, reg, stage, bad);
    p2g_pass<R, FMT, 1, ADJ, AFF>(P, q, bs, n_c, maxn, ci, cj, ck, gi, gj, gk, lane, reg, stage, bad);
    p2g_pass<R, FMT, 2, ADJ, AFF>(P, q, bs, n_c, maxn, ci, cj, ck, gi, gj, gk, lane, reg, stage, bad);
    cp_async_wait<0>();
}

// ---------------------------------------------------------------- lane teams
// For phases whose blocks hold few live cells (a sheet crosses a 4x4x2-cell
// block in one layer: 8 of its 32 cells), k_p2g_tiles<..., TEAMS = true>
// schedules the lanes in two phases instead of one lane per cell throughout.
// Phase 1 (steps 0 .. K-1): every lane takes rounds 0 .. K-1 of its own cell.
// Then the lanes whose cells are done merge their footprints (one partial
// 36-phase merge) and join teams: the cell of a lane with e = n - K > 0
// rounds left takes 1 + floor(f e / E) members (f free lanes, E the excess of
// all cells), member j doing rounds K + j, K + j + t, ... of that cell
// (phase 2).  At the end of a pass member j of every team merges in merge
// pass j, so no two lanes of one merge pass share a cell and the merges stay
// conflict-free; every sum's order follows from the counts alone
// (deterministic).  K minimises the steps plus a quarter round per merge and
// is chosen once per block; blocks of fewer than 4 or more than 64 rounds keep
// one lane per cell.  Phase 2 reads its slots from per-warp tables of the
// round offsets and live masks.
constexpr uint32_t kTeamMaxRounds = 64;

struct Teams {
    uint32_t K, steps;           // phase-1 steps; phase 1 + phase 2 steps
    bool two;                    // phase 2 exists
    bool heavy;                  // the lane's own cell continues in phase 2
    int tc;                      // the lane's phase-2 cell (lane index), -1: idle
    uint32_t member, tsize, tn;  // member index, team size, rounds of the phase-2 cell
    uint32_t maxt;               // largest team
};

__device__ __forceinline__ Teams make_teams(uint32_t n_c, uint32_t maxn, int lane, uint32_t *tabS,
                                            uint32_t *tabM) {
    Teams s;
    s.K = maxn;
    s.steps = maxn;
    s.two = false;
    s.heavy = false;
    s.tc = lane;
    s.member = 0;
    s.tsize = 1;
    s.tn = n_c;
    s.maxt = 0;
    if (maxn < 4 || maxn > kTeamMaxRounds) return s;  // warp-uniform
    // cost in quarter rounds: 4 (K + phase-2 steps) + the merge passes
    uint32_t bestK = maxn, bestc = 4 * maxn + 1;
    for (uint32_t K = 1; K < maxn; ++K) {
        const uint32_t e = n_c > K ? n_c - K : 0u;
        const uint32_t E = __reduce_add_sync(0xffffffffu, e);
        const uint32_t f = 32u - (uint32_t)__popc(__ballot_sync(0xffffffffu, e > 0));
        const uint32_t t = e > 0 ? 1u + (f * e) / E : 0u;
        const uint32_t p2 = e > 0 ? (e + t - 1) / t : 0u;
        const uint32_t c = 4 * (K + __reduce_max_sync(0xffffffffu, p2)) + 2 +
                           __reduce_max_sync(0xffffffffu, t);
        if (c < bestc) {
            bestc = c;
            bestK = K;
        }
    }
    if (bestK == maxn) return s;
    for (uint32_t q = bestK; q < maxn; ++q) {
        const uint32_t sq = __reduce_add_sync(0xffffffffu, min(n_c, q));
        const uint32_t mq = __ballot_sync(0xffffffffu, n_c > q);
        if (lane == 0) {
            tabS[q] = sq;
            tabM[q] = mq;
        }
    }
    __syncwarp();
    const uint32_t K = bestK;
    const uint32_t e = n_c > K ? n_c - K : 0u;
    const uint32_t E = __reduce_add_sync(0xffffffffu, e);
    const unsigned hm = __ballot_sync(0xffffffffu, e > 0);
    const uint32_t f = 32u - (uint32_t)__popc(hm);
    const uint32_t t = e > 0 ? 1u + (f * e) / E : 0u;
    const uint32_t extra = e > 0 ? t - 1 : 0u;
    uint32_t incl = extra;  // inclusive prefix of the helpers taken, in lane order
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    const uint32_t off = incl - extra;
    const uint32_t p2 = e > 0 ? (e + t - 1) / t : 0u;
    s.K = K;
    s.steps = K + __reduce_max_sync(0xffffffffu, p2);
    s.maxt = __reduce_max_sync(0xffffffffu, t);
    s.two = true;
    s.heavy = e > 0;
    if (s.heavy) s.tsize = t;
    else s.tc = -1;
    // a free lane of rank rho joins the team whose helper range holds rho
    // (the shuffles run on every lane: they name the whole warp)
    const uint32_t rho = (uint32_t)__popc(~hm & ((1u << lane) - 1u));
    for (int h = 0; h < 32; ++h) {
        const uint32_t oh = __shfl_sync(0xffffffffu, off, h);
        const uint32_t xh = __shfl_sync(0xffffffffu, extra, h);
        const uint32_t th = __shfl_sync(0xffffffffu, t, h);
        const uint32_t nh = __shfl_sync(0xffffffffu, n_c, h);
        if (!s.heavy && xh > 0 && rho >= oh && rho < oh + xh) {
            s.tc = h;
            s.member = rho - oh + 1;
            s.tsize = th;
            s.tn = nh;
        }
    }
    return s;
}

// The stream of steps through the stage ring, as Pipe, over the schedule's
// steps: phase-1 slots from round_slot, phase-2 slots from the tables.
struct TeamPipe {
    int ia;
    uint32_t ir, sn, pn;
    bool ok;
    int ring;
};

__device__ __forceinline__ void team_locate(const P2GArgs &P, const Teams &sc, TeamPipe &q,
                                            uint32_t bs, uint32_t be, uint32_t n_c, unsigned lt,
                                            int lane, const uint32_t *tabS,
                                            const uint32_t *tabM) {
    if (q.ir < sc.K) {  // warp-uniform: phase 1, every lane calls round_slot
        q.sn = round_slot(bs, n_c, q.ir, lt);
        q.ok = n_c > q.ir;
    } else {
        const uint32_t r = sc.K + sc.member + (q.ir - sc.K) * sc.tsize;
        q.ok = sc.tc >= 0 && r < sc.tn;
        q.sn = q.ok ? bs + tabS[r] + (uint32_t)__popc(tabM[r] & ((1u << sc.tc) - 1u)) : 0u;
        if (q.ok && q.sn >= be) {  // outside the block's slots: record, skip
            atomicOr(P.status, kFlagOutOfDomain);
            q.ok = false;
        }
    }
    q.pn = q.ok ? P.perm[q.sn] : 0u;
}

template <int R, int FMT, bool ADJ, bool AFF>
__device__ __forceinline__ void team_issue(const P2GArgs &P, const Teams &sc, TeamPipe &q,
                                           uint32_t bs, uint32_t be, uint32_t n_c, unsigned lt,
                                           float *st, int lane, const uint32_t *tabS,
                                           const uint32_t *tabM) {
    if (q.ia < 3 && q.ok) {  // q.ia is warp-uniform
        if (q.ia == 0) stage_particle<R, FMT, 0, ADJ, AFF>(P, q.pn, q.sn, st, lane);
        else if (q.ia == 1) stage_particle<R, FMT, 1, ADJ, AFF>(P, q.pn, q.sn, st, lane);
        else stage_particle<R, FMT, 2, ADJ, AFF>(P, q.pn, q.sn, st, lane);
    }
    cp_async_commit();
    if (q.ia < 3 && ++q.ir == sc.steps) {
        q.ir = 0;
        ++q.ia;
    }
    if (q.ia < 3) team_locate(P, sc, q, bs, be, n_c, lt, lane, tabS, tabM);
}

// Adds the footprints of the lanes with `on` set into block region A (the
// lane's cell at (ci, cj, ck) of the block), one node offset per phase.
template <int A>
__device__ __forceinline__ void merge_some(const Foot &F, int ci, int cj, int ck, float *reg,
                                           bool on) {
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
                if (on) {
                    rm[idx] += F.m(d, kv, kw);
                    rv[idx] += F.v(d, kv, kw);
                }
                __syncwarp();
            }
}

// One staged particle into the lane's footprint, checked against the cell
// (gi, gj, gk) it must lie in.
template <int R, int FMT, int A, bool ADJ, bool AFF>
__device__ __forceinline__ void team_consume(const P2GArgs &P, const float *st, int lane, int gi,
                                             int gj, int gk, Foot &F, bool &bad) {
    using S = Stage<R, AFF, FMT>;
    const float px = st[S::kX * 32 + lane], py = st[S::kY * 32 + lane], pz = st[S::kZ * 32 + lane];
    float mt = st[S::kM * 32 + lane];
    if (!ADJ && P.mass_abs) mt += st[S::kMabs * 32 + lane];
    const float v0 = cell_coord(px, P.g.inv_dx), v1 = cell_coord(py, P.g.inv_dx),
                v2 = cell_coord(pz, P.g.inv_dx);
    const bool ok = coord_valid(v0, P.g.n[0]) && coord_valid(v1, P.g.n[1]) &&
                    coord_valid(v2, P.g.n[2]) && (int)floorf(v0) == gi && (int)floorf(v1) == gj &&
                    (int)floorf(v2) == gk;
    if (ok) {
        const float vu = A == 0 ? v0 : (A == 1 ? v1 : v2);
        const float vv = A == 0 ? v1 : v0;
        const float vw = A == 2 ? v1 : v2;
        const Axis au = axis_decide(vu, true), av_ = axis_decide(vv, false),
                   aw = axis_decide(vw, false);
        const int cu = A == 0 ? gi : (A == 1 ? gj : gk);
        const int shift = au.base - (cu - 1);
        accumulate<R, FMT, A, ADJ, AFF>(P, st, lane, mt, shift, stencil_1d_scaled(au.t, P.s1, P.s2),
                                        stencil_1d_scaled(av_.t, P.s1, P.s2),
                                        stencil_1d_scaled(aw.t, P.s1, P.s2), au.guard, av_.guard,
                                        aw.guard, F, au.t, av_.t, aw.t);
    } else {
        bad = true;
    }
}

template <int R, int FMT, int A, bool ADJ, bool AFF>
__device__ __forceinline__ void team_pass(const P2GArgs &P, const Teams &sc, TeamPipe &q,
                                          uint32_t bs, uint32_t be, uint32_t n_c, int i0, int j0,
                                          int k0, int lane, float *reg, float *stage, bool &bad,
                                          const uint32_t *tabS, const uint32_t *tabM) {
    using S = Stage<R, AFF, FMT>;
    Foot F;
    F.zero();
    const unsigned lt = (1u << lane) - 1u;
    const int ci = lane & 3, cj = (lane >> 2) & 3, ck = lane >> 4;
    // phase 1: every lane on its own cell, round r at step r
    for (uint32_t r = 0; r < sc.K; ++r) {
        float *st = stage + q.ring * S::NV * 32;
        cp_async_wait<kStages - 1>();
        if (n_c > r)
            team_consume<R, FMT, A, ADJ, AFF>(P, st, lane, i0 + ci, j0 + cj, k0 + ck, F, bad);
        team_issue<R, FMT, ADJ, AFF>(P, sc, q, bs, be, n_c, lt, st, lane, tabS, tabM);
        q.ring = q.ring + 1 == kStages ? 0 : q.ring + 1;
    }
    if (!sc.two) {
        merge_some<A>(F, ci, cj, ck, reg, true);
        return;
    }
    // the lanes done with their cells merge them and join teams (phase 2)
    merge_some<A>(F, ci, cj, ck, reg, !sc.heavy);
    if (!sc.heavy) F.zero();
    const int tl = sc.tc >= 0 ? sc.tc : lane;
    const int ti = tl & 3, tj = (tl >> 2) & 3, tk = tl >> 4;
    for (uint32_t r = sc.K; r < sc.steps; ++r) {
        float *st = stage + q.ring * S::NV * 32;
        cp_async_wait<kStages - 1>();
        if (sc.tc >= 0 && sc.K + sc.member + (r - sc.K) * sc.tsize < sc.tn)
            team_consume<R, FMT, A, ADJ, AFF>(P, st, lane, i0 + ti, j0 + tj, k0 + tk, F, bad);
        team_issue<R, FMT, ADJ, AFF>(P, sc, q, bs, be, n_c, lt, st, lane, tabS, tabM);
        q.ring = q.ring + 1 == kStages ? 0 : q.ring + 1;
    }
    // merge pass j: member j of every team (distinct cells)
    for (uint32_t j = 0; j < sc.maxt; ++j)
        merge_some<A>(F, ti, tj, tk, reg, sc.tc >= 0 && sc.member == j);
}

// All three passes of one block under the team schedule.
template <int R, int FMT, bool ADJ, bool AFF>
__device__ __forceinline__ void team_block(const P2GArgs &P, uint32_t bs, uint32_t n_c,
                                           uint32_t maxn, uint32_t b, int lane, float *reg,
                                           float *stage, bool &bad, uint32_t *tabS,
                                           uint32_t *tabM) {
    const unsigned lt = (1u << lane) - 1u;
    const Teams sc = make_teams(n_c, maxn, lane, tabS, tabM);
    const uint32_t be = P.cell_start[b * 32 + 32];
    int i0, j0, k0;
    block_origin(P.g, b, i0, j0, k0);
    TeamPipe q;
    q.ia = 0;
    q.ir = 0;
    q.ring = 0;
    team_locate(P, sc, q, bs, be, n_c, lt, lane, tabS, tabM);
#pragma unroll
    for (int k = 0; k < kStages; ++k)
        team_issue<R, FMT, ADJ, AFF>(P, sc, q, bs, be, n_c, lt,
                                     stage + k * Stage<R, AFF, FMT>::NV * 32, lane, tabS, tabM);
    team_pass<R, FMT, 0, ADJ, AFF>(P, sc, q, bs, be, n_c, i0, j0, k0, lane, reg, stage, bad, tabS,
                                   tabM);
    team_pass<R, FMT, 1, ADJ, AFF>(P, sc, q, bs, be, n_c, i0, j0, k0, lane, reg, stage, bad, tabS,
                                   tabM);
    team_pass<R, FMT, 2, ADJ, AFF>(P, sc, q, bs, be, n_c, i0, j0, k0, lane, reg, stage, bad, tabS,
                                   tabM);
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

template <int R, int FMT, bool ADJ, bool AFF, bool TEAMS>
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
    float *stage = s_stage + warp * kStages * Stage<R, AFF, FMT>::NV * 32;
    if (lane == 0) s_empty[warp] = maxn == 0;
    if (maxn > 0) {
        for (int i = lane; i < kRegionFloats; i += 32) reg[i] = 0.0f;
        __syncwarp();
        int i0, j0, k0;
        block_origin(P.g, b, i0, j0, k0);
        const int ci = lane & 3, cj = (lane >> 2) & 3, ck = lane >> 4;
        const int gi = i0 + ci, gj = j0 + cj, gk = k0 + ck;
        bool bad = false;
        if constexpr (TEAMS) {
            __shared__ uint32_t s_tab[kP2GWarps][2][kTeamMaxRounds];
            team_block<R, FMT, ADJ, AFF>(P, bs, n_c, maxn, b, lane, reg, stage, bad,
                                         s_tab[warp][0], s_tab[warp][1]);
        } else {
            p2g_block<R, FMT, ADJ, AFF>(P, bs, n_c, maxn, ci, cj, ck, gi, gj, gk, lane, reg, stage,
                                        bad);
        }
        if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(P.status, kFlagOutOfDomain);
    }
    __syncthreads();
    float *dst = P.scratch + (size_t)tile * kTileFloats;
    merge_tile<0>(s_reg, s_empty, dst);
    merge_tile<1>(s_reg, s_empty, dst);
    merge_tile<2>(s_reg, s_empty, dst);
}

template <int R, int FMT, bool ADJ, bool AFF = false, bool TEAMS = false>
cudaError_t launch_tiles(const P2GArgs &P, int grid, cudaStream_t s) {
    const int smem = p2g_smem_bytes<R, AFF, FMT>();
    // the attribute is a property of the kernel in the current context; it is
    // set on every launch (a cheap host call), which keeps no state shared
    // between host threads or devices
    const cudaError_t e = cudaFuncSetAttribute(k_p2g_tiles<R, FMT, ADJ, AFF, TEAMS>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    k_p2g_tiles<R, FMT, ADJ, AFF, TEAMS><<<grid, kP2GWarps * 32, smem, s>>>(P);
    return cudaGetLastError();
}

// Launchers of the instantiations, one per translation unit.
cudaError_t launch_tiles_f32(const P2GArgs &P, int R, int grid, cudaStream_t s);
cudaError_t launch_tiles_16(const P2GArgs &P, int R, int fmt, int grid, cudaStream_t s);
cudaError_t launch_tiles_adj(const P2GArgs &P, int R, int grid, cudaStream_t s);
cudaError_t launch_tiles_aff(const P2GArgs &P, int R, int grid, cudaStream_t s);
// FP32 with the lane-team schedule (phases whose blocks hold few live cells)
cudaError_t launch_tiles_teams(const P2GArgs &P, int R, int grid, cudaStream_t s);

}  // namespace polypic

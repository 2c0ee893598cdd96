// api.cu -- the C ABI of libpolypic (declared in include/polypic.h).
//
// Every entry point validates its arguments on the host, lays the caller's
// workspace out, and launches kernels on the caller's stream.  No C++
// exception escapes (allocation uses nothrow); errors come back as
// polypic_status values.
#include <cmath>
#include <new>

#include "g2p.cuh"
#include "grid.cuh"
#include "p2g.cuh"
#include "pcg.cuh"
#include "adjoint.cuh"
#include "fabric.cuh"
#include "g2p2g.cuh"
#include "polypic_internal.cuh"
#include "sort.cuh"

using namespace polypic;

namespace {

polypic_status from_cuda(cudaError_t e) { return e == cudaSuccess ? POLYPIC_OK : POLYPIC_ERR_CUDA; }

bool valid_modes(int r) { return r == 1 || r == 4 || r == 8 || r == 27; }

int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }

int64_t face_count(const GridGeom &g, int a) {
    return (int64_t)(g.n[0] + (a == 0)) * (g.n[1] + (a == 1)) * (g.n[2] + (a == 2));
}

size_t face_bytes(const GridGeom &g) {
    size_t t = 0;
    for (int a = 0; a < 3; ++a) t += (size_t)face_count(g, a) * sizeof(float);
    return t;
}

size_t required_ws(const polypic_ctx *c, int64_t nf, int64_t ns) {
    int64_t n = max64(nf, ns);
    size_t a = sort_scratch_bytes(n, c->num_keys);
    size_t b = p2g_scratch_bytes(c->num_keys);
    size_t d = pcg_scratch_bytes(c->geom);
    // the G2P adjoint holds its coefficient adjoint next to the P2G scratch
    size_t e = c->cfg.coeff_format == POLYPIC_COEFF_F32
                   ? adjoint_scratch_bytes(n, c->cfg.num_modes) + b + 256
                   : 0;
    // the grid-update adjoint with the projection: three face arrays, then
    // the projection's scratch
    size_t f = d + face_bytes(c->geom) + 4 * 256;
    // the fabric forces: a slot per lattice id (at most one per solid
    // particle) and three velocity components per solid particle
    size_t fb = (size_t)ns * 16 + 1024;
    size_t m = a > b ? a : b;
    m = m > f ? m : f;
    m = m > fb ? m : fb;
    m = m > e ? m : e;
    return m + 4096;
}

polypic_status check_ws(const polypic_ctx *c, int64_t count, const void *ws, size_t ws_bytes) {
    size_t need = required_ws(c, count, 0);
    if (!ws || ((uintptr_t)ws & 255u) != 0 || ws_bytes < need) return POLYPIC_ERR_WORKSPACE;
    return POLYPIC_OK;
}

polypic_status check_positions(const polypic_particles *p) {
    if (!p || p->count < 0 || p->count >= ((int64_t)1 << 31)) return POLYPIC_ERR_INVALID_ARG;
    if (p->count > 0 && (!p->x[0] || !p->x[1] || !p->x[2])) return POLYPIC_ERR_INVALID_ARG;
    return POLYPIC_OK;
}

polypic_status check_sorted(const polypic_particles *p) {
    polypic_status s = check_positions(p);
    if (s != POLYPIC_OK) return s;
    if (!p->cell_start || (p->count > 0 && !p->perm)) return POLYPIC_ERR_INVALID_ARG;
    return POLYPIC_OK;
}

polypic_status check_coeff(const polypic_ctx *c, const polypic_particles *p) {
    if (p->count == 0) return POLYPIC_OK;
    if (!p->coeff || !p->mass) return POLYPIC_ERR_INVALID_ARG;
    // FP32 values and the 16-bit formats' code pairs are 32-bit words
    if (((uintptr_t)p->coeff & 3u) != 0) return POLYPIC_ERR_INVALID_ARG;
    if (c->cfg.coeff_format != POLYPIC_COEFF_F32 && !p->coeff_scale) return POLYPIC_ERR_INVALID_ARG;
    return POLYPIC_OK;
}

bool grid_ok(const polypic_grid *g, bool need_mass, bool need_mom, bool need_vel) {
    if (!g) return false;
    for (int a = 0; a < 3; ++a) {
        if (need_mass && !g->mass[a]) return false;
        if (need_mom && !g->mom[a]) return false;
        if (need_vel && !g->vel[a]) return false;
    }
    return true;
}

cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

polypic_status do_sort(polypic_ctx *c, polypic_particles *p, void *ws, size_t ws_bytes,
                       cudaStream_t s) {
    if (p->count > 0 && !p->key) return POLYPIC_ERR_INVALID_ARG;
    Workspace W{static_cast<char *>(ws), ws_bytes, 0};
    return from_cuda(sort_particles(c->geom, c->num_keys, p->count, p->x[0], p->x[1], p->x[2],
                                    p->key, p->perm, p->cell_start, c->d_status, W, s));
}

// Eq 12's map changes the transfer (with one mode C = 0 and M = I).
bool mapped(const polypic_ctx *c) {
    return c->cfg.map == POLYPIC_MAP_AFFINE && c->cfg.num_modes >= 4;
}

// The P2G launch arguments of phase p on context c, except the scratch (tile
// regions and live flags), which the caller supplies.
P2GArgs p2g_args(const polypic_ctx *c, const polypic_particles *p, float map_dt) {
    P2GArgs P{};
    P.affine = mapped(c);
    P.map_dt = map_dt;
    P.g = c->geom;
    P.count = p->count;
    P.x = p->x[0];
    P.y = p->x[1];
    P.z = p->x[2];
    P.mass = p->mass;
    P.mass_abs = p->mass_abs;
    P.coeff = p->coeff;
    P.scale = p->coeff_scale;
    P.perm = p->perm;
    P.cell_start = p->cell_start;
    P.status = c->d_status;
    P.nblocks = (uint32_t)(c->num_keys / 32);
    for (int l = 0; l < 7; ++l) P.dxpow[l] = (float)std::pow(c->cfg.dx, (double)l);
    // FP32 coefficients are physical: the stencil's degree-1 and -2 factors carry dx, dx^2
    const bool phys = c->cfg.coeff_format == POLYPIC_COEFF_F32;
    P.s1 = phys ? P.dxpow[1] : 1.0f;
    P.s2 = phys ? P.dxpow[2] : 1.0f;
    return P;
}

polypic_status do_p2g(polypic_ctx *c, const polypic_particles *p, polypic_grid *g, void *ws,
                      size_t ws_bytes, cudaStream_t s, const polypic_update_params *fused = nullptr,
                      float map_dt = 0.0f) {
    P2GArgs P = p2g_args(c, p, map_dt);
    Workspace W{static_cast<char *>(ws), ws_bytes, 0};
    P.scratch = W.take<float>((size_t)(c->num_keys / 256) * kTileFloats);
    P.tile_live = W.take<uint8_t>((size_t)(c->num_keys / 256));
    if (W.overflow) return POLYPIC_ERR_WORKSPACE;
    return from_cuda(p2g(P, g->mass, g->mom, fused ? g->vel : nullptr, fused ? fused->dt : 0.0f,
                         fused ? fused->gravity : nullptr, c->cfg.num_modes, c->cfg.coeff_format,
                         s));
}

polypic_status do_g2p(polypic_ctx *c, const polypic_grid *g, const polypic_particles *in,
                      polypic_particles *out, float dt, cudaStream_t s) {
    G2PArgs A{};
    A.g = c->geom;
    A.count = in->count;
    A.dt = dt;
    for (int a = 0; a < 3; ++a) A.vel[a] = g->vel[a];
    A.x = in->x[0];
    A.y = in->x[1];
    A.z = in->x[2];
    A.mass = in->mass;
    A.mass_abs = in->mass_abs;
    A.perm = in->perm;
    A.cell_start = in->cell_start;
    A.ox = out->x[0];
    A.oy = out->x[1];
    A.oz = out->x[2];
    A.omass = out->mass;
    A.omass_abs = in->mass_abs ? out->mass_abs : nullptr;
    A.ocoeff = out->coeff;
    A.oscale = out->coeff_scale;
    A.status = c->d_status;
    for (int l = 0; l < 7; ++l) A.inv_dxpow[l] = (float)std::pow(c->cfg.dx, -(double)l);
    A.grad_w = c->cfg.apic_variant == POLYPIC_APIC_GRAD_W;
    int64_t tiles = c->num_keys / 256;
    return from_cuda(g2p(A, tiles, c->cfg.num_modes, c->cfg.coeff_format, s));
}

polypic_status check_g2p_out(const polypic_ctx *c, const polypic_particles *in,
                             const polypic_particles *out) {
    if (!out || out->count != in->count) return POLYPIC_ERR_INVALID_ARG;
    if (in->count == 0) return POLYPIC_OK;
    if (!out->x[0] || !out->x[1] || !out->x[2] || !out->mass || !out->coeff)
        return POLYPIC_ERR_INVALID_ARG;
    if (((uintptr_t)out->coeff & 3u) != 0) return POLYPIC_ERR_INVALID_ARG;
    if (c->cfg.coeff_format != POLYPIC_COEFF_F32 && !out->coeff_scale) return POLYPIC_ERR_INVALID_ARG;
    if (in->mass_abs && !out->mass_abs) return POLYPIC_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            if (out->x[a] == in->x[b]) return POLYPIC_ERR_INVALID_ARG;
    if (out->mass == in->mass || out->coeff == in->coeff) return POLYPIC_ERR_INVALID_ARG;
    return POLYPIC_OK;
}

polypic_status check_params(const polypic_update_params *u) {
    if (!u || !std::isfinite(u->dt) || !std::isfinite(u->gravity[0]) ||
        !std::isfinite(u->gravity[1]) || !std::isfinite(u->gravity[2]) ||
        !std::isfinite(u->drag_k) || u->drag_k < 0.0f)
        return POLYPIC_ERR_INVALID_ARG;
    if (u->project) {
        if (!(u->rho > 0.0f) || u->pcg_maxiter <= 0 || !(u->pcg_rtol > 0.0))
            return POLYPIC_ERR_INVALID_ARG;
    }
    return POLYPIC_OK;
}

polypic_status do_grid_update(polypic_ctx *c, polypic_grid *fluid, polypic_grid *solid,
                              const polypic_particles *fp, const polypic_update_params *u,
                              void *ws, size_t ws_bytes, cudaStream_t s) {
    GridUpdateArgs U{};
    U.g = c->geom;
    U.dt = u->dt;
    for (int a = 0; a < 3; ++a) {
        U.gravity[a] = u->gravity[a];
        U.fm[a] = fluid->mass[a];
        U.fp[a] = fluid->mom[a];
        U.fv[a] = fluid->vel[a];
        U.sm[a] = solid ? solid->mass[a] : nullptr;
        U.sp[a] = solid ? solid->mom[a] : nullptr;
        U.sv[a] = solid ? solid->vel[a] : nullptr;
    }
    U.drag_k = u->drag_k;
    polypic_status st = from_cuda(grid_update(U, s));
    if (st != POLYPIC_OK || !u->project) return st;
    Workspace W{static_cast<char *>(ws), ws_bytes, 0};
    return pcg_project(c->geom, c->num_keys, fp->cell_start, fluid->vel, u->dt, u->rho,
                       u->pcg_maxiter, u->pcg_rtol, c->d_status, W, s, &c->pcg_graphs);
}

}  // namespace

extern "C" {

polypic_status polypic_create(const polypic_config *cfg, polypic_ctx **out) {
    if (!out) return POLYPIC_ERR_INVALID_ARG;
    *out = nullptr;
    if (!cfg) return POLYPIC_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a)
        if (cfg->n[a] < 4 || cfg->n[a] > 2048) return POLYPIC_ERR_INVALID_ARG;
    if (!(cfg->dx > 0.0) || !std::isfinite(cfg->dx)) return POLYPIC_ERR_INVALID_ARG;
    if (!valid_modes(cfg->num_modes)) return POLYPIC_ERR_INVALID_ARG;
    if (cfg->coeff_format < POLYPIC_COEFF_F32 || cfg->coeff_format > POLYPIC_COEFF_F16)
        return POLYPIC_ERR_INVALID_ARG;
    if (cfg->map != POLYPIC_MAP_CONSTANT && cfg->map != POLYPIC_MAP_AFFINE)
        return POLYPIC_ERR_INVALID_ARG;
    // Eq 12's map is built for FP32 coefficients (a transform of the linear
    // coefficients for 4 modes, per-node evaluation for 8 and 27)
    if (cfg->map == POLYPIC_MAP_AFFINE && cfg->coeff_format != POLYPIC_COEFF_F32)
        return POLYPIC_ERR_UNSUPPORTED;
    if (cfg->apic_variant != POLYPIC_APIC_TRUNCATION && cfg->apic_variant != POLYPIC_APIC_GRAD_W)
        return POLYPIC_ERR_INVALID_ARG;
    // Eq 10's gradient form replaces the linear modes of the 4-mode set
    if (cfg->apic_variant == POLYPIC_APIC_GRAD_W && cfg->num_modes != 4)
        return POLYPIC_ERR_INVALID_ARG;

    GridGeom g{};
    for (int a = 0; a < 3; ++a) g.n[a] = cfg->n[a];
    g.tiles[0] = (cfg->n[0] + 7) / 8;
    g.tiles[1] = (cfg->n[1] + 7) / 8;
    g.tiles[2] = (cfg->n[2] + 3) / 4;
    int64_t K = (int64_t)g.tiles[0] * g.tiles[1] * g.tiles[2] * 256;
    // scans handle up to 256 * 256 chunks of 4096 keys
    if (K + 1 > (int64_t)kScanThreads * 256 * kScanTile) return POLYPIC_ERR_UNSUPPORTED;
    g.dx = (float)cfg->dx;
    g.inv_dx = (float)(1.0 / cfg->dx);
    for (int a = 0; a < 3; ++a) {
        g.lo[a] = (float)(1.5 * cfg->dx);
        g.hi[a] = (float)(((double)cfg->n[a] - 1.5) * cfg->dx);
    }

    polypic_ctx *c = new (std::nothrow) polypic_ctx;
    if (!c) return POLYPIC_ERR_CUDA;
    c->cfg = *cfg;
    c->geom = g;
    c->num_keys = K;
    c->d_status = nullptr;
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaMalloc(&c->d_status, 4 * sizeof(uint32_t)) != cudaSuccess ||
        cudaMemset(c->d_status, 0, 4 * sizeof(uint32_t)) != cudaSuccess) {
        if (c->d_status) cudaFree(c->d_status);
        delete c;
        return POLYPIC_ERR_CUDA;
    }
    *out = c;
    return POLYPIC_OK;
}

void polypic_destroy(polypic_ctx *ctx) {
    if (!ctx) return;
    if (ctx->d_status) cudaFree(ctx->d_status);
    pcg_graphs_free(ctx->pcg_graphs);
    delete ctx;
}

int64_t polypic_num_keys(const polypic_ctx *ctx) { return ctx ? ctx->num_keys : -1; }

uint32_t polypic_cell_key(const polypic_ctx *ctx, int32_t i, int32_t j, int32_t k) {
    if (!ctx) return 0xffffffffu;
    return cell_key(ctx->geom, i, j, k);
}

polypic_status polypic_grid_dims(const polypic_ctx *ctx, int32_t axis, int32_t dims[3]) {
    if (!ctx || !dims || axis < 0 || axis > 2) return POLYPIC_ERR_INVALID_ARG;
    for (int b = 0; b < 3; ++b) dims[b] = ctx->cfg.n[b] + (b == axis ? 1 : 0);
    return POLYPIC_OK;
}

size_t polypic_workspace_bytes(const polypic_ctx *ctx, int64_t n_fluid, int64_t n_solid) {
    if (!ctx || n_fluid < 0 || n_solid < 0) return 0;
    return required_ws(ctx, n_fluid, n_solid);
}

polypic_status polypic_sort(polypic_ctx *ctx, polypic_particles *p, void *ws, size_t ws_bytes,
                            void *stream) {
    if (!ctx) return POLYPIC_ERR_INVALID_ARG;
    polypic_status s = check_sorted(p);
    if (s != POLYPIC_OK) return s;
    if ((s = check_ws(ctx, p->count, ws, ws_bytes)) != POLYPIC_OK) return s;
    return do_sort(ctx, p, ws, ws_bytes, as_stream(stream));
}

polypic_status polypic_p2g(polypic_ctx *ctx, const polypic_particles *p, polypic_grid *g,
                           void *ws, size_t ws_bytes, void *stream) {
    if (!ctx || mapped(ctx)) return POLYPIC_ERR_INVALID_ARG;  // the map needs dt
    polypic_status s = check_sorted(p);
    if (s != POLYPIC_OK) return s;
    if ((s = check_coeff(ctx, p)) != POLYPIC_OK) return s;
    if (!grid_ok(g, true, true, false)) return POLYPIC_ERR_INVALID_ARG;
    if ((s = check_ws(ctx, p->count, ws, ws_bytes)) != POLYPIC_OK) return s;
    return do_p2g(ctx, p, g, ws, ws_bytes, as_stream(stream));
}

polypic_status polypic_p2g_mapped(polypic_ctx *ctx, const polypic_particles *p, polypic_grid *g,
                                  float dt, void *ws, size_t ws_bytes, void *stream) {
    if (!ctx || !std::isfinite(dt)) return POLYPIC_ERR_INVALID_ARG;
    polypic_status s = check_sorted(p);
    if (s != POLYPIC_OK) return s;
    if ((s = check_coeff(ctx, p)) != POLYPIC_OK) return s;
    if (!grid_ok(g, true, true, false)) return POLYPIC_ERR_INVALID_ARG;
    if ((s = check_ws(ctx, p->count, ws, ws_bytes)) != POLYPIC_OK) return s;
    return do_p2g(ctx, p, g, ws, ws_bytes, as_stream(stream), nullptr, dt);
}

polypic_status polypic_p2g_noalloc(polypic_ctx *ctx, const polypic_particles *p, polypic_grid *g,
                                   void *stream) {
    if (!ctx || mapped(ctx)) return POLYPIC_ERR_INVALID_ARG;  // the map needs dt
    polypic_status s = check_sorted(p);
    if (s != POLYPIC_OK) return s;
    if ((s = check_coeff(ctx, p)) != POLYPIC_OK) return s;
    if (!grid_ok(g, true, true, false)) return POLYPIC_ERR_INVALID_ARG;
    if (ctx->num_keys / 256 > (int64_t)p2g_builtin_max_tiles()) return POLYPIC_ERR_WORKSPACE;
    P2GArgs P = p2g_args(ctx, p, 0.0f);
    if (p2g_builtin_scratch(as_stream(stream), &P.scratch, &P.tile_live) != cudaSuccess)
        return POLYPIC_ERR_CUDA;
    return from_cuda(p2g(P, g->mass, g->mom, nullptr, 0.0f, nullptr, ctx->cfg.num_modes,
                         ctx->cfg.coeff_format, as_stream(stream)));
}

polypic_status polypic_grid_update(polypic_ctx *ctx, polypic_grid *fluid, polypic_grid *solid,
                                   const polypic_particles *fluid_particles,
                                   const polypic_update_params *params, void *ws,
                                   size_t ws_bytes, void *stream) {
    if (!ctx) return POLYPIC_ERR_INVALID_ARG;
    if (!grid_ok(fluid, true, true, true)) return POLYPIC_ERR_INVALID_ARG;
    if (solid && !grid_ok(solid, true, true, true)) return POLYPIC_ERR_INVALID_ARG;
    polypic_status s = check_params(params);
    if (s != POLYPIC_OK) return s;
    if (params->project) {
        if (!fluid_particles || !fluid_particles->cell_start) return POLYPIC_ERR_INVALID_ARG;
        if ((s = check_ws(ctx, 0, ws, ws_bytes)) != POLYPIC_OK) return s;
    }
    return do_grid_update(ctx, fluid, solid, fluid_particles, params, ws, ws_bytes,
                          as_stream(stream));
}

polypic_status polypic_g2p(polypic_ctx *ctx, const polypic_grid *g, const polypic_particles *in,
                           polypic_particles *out, float dt, void *ws, size_t ws_bytes,
                           void *stream) {
    (void)ws;
    (void)ws_bytes;
    if (!ctx || !std::isfinite(dt)) return POLYPIC_ERR_INVALID_ARG;
    polypic_status s = check_sorted(in);
    if (s != POLYPIC_OK) return s;
    if (in->count > 0 && !in->mass) return POLYPIC_ERR_INVALID_ARG;
    if (!grid_ok(g, false, false, true)) return POLYPIC_ERR_INVALID_ARG;
    if ((s = check_g2p_out(ctx, in, out)) != POLYPIC_OK) return s;
    return do_g2p(ctx, g, in, out, dt, as_stream(stream));
}

polypic_status polypic_step(polypic_ctx *ctx, polypic_particles *fluid_in,
                            polypic_particles *fluid_out, polypic_particles *solid_in,
                            polypic_particles *solid_out, polypic_grid *gf, polypic_grid *gs,
                            const polypic_update_params *params, void *ws, size_t ws_bytes,
                            void *stream) {
    if (!ctx) return POLYPIC_ERR_INVALID_ARG;
    const bool solid = solid_in != nullptr;
    if (solid && (!solid_out || !gs)) return POLYPIC_ERR_INVALID_ARG;
    polypic_status s;
    if ((s = check_sorted(fluid_in)) != POLYPIC_OK) return s;
    if (fluid_in->count > 0 && !fluid_in->key) return POLYPIC_ERR_INVALID_ARG;
    if ((s = check_coeff(ctx, fluid_in)) != POLYPIC_OK) return s;
    if ((s = check_g2p_out(ctx, fluid_in, fluid_out)) != POLYPIC_OK) return s;
    if (solid) {
        if ((s = check_sorted(solid_in)) != POLYPIC_OK) return s;
        if (solid_in->count > 0 && !solid_in->key) return POLYPIC_ERR_INVALID_ARG;
        if ((s = check_coeff(ctx, solid_in)) != POLYPIC_OK) return s;
        if ((s = check_g2p_out(ctx, solid_in, solid_out)) != POLYPIC_OK) return s;
        if (!grid_ok(gs, true, true, true)) return POLYPIC_ERR_INVALID_ARG;
    }
    if (!grid_ok(gf, true, true, true)) return POLYPIC_ERR_INVALID_ARG;
    if ((s = check_params(params)) != POLYPIC_OK) return s;
    const int64_t nmax = max64(fluid_in->count, solid ? solid_in->count : 0);
    if ((s = check_ws(ctx, nmax, ws, ws_bytes)) != POLYPIC_OK) return s;
    cudaStream_t st = as_stream(stream);
    // a single phase without projection gets the grid update fused into P2G's reduce
    const bool fuse = !solid && !params->project;
    if ((s = do_sort(ctx, fluid_in, ws, ws_bytes, st)) != POLYPIC_OK) return s;
    if ((s = do_p2g(ctx, fluid_in, gf, ws, ws_bytes, st, fuse ? params : nullptr, params->dt)) !=
        POLYPIC_OK)
        return s;
    if (solid) {
        if ((s = do_sort(ctx, solid_in, ws, ws_bytes, st)) != POLYPIC_OK) return s;
        if ((s = do_p2g(ctx, solid_in, gs, ws, ws_bytes, st, nullptr, params->dt)) !=
            POLYPIC_OK)
            return s;
    }
    if (!fuse && (s = do_grid_update(ctx, gf, solid ? gs : nullptr, fluid_in, params, ws, ws_bytes,
                                     st)) != POLYPIC_OK)
        return s;
    if ((s = do_g2p(ctx, gf, fluid_in, fluid_out, params->dt, st)) != POLYPIC_OK) return s;
    if (solid && (s = do_g2p(ctx, gs, solid_in, solid_out, params->dt, st)) != POLYPIC_OK) return s;
    return POLYPIC_OK;
}

polypic_status polypic_g2p2g(polypic_ctx *ctx, const polypic_grid *g,
                             const polypic_particles *in, polypic_particles *out,
                             polypic_particles *spill, polypic_grid *g_next, float dt, void *ws,
                             size_t ws_bytes, void *stream) {
    if (!ctx) return POLYPIC_ERR_INVALID_ARG;
    if (ctx->cfg.coeff_format != POLYPIC_COEFF_F32 || mapped(ctx) ||
        ctx->cfg.apic_variant == POLYPIC_APIC_GRAD_W)
        return POLYPIC_ERR_UNSUPPORTED;
    polypic_status s;
    if ((s = check_sorted(in)) != POLYPIC_OK) return s;
    if ((s = check_g2p_out(ctx, in, out)) != POLYPIC_OK) return s;
    if (!std::isfinite(dt)) return POLYPIC_ERR_INVALID_ARG;
    if (!grid_ok(g, false, false, true) || !grid_ok(g_next, true, true, false))
        return POLYPIC_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            if (g_next->mass[a] == g->vel[b] || g_next->mom[a] == g->vel[b])
                return POLYPIC_ERR_INVALID_ARG;
    if (!spill || spill->count < 0 || spill->count >= ((int64_t)1 << 31))
        return POLYPIC_ERR_INVALID_ARG;
    if (spill->count > 0 && (!spill->x[0] || !spill->x[1] || !spill->x[2] || !spill->mass ||
                             !spill->coeff || !spill->key || !spill->perm))
        return POLYPIC_ERR_INVALID_ARG;
    if (!spill->cell_start || (in->mass_abs && spill->count > 0 && !spill->mass_abs))
        return POLYPIC_ERR_INVALID_ARG;
    if (((uintptr_t)spill->coeff & 3u) != 0) return POLYPIC_ERR_INVALID_ARG;
    if ((s = check_ws(ctx, in->count, ws, ws_bytes)) != POLYPIC_OK) return s;
    cudaStream_t st = as_stream(stream);
    const int64_t tiles = ctx->num_keys / 256;
    const int R = ctx->cfg.num_modes;
    Workspace W{static_cast<char *>(ws), ws_bytes, 0};
    P2GArgs P = p2g_args(ctx, in, 0.0f);
    P.scratch = W.take<float>((size_t)tiles * kTileFloats);
    P.tile_live = W.take<uint8_t>((size_t)tiles);
    uint8_t *moved = W.take<uint8_t>((size_t)in->count + 1);
    uint32_t *counts = W.take<uint32_t>((size_t)tiles);
    uint32_t *offsets = W.take<uint32_t>((size_t)tiles + 1);
    if (W.overflow) return POLYPIC_ERR_WORKSPACE;
    G2P2GArgs Q{};
    Q.p2g = P;
    Q.x = in->x[0];
    Q.y = in->x[1];
    Q.z = in->x[2];
    for (int a = 0; a < 3; ++a) Q.vel[a] = g->vel[a];
    Q.dt = dt;
    Q.inv1 = (float)(1.0 / ctx->cfg.dx);
    Q.inv2 = (float)(1.0 / (ctx->cfg.dx * ctx->cfg.dx));
    Q.ox = out->x[0];
    Q.oy = out->x[1];
    Q.oz = out->x[2];
    Q.omass = out->mass;
    Q.omass_abs = in->mass_abs ? out->mass_abs : nullptr;
    Q.ocoeff = static_cast<float *>(out->coeff);
    Q.moved = moved;
    if (g2p2g_tiles(Q, R, st) != cudaSuccess) return POLYPIC_ERR_CUDA;
    float *gm[3] = {g_next->mass[0], g_next->mass[1], g_next->mass[2]};
    float *gp[3] = {g_next->mom[0], g_next->mom[1], g_next->mom[2]};
    if (p2g_reduce(P, gm, gp, false, st) != cudaSuccess) return POLYPIC_ERR_CUDA;
    if (in->count == 0) return POLYPIC_OK;
    // the movers: a compact spill phase in slot order, sorted and added on
    if (count_and_scan_movers(in->cell_start, moved, tiles, counts, offsets, st) != cudaSuccess)
        return POLYPIC_ERR_CUDA;
    SpillArgs S{};
    S.count = in->count;
    S.ntiles = tiles;
    S.R = R;
    S.capacity = (uint32_t)spill->count;
    S.cell_start = in->cell_start;
    S.offsets = offsets;
    S.moved = moved;
    S.ox = out->x[0];
    S.oy = out->x[1];
    S.oz = out->x[2];
    S.omass = out->mass;
    S.omass_abs = Q.omass_abs;
    S.ocoeff = Q.ocoeff;
    S.x = spill->x[0];
    S.y = spill->x[1];
    S.z = spill->x[2];
    S.mass = spill->mass;
    S.mass_abs = in->mass_abs ? spill->mass_abs : nullptr;
    S.coeff = static_cast<float *>(spill->coeff);
    if (compact_movers(S, st) != cudaSuccess) return POLYPIC_ERR_CUDA;
    uint32_t total = 0;
    if (cudaMemcpyAsync(&total, offsets + tiles, sizeof(uint32_t), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return POLYPIC_ERR_CUDA;
    if ((int64_t)total > spill->count) return POLYPIC_ERR_WORKSPACE;
    if (total == 0) return POLYPIC_OK;
    polypic_particles sp = *spill;
    sp.count = total;
    sp.mass_abs = S.mass_abs;
    sp.coeff_scale = nullptr;
    if ((s = do_sort(ctx, &sp, ws, ws_bytes, st)) != POLYPIC_OK) return s;
    P2GArgs P2 = p2g_args(ctx, &sp, 0.0f);
    Workspace W2{static_cast<char *>(ws), ws_bytes, 0};
    P2.scratch = W2.take<float>((size_t)tiles * kTileFloats);
    P2.tile_live = W2.take<uint8_t>((size_t)tiles);
    if (W2.overflow) return POLYPIC_ERR_WORKSPACE;
    return from_cuda(p2g_accumulate(P2, gm, gp, R, st));
}

namespace {

bool fabric_ok(const polypic_fabric_params *f) {
    return f && f->verts_per_side >= 0 && f->verts_per_side <= 65535 &&
           std::isfinite(f->rest_length) && f->rest_length >= 0.0f &&
           std::isfinite(f->k_stretch) && std::isfinite(f->k_shear) && std::isfinite(f->k_bend) &&
           std::isfinite(f->damping) && std::isfinite(f->absorb_rate) &&
           f->absorb_rate >= 0.0f && std::isfinite(f->absorb_capacity) &&
           std::isfinite(f->absorb_max_fraction) && f->absorb_max_fraction >= 0.0f &&
           f->absorb_max_fraction <= 1.0f;
}

bool forces_on(const polypic_fabric_params *f) {
    return f->verts_per_side > 0 && (f->k_stretch != 0.0f || f->k_shear != 0.0f ||
                                     f->k_bend != 0.0f || f->damping != 0.0f);
}

polypic_status do_fabric_forces(polypic_ctx *c, polypic_particles *p,
                                const polypic_fabric_params *f, float dt, void *ws,
                                size_t ws_bytes, cudaStream_t s) {
    if (p->count == 0) return POLYPIC_OK;
    FabricForceArgs A{};
    A.count = p->count;
    const int R = c->cfg.num_modes;
    float *coeff = static_cast<float *>(p->coeff);
    for (int a = 0; a < 3; ++a) {
        A.x[a] = p->x[a];
        A.vel[a] = coeff + (size_t)a * R * (size_t)p->count;
    }
    A.mass = p->mass;
    A.mass_abs = p->mass_abs;
    A.id = p->id;
    A.m = f->verts_per_side;
    A.h = f->rest_length;
    A.k_stretch = f->k_stretch;
    A.k_shear = f->k_shear;
    A.k_bend = f->k_bend;
    A.damping = f->damping;
    A.dt = dt;
    Workspace W{static_cast<char *>(ws), ws_bytes, 0};
    if (fabric_scratch_bytes(p->count, A.m) > ws_bytes) return POLYPIC_ERR_WORKSPACE;
    return from_cuda(fabric_forces(A, W, s));
}

polypic_status do_absorb(polypic_ctx *c, polypic_particles *fl, polypic_particles *so,
                         const polypic_fabric_params *f, float dt, cudaStream_t s) {
    if (f->absorb_rate == 0.0f || fl->count == 0 || so->count == 0) return POLYPIC_OK;
    AbsorbCall A{};
    A.num_keys = c->num_keys;
    A.fluid_cell_start = fl->cell_start;
    A.fluid_perm = fl->perm;
    A.solid_cell_start = so->cell_start;
    A.solid_perm = so->perm;
    A.fluid_mass = fl->mass;
    A.solid_mass = so->mass;
    A.mass_abs = so->mass_abs;
    A.rate = f->absorb_rate;
    A.dt = dt;
    A.capacity = f->absorb_capacity;
    A.max_fraction = f->absorb_max_fraction;
    return from_cuda(absorb(A, s));
}

polypic_status check_fabric_solid(polypic_ctx *c, const polypic_particles *p, bool need_id) {
    if (!p || !p->mass || (p->count > 0 && !p->coeff)) return POLYPIC_ERR_INVALID_ARG;
    if (((uintptr_t)p->coeff & 3u) != 0) return POLYPIC_ERR_INVALID_ARG;
    if (need_id && p->count > 0 && !p->id) return POLYPIC_ERR_INVALID_ARG;
    if (c->cfg.coeff_format != POLYPIC_COEFF_F32) return POLYPIC_ERR_UNSUPPORTED;
    return POLYPIC_OK;
}

}  // namespace

polypic_status polypic_fabric_forces(polypic_ctx *ctx, polypic_particles *solid,
                                     const polypic_fabric_params *fabric, float dt, void *ws,
                                     size_t ws_bytes, void *stream) {
    if (!ctx || !fabric_ok(fabric) || !std::isfinite(dt)) return POLYPIC_ERR_INVALID_ARG;
    polypic_status s;
    if ((s = check_positions(solid)) != POLYPIC_OK) return s;
    if ((s = check_fabric_solid(ctx, solid, true)) != POLYPIC_OK) return s;
    if (!forces_on(fabric)) return POLYPIC_OK;
    if (!ws || ((uintptr_t)ws & 255u) != 0) return POLYPIC_ERR_WORKSPACE;
    return do_fabric_forces(ctx, solid, fabric, dt, ws, ws_bytes, as_stream(stream));
}

polypic_status polypic_absorb(polypic_ctx *ctx, polypic_particles *fluid,
                              polypic_particles *solid, const polypic_fabric_params *fabric,
                              float dt, void *stream) {
    if (!ctx || !fabric_ok(fabric) || !std::isfinite(dt)) return POLYPIC_ERR_INVALID_ARG;
    polypic_status s;
    if ((s = check_sorted(fluid)) != POLYPIC_OK) return s;
    if ((s = check_sorted(solid)) != POLYPIC_OK) return s;
    if (!fluid->mass || !solid->mass || !solid->mass_abs) return POLYPIC_ERR_INVALID_ARG;
    return do_absorb(ctx, fluid, solid, fabric, dt, as_stream(stream));
}

polypic_status polypic_step_coupled(polypic_ctx *ctx, polypic_particles *fluid_in,
                                    polypic_particles *fluid_out, polypic_particles *solid_in,
                                    polypic_particles *solid_out, polypic_grid *gf,
                                    polypic_grid *gs, const polypic_update_params *params,
                                    const polypic_fabric_params *fabric, void *ws,
                                    size_t ws_bytes, void *stream) {
    if (!ctx || !solid_in || !solid_out || !gs || !fabric_ok(fabric))
        return POLYPIC_ERR_INVALID_ARG;
    polypic_status s;
    if ((s = check_sorted(fluid_in)) != POLYPIC_OK) return s;
    if (fluid_in->count > 0 && !fluid_in->key) return POLYPIC_ERR_INVALID_ARG;
    if ((s = check_coeff(ctx, fluid_in)) != POLYPIC_OK) return s;
    if ((s = check_g2p_out(ctx, fluid_in, fluid_out)) != POLYPIC_OK) return s;
    if ((s = check_sorted(solid_in)) != POLYPIC_OK) return s;
    if (solid_in->count > 0 && !solid_in->key) return POLYPIC_ERR_INVALID_ARG;
    if ((s = check_coeff(ctx, solid_in)) != POLYPIC_OK) return s;
    if ((s = check_g2p_out(ctx, solid_in, solid_out)) != POLYPIC_OK) return s;
    if (!solid_in->mass_abs) return POLYPIC_ERR_INVALID_ARG;
    if ((s = check_fabric_solid(ctx, solid_in, true)) != POLYPIC_OK) return s;
    if (solid_in->count > 0 && (!solid_out->id || solid_out->id == solid_in->id))
        return POLYPIC_ERR_INVALID_ARG;
    if (!grid_ok(gf, true, true, true) || !grid_ok(gs, true, true, true))
        return POLYPIC_ERR_INVALID_ARG;
    if ((s = check_params(params)) != POLYPIC_OK) return s;
    const int64_t nmax = max64(fluid_in->count, solid_in->count);
    if ((s = check_ws(ctx, nmax, ws, ws_bytes)) != POLYPIC_OK) return s;
    if (ws_bytes < required_ws(ctx, fluid_in->count, solid_in->count)) return POLYPIC_ERR_WORKSPACE;
    cudaStream_t st = as_stream(stream);
    if ((s = do_sort(ctx, fluid_in, ws, ws_bytes, st)) != POLYPIC_OK) return s;
    if ((s = do_sort(ctx, solid_in, ws, ws_bytes, st)) != POLYPIC_OK) return s;
    if ((s = do_absorb(ctx, fluid_in, solid_in, fabric, params->dt, st)) != POLYPIC_OK) return s;
    if (forces_on(fabric) &&
        (s = do_fabric_forces(ctx, solid_in, fabric, params->dt, ws, ws_bytes, st)) != POLYPIC_OK)
        return s;
    if ((s = do_p2g(ctx, fluid_in, gf, ws, ws_bytes, st, nullptr, params->dt)) != POLYPIC_OK)
        return s;
    if ((s = do_p2g(ctx, solid_in, gs, ws, ws_bytes, st, nullptr, params->dt)) != POLYPIC_OK)
        return s;
    if ((s = do_grid_update(ctx, gf, gs, fluid_in, params, ws, ws_bytes, st)) != POLYPIC_OK)
        return s;
    if ((s = do_g2p(ctx, gf, fluid_in, fluid_out, params->dt, st)) != POLYPIC_OK) return s;
    if ((s = do_g2p(ctx, gs, solid_in, solid_out, params->dt, st)) != POLYPIC_OK) return s;
    return from_cuda(gather_ids(solid_in->id, solid_in->perm, solid_in->count, solid_out->id, st));
}

polypic_status polypic_g2p_adjoint(polypic_ctx *ctx, const polypic_grid *g,
                                   const polypic_particles *in, float dt,
                                   const polypic_particles *bar_out, polypic_grid *bar_grid,
                                   polypic_particles *bar_in, int32_t flags, void *ws,
                                   size_t ws_bytes, void *stream) {
    if (!ctx || !std::isfinite(dt)) return POLYPIC_ERR_INVALID_ARG;
    // the adjoints transpose the constant map and the truncation form
    if (mapped(ctx) || ctx->cfg.apic_variant != POLYPIC_APIC_TRUNCATION)
        return POLYPIC_ERR_UNSUPPORTED;
    if (ctx->cfg.coeff_format != POLYPIC_COEFF_F32) return POLYPIC_ERR_UNSUPPORTED;
    polypic_status s = check_sorted(in);
    if (s != POLYPIC_OK) return s;
    if (!grid_ok(g, false, false, true) || !grid_ok(bar_grid, false, false, true))
        return POLYPIC_ERR_INVALID_ARG;
    if (!bar_out || !bar_in || bar_out->count != in->count || bar_in->count != in->count)
        return POLYPIC_ERR_INVALID_ARG;
    if (in->count > 0 && (!bar_out->coeff || !bar_out->x[0] || !bar_out->x[1] || !bar_out->x[2] ||
                          !bar_in->x[0] || !bar_in->x[1] || !bar_in->x[2]))
        return POLYPIC_ERR_INVALID_ARG;
    if ((flags & ~POLYPIC_ADJ_ACCUMULATE) != 0) return POLYPIC_ERR_INVALID_ARG;
    if ((s = check_ws(ctx, in->count, ws, ws_bytes)) != POLYPIC_OK) return s;
    Workspace W{static_cast<char *>(ws), ws_bytes, 0};
    return from_cuda(adjoint_g2p(ctx->geom, ctx->num_keys, ctx->cfg.num_modes, (float)ctx->cfg.dx,
                                 g, in, dt, bar_out, bar_grid, bar_in,
                                 (flags & POLYPIC_ADJ_ACCUMULATE) != 0, ctx->d_status, W,
                                 as_stream(stream)));
}

polypic_status polypic_grid_update_adjoint(polypic_ctx *ctx, const polypic_grid *fluid,
                                           const polypic_grid *solid,
                                           const polypic_particles *fluid_particles,
                                           const polypic_update_params *params,
                                           const polypic_grid *bar_fluid_out,
                                           const polypic_grid *bar_solid_out,
                                           polypic_grid *bar_fluid_in, polypic_grid *bar_solid_in,
                                           void *ws, size_t ws_bytes, void *stream) {
    if (!ctx) return POLYPIC_ERR_INVALID_ARG;
    polypic_status s = check_params(params);
    if (s != POLYPIC_OK) return s;
    if (!grid_ok(fluid, true, true, false) || !grid_ok(bar_fluid_out, false, false, true) ||
        !grid_ok(bar_fluid_in, true, true, false))
        return POLYPIC_ERR_INVALID_ARG;
    const bool two = solid != nullptr;
    if (two != (bar_solid_out != nullptr) || two != (bar_solid_in != nullptr))
        return POLYPIC_ERR_INVALID_ARG;
    if (two && (!grid_ok(solid, true, true, false) || !grid_ok(bar_solid_out, false, false, true) ||
                !grid_ok(bar_solid_in, true, true, false)))
        return POLYPIC_ERR_INVALID_ARG;
    cudaStream_t st = as_stream(stream);
    GridAdjointArgs U{};
    U.g = ctx->geom;
    U.dt = params->dt;
    U.drag_k = params->drag_k;
    for (int a = 0; a < 3; ++a) {
        U.gravity[a] = params->gravity[a];
        U.fm[a] = fluid->mass[a];
        U.fp[a] = fluid->mom[a];
        U.lv[a] = bar_fluid_out->vel[a];
        U.lm[a] = bar_fluid_in->mass[a];
        U.lp[a] = bar_fluid_in->mom[a];
        U.sm[a] = two ? solid->mass[a] : nullptr;
        U.sp[a] = two ? solid->mom[a] : nullptr;
        U.lsv[a] = two ? bar_solid_out->vel[a] : nullptr;
        U.lsm[a] = two ? bar_solid_in->mass[a] : nullptr;
        U.lsp[a] = two ? bar_solid_in->mom[a] : nullptr;
    }
    if (params->project) {
        // (P W)^T = P W: the walls-then-projection map is an orthogonal
        // projector, so its transpose is the forward projection applied to
        // the wall-zeroed adjoint (same fluid cells, any dt and rho)
        if (!fluid_particles || !fluid_particles->cell_start) return POLYPIC_ERR_INVALID_ARG;
        if (!ws || ((uintptr_t)ws & 255u) != 0 || ws_bytes < required_ws(ctx, 0, 0))
            return POLYPIC_ERR_WORKSPACE;
        Workspace W{static_cast<char *>(ws), ws_bytes, 0};
        float *lam[3];
        for (int a = 0; a < 3; ++a) lam[a] = W.take<float>((size_t)face_count(ctx->geom, a));
        if (W.overflow) return POLYPIC_ERR_WORKSPACE;
        if (wall_zeroed_copy(ctx->geom, bar_fluid_out->vel, lam, st) != cudaSuccess)
            return POLYPIC_ERR_CUDA;
        s = pcg_project(ctx->geom, ctx->num_keys, fluid_particles->cell_start, lam, params->dt,
                        params->rho, params->pcg_maxiter, params->pcg_rtol, ctx->d_status, W, st,
                        &ctx->pcg_graphs);
        if (s != POLYPIC_OK) return s;
        for (int a = 0; a < 3; ++a) U.lv[a] = lam[a];
    }
    return from_cuda(grid_update_adjoint(U, st));
}

polypic_status polypic_p2g_adjoint(polypic_ctx *ctx, const polypic_particles *in,
                                   const polypic_grid *bar_grid, polypic_particles *bar_in,
                                   int32_t flags, void *ws, size_t ws_bytes, void *stream) {
    if (!ctx) return POLYPIC_ERR_INVALID_ARG;
    if (ctx->cfg.coeff_format != POLYPIC_COEFF_F32 || mapped(ctx)) return POLYPIC_ERR_UNSUPPORTED;
    polypic_status s = check_sorted(in);
    if (s != POLYPIC_OK) return s;
    if ((s = check_coeff(ctx, in)) != POLYPIC_OK) return s;
    if (!grid_ok(bar_grid, true, true, false)) return POLYPIC_ERR_INVALID_ARG;
    if (!bar_in || bar_in->count != in->count) return POLYPIC_ERR_INVALID_ARG;
    if (in->count > 0 && (!bar_in->coeff || !bar_in->x[0] || !bar_in->x[1] || !bar_in->x[2]))
        return POLYPIC_ERR_INVALID_ARG;
    if ((flags & ~POLYPIC_ADJ_ACCUMULATE) != 0) return POLYPIC_ERR_INVALID_ARG;
    if ((s = check_ws(ctx, in->count, ws, ws_bytes)) != POLYPIC_OK) return s;
    Workspace W{static_cast<char *>(ws), ws_bytes, 0};
    return from_cuda(adjoint_p2g(ctx->geom, ctx->num_keys, ctx->cfg.num_modes, (float)ctx->cfg.dx,
                                 in, bar_grid, bar_in, (flags & POLYPIC_ADJ_ACCUMULATE) != 0,
                                 ctx->d_status, W, as_stream(stream)));
}

polypic_status polypic_check_device_status(polypic_ctx *ctx, void *stream) {
    if (!ctx) return POLYPIC_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(as_stream(stream)) != cudaSuccess) return POLYPIC_ERR_CUDA;
    uint32_t h = 0;
    if (cudaMemcpy(&h, ctx->d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost) != cudaSuccess)
        return POLYPIC_ERR_CUDA;
    if (h && cudaMemset(ctx->d_status, 0, sizeof(uint32_t)) != cudaSuccess) return POLYPIC_ERR_CUDA;
    if (h & kFlagOutOfDomain) return POLYPIC_ERR_OUT_OF_DOMAIN;
    if (h & kFlagNonFinite) return POLYPIC_ERR_NONFINITE;
    if (h & kFlagNotConverged) return POLYPIC_ERR_NOT_CONVERGED;
    if (h & kFlagTimeout) return POLYPIC_ERR_TIMEOUT;
    return POLYPIC_OK;
}

const char *polypic_status_string(polypic_status s) {
    switch (s) {
        case POLYPIC_OK: return "ok";
        case POLYPIC_ERR_INVALID_ARG: return "invalid argument";
        case POLYPIC_ERR_UNSUPPORTED: return "unsupported configuration";
        case POLYPIC_ERR_OUT_OF_DOMAIN: return "particle outside the valid region";
        case POLYPIC_ERR_NONFINITE: return "non-finite velocity";
        case POLYPIC_ERR_NOT_CONVERGED: return "pressure solve did not converge";
        case POLYPIC_ERR_TIMEOUT: return "bounded device wait timed out";
        case POLYPIC_ERR_CUDA: return "CUDA runtime error";
        case POLYPIC_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    }
    return "unknown status";
}

}  // extern "C"

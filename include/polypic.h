/*
 * polypic.h -- C ABI of libpolypic, a GB300 (sm_103a) implementation of the
 * polynomial particle-in-cell (PolyPIC) particle<->grid transfers of
 * "Using The Polynomial Particle-in-Cell Method for Liquid-Fabric
 * Interaction" (arXiv 2308.01060), with the APIC transfer as its affine-mode
 * truncation.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Domain: the box [0, n_x dx] x [0, n_y dx] x [0, n_z dx] of n_x n_y n_z
 *    cells.  Staggered MAC grid (Section 3): face grid a stores velocity
 *    component a at ((i + o_x) dx, (j + o_y) dx, (k + o_z) dx) with o_b = 0
 *    for b == a and 1/2 otherwise.  Face grid a has dims
 *    (n_x + [a==0], n_y + [a==1], n_z + [a==2]) and is stored x fastest:
 *    index = (k * d_y + j) * d_x + i.
 *  - Weights: quadratic B-spline, w_ipa = N(x_p - x_ia) = prod_b N(.)
 *    (Section 3.1; quadratic per Eq 14's dx^2/4).
 *  - Modes (Section 3.3, Eq 11 with the Eq 14 substitution): per axis
 *    f_0 = 1, f_1 = z, f_2 = g(z) = z^2 - (mu3/mu2) z - mu2 with
 *    z = x_node - x_p and mu_n the B-spline-weighted moments of the particle's
 *    three stencil nodes; s_r = f_a(z_x) f_b(z_y) f_c(z_z).  Canonical order
 *    r <-> (a,b,c): r = 0 (000); 1..3 (100)(010)(001); 4..7 (110)(101)(011)
 *    (111); 8..26 the triples containing a 2 in lexicographic order of
 *    (c, b, a).  num_modes = 1 (PIC), 4 (APIC), 8 (the paper's setting),
 *    27 (full PolyPIC) take prefixes of this order.
 *  - Particle arrays are structure-of-arrays in device memory owned by the
 *    caller.  FP32 coefficients are laid out [3][num_modes][count]: element
 *    (a, r, p) at (a * num_modes + r) * count + p.  The 16-bit formats pack
 *    two modes per 32-bit word: [3][H][count] words, H = (num_modes + 1) / 2,
 *    word (a, k, p) at (a * H + k) * count + p holding the code of mode 2k in
 *    its low 16 bits and of mode 2k + 1 in its high 16 bits (0 when
 *    2k + 1 = num_modes), so that one 4-byte load serves two modes of a
 *    particle.  Coefficient arrays must be 4-byte aligned.
 *  - Every call is asynchronous on `stream` (a cudaStream_t, NULL = legacy
 *    default stream).  Arguments are validated on the host before anything
 *    is launched; a bad argument returns an error and launches nothing.  No
 *    C++ exception crosses this interface.
 *  - Conditions found on the device (a particle outside the valid region, a
 *    non-finite velocity) latch bits of a device status word in the context;
 *    polypic_check_device_status() synchronises the stream, returns the first
 *    latched condition and clears it.  Kernels never trap.
 *  - Scratch memory is the caller's `ws` buffer (device memory of at least
 *    polypic_workspace_bytes() bytes, 256-byte aligned).  The library itself
 *    owns only the context (a few bytes of device memory for the status
 *    word).  Calls that share a workspace must not overlap on the GPU.
 *  - Decisions that pick an integer (a particle's cell, the lowest stencil
 *    node, the quadratic-mode guard) are taken in FP32 with every operation
 *    rounded separately (no fused multiply-add) from the FP32 position, so
 *    that any reimplementation following this text takes the same decision:
 *       v = fl(x * inv_dx), inv_dx = (float)(1.0 / dx)
 *       cell = clamp(floor(v), 0, n - 1)
 *       X = v (face axis, o = 0) or fl(v - 0.5) (other axes, o = 1/2)
 *       base = floor(fl(X - 0.5)), t = fl(X - (base + 1)) in [-1/2, 1/2)
 *       guard = fl(fl(1 - 2t) * fl(1 + 2t)) < 2^-10.
 *  - Valid particles satisfy 1 <= v < n - 1 on every axis; the transfers
 *    skip any other particle and latch POLYPIC_ERR_OUT_OF_DOMAIN.
 */
#ifndef POLYPIC_H
#define POLYPIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum polypic_status {
    POLYPIC_OK = 0,
    POLYPIC_ERR_INVALID_ARG = 1,   /* bad pointer, size, or enum value */
    POLYPIC_ERR_UNSUPPORTED = 2,   /* valid but not implemented combination */
    POLYPIC_ERR_OUT_OF_DOMAIN = 3, /* a particle outside 1 <= x/dx < n-1 */
    POLYPIC_ERR_NONFINITE = 4,     /* a NaN or Inf reached a velocity */
    POLYPIC_ERR_NOT_CONVERGED = 5, /* PCG hit its iteration cap */
    POLYPIC_ERR_TIMEOUT = 6,       /* a bounded device wait gave up */
    POLYPIC_ERR_CUDA = 7,          /* a CUDA runtime call failed */
    POLYPIC_ERR_WORKSPACE = 8      /* ws NULL, misaligned, or too small */
} polypic_status;

enum {
    POLYPIC_COEFF_F32 = 0,   /* float c_pra, physical units */
    POLYPIC_COEFF_BF16 = 1,  /* bfloat16 codes with a per-particle FP32 scale */
    POLYPIC_COEFF_F16 = 2    /* IEEE half codes with a per-particle FP32 scale */
};

enum { POLYPIC_MAP_CONSTANT = 0, POLYPIC_MAP_AFFINE = 1 };
enum { POLYPIC_APIC_TRUNCATION = 0, POLYPIC_APIC_GRAD_W = 1 };

/* Adjoint flags. */
enum { POLYPIC_ADJ_ACCUMULATE = 1 };   /* add into the outputs instead of overwriting */

typedef struct polypic_ctx polypic_ctx;

/* Problem definition.  Fixed for the life of a context. */
typedef struct polypic_config {
    int32_t n[3];          /* cells per axis, each >= 4 */
    double dx;             /* cell width (> 0) */
    int32_t num_modes;     /* N_r: 1, 4, 8 or 27 */
    int32_t coeff_format;  /* POLYPIC_COEFF_* */
    int32_t map;           /* POLYPIC_MAP_CONSTANT, or POLYPIC_MAP_AFFINE (Eq 12):
                              P2G evaluates the modes at xi = (I + dt C_p)^-1 (x_ia - x_p),
                              C_p the linear-mode coefficients (C_ab = c_{a,1+b}); the
                              identity when |det(I + dt C_p)| < 1e-6.  FP32
                              coefficients only (16-bit: UNSUPPORTED); 8 and 27 modes
                              evaluate the mapped modes per stencil node, ~3.5x the
                              arithmetic of the constant map */
    int32_t apic_variant;  /* POLYPIC_APIC_TRUNCATION, or POLYPIC_APIC_GRAD_W (Eq 10,
                              num_modes 4 only, else INVALID_ARG): G2P sets the linear
                              modes to sum_i (dw_ipa/dx_pb) v~_ia instead of the fit */
} polypic_config;

/* One phase of particles (Section 3.4: fluid, or solid with absorbed mass).
 * All pointers are device memory owned by the caller.
 *   x[3]        [count] float positions (in)
 *   mass        [count] float particle mass m_p (in)
 *   mass_abs    [count] float absorbed fluid mass, or NULL for fluid (Eq 18)
 *   coeff       [3][num_modes][count] float for POLYPIC_COEFF_F32; for the
 *               16-bit formats [3][(num_modes + 1) / 2][count] words of two
 *               codes (see above), the codes of c_pra dx^L_r / s_p, where L_r
 *               is the total degree of mode r and s_p = max |c_pra dx^L_r|
 *   coeff_scale [count] float s_p (16-bit formats only, else NULL)
 *   key, perm   [count] uint32, written by polypic_sort (perm: slot order)
 *   cell_start  [polypic_num_keys() + 1] uint32, written by polypic_sort
 *   id          [count] uint32 or NULL: a label carried with each particle by
 *               polypic_step_coupled (the sheet's lattice ids)              */
typedef struct polypic_particles {
    int64_t count;
    float *x[3];
    float *mass;
    float *mass_abs;
    void *coeff;
    float *coeff_scale;
    uint32_t *key;
    uint32_t *perm;
    uint32_t *cell_start;
    uint32_t *id;
} polypic_particles;

/* The three face grids of one phase (device memory, caller-owned). */
typedef struct polypic_grid {
    float *mass[3];   /* m_ia   (Eqs 1, 4) */
    float *mom[3];    /* (mv)_ia (Eqs 3, 13) */
    float *vel[3];    /* v~_ia after the grid update */
} polypic_grid;

typedef struct polypic_update_params {
    float dt;
    float gravity[3];
    float drag_k;        /* two-phase drag coefficient K (kg/s per face), 0 = none */
    float rho;           /* fluid density for the projection */
    int32_t project;     /* 1: pressure projection on fluid cells */
    int32_t pcg_maxiter;
    double pcg_rtol;
} polypic_update_params;

/* Stand-ins for the fabric mechanics and the absorption, which the paper
 * takes from Fei et al. (Sections 3.4 and 4; Eqs 18-20 take m_abs as given).
 *   verts_per_side  m <= 65535: the sheet's vertex particles carry lattice
 *                   ids k m + i (ids >= m^2: element particles, no springs)
 *   rest_length     h, the lattice spacing at rest
 *   k_stretch, k_shear, k_bend  spring constants (N/m) of the springs to the
 *                   neighbours at (+-1, 0), (0, +-1); (+-1, +-1); (+-2, 0),
 *                   (0, +-2), rest lengths h, h sqrt 2, 2h
 *   damping         c (kg/s) of the dampers along the same springs
 *   absorb_rate     rate (1/s) at which a solid particle takes fluid mass,
 *                   relative to its own mass m_s; 0 disables absorption
 *   absorb_capacity the most m_abs a solid particle holds, relative to m_s
 *   absorb_max_fraction  the most of a cell's fluid mass taken in one step */
typedef struct polypic_fabric_params {
    int32_t verts_per_side;
    float rest_length;
    float k_stretch, k_shear, k_bend;
    float damping;
    float absorb_rate, absorb_capacity, absorb_max_fraction;
} polypic_fabric_params;

/* ---- context ------------------------------------------------------------ */

/* Validates *cfg and allocates the context (and its device status word) on
 * the current device.  Returns INVALID_ARG / UNSUPPORTED / CUDA on failure,
 * leaving *out NULL. */
polypic_status polypic_create(const polypic_config *cfg, polypic_ctx **out);
void polypic_destroy(polypic_ctx *ctx);

/* Number of sort keys K (cell_start has K + 1 entries).  Keys order cells in
 * tiles of 8x8x4 cells (row-major tile order); a tile is 2x2x2 blocks of
 * 4x4x2 cells (x fastest); cells in a block are x fastest:
 *   key = tile * 256 + block_in_tile * 32 + cell_in_block.  Returns -1 for a
 * NULL context. */
int64_t polypic_num_keys(const polypic_ctx *ctx);

/* Key of cell (i, j, k) under the layout above (host helper). */
uint32_t polypic_cell_key(const polypic_ctx *ctx, int32_t i, int32_t j, int32_t k);

/* dims[0..2] of face grid `axis` (0, 1, 2). */
polypic_status polypic_grid_dims(const polypic_ctx *ctx, int32_t axis, int32_t dims[3]);

/* Bytes of scratch needed by any call on phases of up to n_fluid and n_solid
 * particles (0 on a NULL context). */
size_t polypic_workspace_bytes(const polypic_ctx *ctx, int64_t n_fluid, int64_t n_solid);

/* ---- forward transfers --------------------------------------------------- */

/* Bit-exact sort of the particles by cell key (an implementation device; the
 * paper has none).  Writes p->key (key of each particle), p->cell_start
 * (cell_start[k] = number of particles with key < k; entry K = count) and
 * p->perm, the slot order used by the transfers: take the stable (key,
 * index) order; every block of 32 consecutive keys keeps its slot range
 * [cell_start[32b], cell_start[32b + 32]), inside which round r = 0, 1, ...
 * lists the r-th particle of every key of the block that holds more than r
 * particles, keys ascending.  perm[j] = index of the particle in slot j.
 * Latches OUT_OF_DOMAIN for particles outside the valid region. */
polypic_status polypic_sort(polypic_ctx *ctx, polypic_particles *p, void *ws, size_t ws_bytes,
                            void *stream);

/* P2G, Eqs 1-5 and 13 (fluid, Eqs 15-17; solid with m_s + m_abs, Eqs 18-19):
 *   m_ia  = sum_p mt_p w_ipa
 *   mv_ia = sum_p mt_p w_ipa sum_{r<N_r} c_pra s_r(x_ia - x_p)
 * with the modes evaluated at the particle's current position.  Needs
 * p->perm and p->cell_start from polypic_sort on the same positions.
 * Overwrites g->mass and g->mom (every face).  Deterministic: the result is
 * bit-identical from run to run (fixed summation order, no float atomics). */
polypic_status polypic_p2g(polypic_ctx *ctx, const polypic_particles *p, polypic_grid *g,
                           void *ws, size_t ws_bytes, void *stream);

/* P2G over a step of dt: polypic_p2g for the constant map; with
 * POLYPIC_MAP_AFFINE the modes are evaluated at Eq 12's mapped offsets
 * xi = (I + dt C_p)^-1 (x_ia - x_p) (for 4 modes this turns the linear
 * coefficients of component a into sum_b c_{a,1+b} M_bg, M = the inverse).
 * polypic_p2g and polypic_p2g_noalloc return INVALID_ARG on such contexts
 * (they have no dt); polypic_step passes its own.  Non-finite dt:
 * INVALID_ARG. */
polypic_status polypic_p2g_mapped(polypic_ctx *ctx, const polypic_particles *p, polypic_grid *g,
                                  float dt, void *ws, size_t ws_bytes, void *stream);

/* P2G exactly as polypic_p2g, but without a caller workspace: for callers
 * that cannot allocate device memory while they run, e.g. a host application
 * that reserves all of the GPU's memory at start-up and forbids allocation
 * afterwards, or code whose allocator may not be entered from where the
 * transfer is issued.  The paper has no counterpart; this is a deployment
 * convenience.  Its scratch is a fixed array built into the library (about
 * 33 MB, held on every GPU that loads the library until the process exits),
 * enough for grids of at most 2048 key tiles, i.e.
 * ceil(n_x/8) * ceil(n_y/8) * ceil(n_z/4) <= 2048 (64^3 uses 1024); larger
 * grids return POLYPIC_ERR_WORKSPACE before anything is launched.  The call
 * allocates nothing itself.  Every call made outside a stream capture looks
 * the array's device address up in the current CUDA context
 * (cudaGetSymbolAddress) and remembers it for that context; a call issued
 * while `stream` is being captured uses the remembered address (CUDA error
 * if there is none), so make one call on the context before capturing.
 * Every call shares the one array and it keeps the previous call's contents
 * (every launch writes each entry it later reads, so nothing needs
 * clearing); calls that overlap on the GPU, on any stream or context of the
 * process, race on it and must be serialised by the caller.  Inputs and
 * outputs are as for polypic_p2g. */
polypic_status polypic_p2g_noalloc(polypic_ctx *ctx, const polypic_particles *p, polypic_grid *g,
                                   void *stream);

/* Grid update (delegated to the host simulator by the paper; this minimal
 * form): v = mv/m where m > 0 else 0 (Eq 5, Eq 20 for the solid grid);
 * v~ = v + dt g; with a solid grid and drag_k > 0, implicit two-phase drag on
 * faces where both masses are positive, u' = u / (1 + dt K (1/m_f + 1/m_s))
 * for u = v_f - v_s, keeping the mass-weighted mean; v~_a = 0 on the wall
 * faces i_a in {0, n_a}; optional pressure projection (CG preconditioned by
 * a multigrid V-cycle on cells
 * holding fluid particles, FP64 dot products and norms) needs
 * fluid_particles->cell_start.  Writes fluid->vel (and solid->vel).
 * `solid` and `fluid_particles` may be NULL.  The projection runs its CG in
 * batches of 8 iterations between host reads of the residual (so it cannot
 * be captured into a CUDA graph by the caller); the context captures the
 * batches itself once per workspace address, on a stream of its own, keeps
 * them until polypic_destroy and replays them on `stream`.  A context must
 * not be used by two host threads at once. */
polypic_status polypic_grid_update(polypic_ctx *ctx, polypic_grid *fluid, polypic_grid *solid,
                                   const polypic_particles *fluid_particles,
                                   const polypic_update_params *params, void *ws,
                                   size_t ws_bytes, void *stream);

/* G2P (Eqs 6-8 per component, and the decoupled least-squares mode fit of
 * Section 3.3): c_pra = sum_i w s_r v~_ia / d_r with d_r = sum_i w s_r^2,
 * setting to 0 the coefficient of every mode with a quadratic factor on an
 * axis where the guard holds; v_p = c_p0; x_p <- clamp(x_p + dt v_p,
 * 1.5 dx, (n - 1.5) dx).  Reads `in` (positions, masses) through in->perm and
 * writes the new state of the particle in slot j = 0..count-1 to
 * out->x, out->mass, out->mass_abs (if non-NULL), out->coeff and
 * out->coeff_scale: `out` must not alias `in`. */
polypic_status polypic_g2p(polypic_ctx *ctx, const polypic_grid *g, const polypic_particles *in,
                           polypic_particles *out, float dt, void *ws, size_t ws_bytes,
                           void *stream);

/* One transfer step of each phase: sort, P2G, grid update, G2P
 * (Figure 2's step with PolyPIC transfers).  solid_in / solid_out / gs may be
 * NULL for a fluid-only step.  New states go to fluid_out / solid_out in
 * sorted order. */
polypic_status polypic_step(polypic_ctx *ctx, polypic_particles *fluid_in,
                            polypic_particles *fluid_out, polypic_particles *solid_in,
                            polypic_particles *solid_out, polypic_grid *gf, polypic_grid *gs,
                            const polypic_update_params *params, void *ws, size_t ws_bytes,
                            void *stream);

/* Fused transfer: the G2P of step n and the P2G of step n + 1 in one pass
 * (Section 3: only the transfers differ from the host simulator's step, so
 * the new coefficients can feed the next P2G directly).  From the grid
 * velocity g->vel (step n, after the update) and the sorted state `in`,
 * writes the new positions, masses (and m_abs) of every particle to `out` in
 * slot order, with the same bits as polypic_g2p, and the P2G of that new
 * state -- m and mv of Eqs 1-5 and 13 with the freshly fitted coefficients --
 * to g_next->mass and g_next->mom, without storing the coefficients of the
 * particles that stay in their cell: out->coeff receives only those of the
 * particles whose new position lies in another cell (the movers; the other
 * entries are left as they were).  The movers go through `spill`, a
 * caller-owned phase whose count is its capacity (x, mass, mass_abs when
 * `in` has it, coeff, key, perm, cell_start): more movers than that returns
 * POLYPIC_ERR_WORKSPACE, g_next then holding the stayers' share only.  The
 * host reads the mover count once (a stream synchronisation).  FP32
 * coefficients, constant map and the truncation fit only (UNSUPPORTED
 * otherwise).  Deterministic: bit-identical from run to run (its sums run
 * in another order than polypic_p2g's, so the two agree to rounding). */
polypic_status polypic_g2p2g(polypic_ctx *ctx, const polypic_grid *g,
                             const polypic_particles *in, polypic_particles *out,
                             polypic_particles *spill, polypic_grid *g_next, float dt, void *ws,
                             size_t ws_bytes, void *stream);

/* Fabric forces (stand-in): for every vertex particle of `solid` (id <
 * m^2), with d = x_j - x_i, L = |d|, e = d / L over the lattice neighbours
 * present, f = sum k (L - L0) e + c ((v_j - v_i) . e) e, and the velocity
 * (mode 0 of the coefficients, FP32 contexts only: UNSUPPORTED otherwise)
 * takes v_i += dt f / (m_i + m_abs,i), in place; all velocities are read
 * before any is written.  Needs solid->id and the workspace; the arrays may
 * be in any order (ids are unique). */
polypic_status polypic_fabric_forces(polypic_ctx *ctx, polypic_particles *solid,
                                     const polypic_fabric_params *fabric, float dt, void *ws,
                                     size_t ws_bytes, void *stream);

/* Absorption (stand-in), per cell, both phases sorted (polypic_sort): with
 * M_f the mass of the cell's fluid particles, each solid particle asks
 * d_p = min(rate dt m_s, max(0, capacity m_s - m_abs)), the cell gives
 * D = min(sum d_p, max_fraction M_f); solid particle p gains d_p D / sum d
 * (in solid->mass_abs), each fluid particle loses m_q D / M_f (in
 * fluid->mass).  The cell's total mass is kept; sums run in slot order
 * (deterministic).  In place. */
polypic_status polypic_absorb(polypic_ctx *ctx, polypic_particles *fluid,
                              polypic_particles *solid, const polypic_fabric_params *fabric,
                              float dt, void *stream);

/* polypic_step for a fluid and a fabric sheet with the stand-ins: sort both
 * phases, absorption, fabric forces (both in place on the input states), P2G
 * of both, the grid update (drag, projection), G2P of both, and the lattice
 * ids carried to solid_out->id through the solid's slot order.  Requires a
 * solid phase with ids (solid_in->id, solid_out->id). */
polypic_status polypic_step_coupled(polypic_ctx *ctx, polypic_particles *fluid_in,
                                    polypic_particles *fluid_out, polypic_particles *solid_in,
                                    polypic_particles *solid_out, polypic_grid *gf,
                                    polypic_grid *gs, const polypic_update_params *params,
                                    const polypic_fabric_params *fabric, void *ws,
                                    size_t ws_bytes, void *stream);

/* ---- adjoints (constant map) ---------------------------------------------- *
 * Contexts with POLYPIC_MAP_AFFINE (4 modes or more) or POLYPIC_APIC_GRAD_W get
 * UNSUPPORTED from the G2P adjoint, and with the affine map from the P2G
 * adjoint.
 * Transposes of the forward calls at the forward state.  Adjoint particle
 * data reuse polypic_particles (x[3] = dL/dx, coeff = dL/dc as float
 * [3][num_modes][count]) and adjoint grids reuse polypic_grid (mass = dL/dm,
 * mom = dL/d(mv), vel = dL/dv~).  Outputs are overwritten unless flags has
 * POLYPIC_ADJ_ACCUMULATE.  Supported for POLYPIC_COEFF_F32 only.            */

/* Adjoint of polypic_g2p at (g->vel, in positions): given bar_out->coeff and
 * bar_out->x (dL/d of the outputs, in sorted slot order), writes
 * bar_grid->vel = dL/dv~ and bar_in->x = dL/dx of the inputs (input order,
 * through in->perm), including the advection and the position dependence of
 * w, s_r and d_r.  Clamped axes pass no gradient. */
polypic_status polypic_g2p_adjoint(polypic_ctx *ctx, const polypic_grid *g,
                                   const polypic_particles *in, float dt,
                                   const polypic_particles *bar_out, polypic_grid *bar_grid,
                                   polypic_particles *bar_in, int32_t flags, void *ws,
                                   size_t ws_bytes, void *stream);

/* Adjoint of polypic_grid_update with the same params (the update is
 * delegated to the host simulator by the paper; this is the transpose of its
 * stated minimal form), last step first:
 *   projection (params->project): (P W)^T = P W -- walls then the projection
 *     form an orthogonal projector onto the discretely divergence-free
 *     fields of the fluid cells, so the wall-zeroed bar_fluid_out->vel is
 *     projected exactly as the forward projects a velocity (same fluid cells
 *     from fluid_particles->cell_start, same CG to params->pcg_rtol; needs
 *     the workspace; NOT_CONVERGED as for the forward, and then bar_fluid_in
 *     and bar_solid_in are not written);
 *   walls: no gradient on the wall faces;
 *   drag (solid grid, drag_k > 0, faces holding both masses): the
 *     transposed Jacobian of (v_f, v_s) -> (v_f', v_s') and the drag's
 *     derivatives in m_f and m_s (through the mean, the weights m/(m_f+m_s)
 *     and the factor 1/(1 + dt K (1/m_f + 1/m_s)));
 *   gravity: identity;
 *   v = mv/m: bar(mv) = bar v / m, bar m = (drag term) - bar v mv / m^2 on
 *     faces with m > 0; faces with m = 0 pass no gradient.
 * fluid / solid hold the forward's inputs (mass, mom).  Writes
 * bar_fluid_in->mass and ->mom (and bar_solid_in's with a solid grid) from
 * bar_fluid_out->vel (and bar_solid_out->vel).  solid, bar_solid_out and
 * bar_solid_in are all NULL or all set; fluid_particles and ws may be NULL
 * without the projection.  bar_fluid_in may be the same grid as
 * bar_fluid_out (its mass and mom are written, its vel only read), and
 * likewise for the solid. */
polypic_status polypic_grid_update_adjoint(polypic_ctx *ctx, const polypic_grid *fluid,
                                           const polypic_grid *solid,
                                           const polypic_particles *fluid_particles,
                                           const polypic_update_params *params,
                                           const polypic_grid *bar_fluid_out,
                                           const polypic_grid *bar_solid_out,
                                           polypic_grid *bar_fluid_in, polypic_grid *bar_solid_in,
                                           void *ws, size_t ws_bytes, void *stream);

/* Adjoint of polypic_p2g at the state `in`: given bar_grid->mass and
 * bar_grid->mom, writes bar_in->coeff = dL/dc and bar_in->x = dL/dx (input
 * order, through in->perm). */
polypic_status polypic_p2g_adjoint(polypic_ctx *ctx, const polypic_particles *in,
                                   const polypic_grid *bar_grid, polypic_particles *bar_in,
                                   int32_t flags, void *ws, size_t ws_bytes, void *stream);

/* ---- status -------------------------------------------------------------- */

/* Synchronises `stream`, returns the first latched device condition
 * (OUT_OF_DOMAIN, NONFINITE, NOT_CONVERGED, TIMEOUT) or OK, and clears it.
 * Returns CUDA if an earlier asynchronous launch failed. */
polypic_status polypic_check_device_status(polypic_ctx *ctx, void *stream);

/* Static description of a status code. */
const char *polypic_status_string(polypic_status s);

#ifdef __cplusplus
}
#endif

#endif /* POLYPIC_H */

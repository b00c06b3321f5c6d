/*
 * lbm.h -- C ABI of the GB300 (sm_103a) implementation of the coupled
 * three-lattice lattice Boltzmann (LB) time step for three-phase freezing of
 * Huang, Zhan, Chai & Huang, arXiv 2510.18688 ("A diffuse-interface method
 * for the containerless freezing of three-phase flows in complex
 * geometries").
 *
 * One context owns the device state of one 2-D D2Q9 grid: the flow
 * populations f (Sec. 3.1, Eqs. (11)-(17)), the phase-field populations g
 * (Sec. 3.2, Eqs. (18)-(22)), the total-enthalpy populations h (Sec. 3.3,
 * Eqs. (23)-(28)), the lagged fields one step needs (liquid fraction,
 * material weight, pressure, phi*u, enthalpy source) and the static solid
 * field phi0 (Sec. 2) with an optional cold mask.  Lattice units:
 * dx = dt = 1, cs^2 = 1/3, melting temperature T_m = 0.
 *
 * Conventions for every call:
 *   - Return value is an lbm_status; no call aborts or throws across the
 *     ABI.  lbm_last_error() describes the most recent failure of a context.
 *   - Grid arrays are row-major [ny][nx] with x fastest, no padding.
 *   - `where` is LBM_HOST (plain host memory, pinned or pageable) or
 *     LBM_DEVICE (device memory of the current CUDA device, for example
 *     torch.Tensor.data_ptr()).  Caller buffers stay owned by the caller and
 *     are only accessed during the call (device inputs until the call's work
 *     on `stream` completes).
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  lbm_step
 *     and lbm_compute_diagnostics only enqueue work; lbm_set_geometry with
 *     host inputs, lbm_read_fields with host outputs, lbm_read_diagnostics
 *     and the state calls synchronise the stream they use.
 *   - A context is not thread-safe; use one context per host thread.
 */
#ifndef LBM_GB300_H
#define LBM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;

typedef enum {
  LBM_OK = 0,
  LBM_ERR_ARG = -1,         /* null pointer, bad size or bad enum value      */
  LBM_ERR_PARAM = -2,       /* physically invalid parameter (tau <= 1/2 ...)  */
  LBM_ERR_CUDA = -3,        /* a CUDA runtime call failed                     */
  LBM_ERR_OOM = -4,         /* device or pinned host allocation failed        */
  LBM_ERR_NONFINITE = -5,   /* diagnostics found non-finite populations       */
  LBM_ERR_UNSUPPORTED = -6, /* valid request the library does not implement  */
  LBM_ERR_TIMEOUT = -7,     /* a kernel's bounded wait for its own tile copies
                               ran out (reported by the next synchronising
                               read; the state is then undefined)            */
  LBM_ERR_STATE = -8        /* call out of order (e.g. step before geometry)  */
} lbm_status;

/* Arithmetic and storage of the populations.  LBM_FP64: everything in
 * double.  LBM_FP32: populations, lag fields and arithmetic in float, with
 * well-balanced storage: every population that carries a large, slowly
 * varying part is stored as its difference from a reference that writer and
 * reader form identically from the lag fields (g0 from 2 w - 1 + phi0; h0
 * from the node's previous enthalpy state ell fl + (C - 5/9 rho_ref Cp_ref)
 * T; h_i, i > 0, from w_i rho_ref Cp_ref T of the node it is streamed to;
 * f_i from 3 (w_i - delta_i0) p of the node it is streamed from), so that
 * float rounds only the small remainders; the inversion of Eq. (8) near the
 * melting point (branch test, liquid fraction and its clamp) runs in FP64.
 * Float states carry one more lag plane, the temperature T of the previous
 * step.  LBM_FP16S: the same with the 27 populations in IEEE binary16.
 * Neither storage format is in the paper (which gives no precision);
 * LBM_FP16S trades accuracy for 169 instead of 277 bytes of state traffic
 * per node update.  Batches and lbm_diagnostics_noalloc do not take
 * LBM_FP16S (LBM_ERR_UNSUPPORTED). */
/* LBM_FP64_TANGENT: the FP64 step in forward-mode (dual-number)
 * arithmetic: every value carries its derivative with respect to the
 * parameter direction given by the tan_* fields of lbm_params (16 bytes per
 * population).  Branches (the inversion of Eq. (8), clamps) follow the
 * values, so the derivative is that of the branch taken.  Read the
 * derivatives with lbm_read_tangent_fields, lbm_read_tangent_diagnostics and
 * lbm_read_crossings_tangent; the values read as from an LBM_FP64 context.
 * Batches and lbm_diagnostics_noalloc do not take it. */
typedef enum { LBM_FP64 = 0, LBM_FP32 = 1, LBM_FP16S = 2, LBM_FP64_TANGENT = 3 } lbm_precision;

enum { LBM_BC_PERIODIC = 0, LBM_BC_DIRICHLET = 1, LBM_BC_ADIABATIC = 2 };
enum { LBM_LAT_FLOW = 1, LBM_LAT_PHASE = 2, LBM_LAT_HEAT = 4 };
enum { LBM_HOST = 0, LBM_DEVICE = 1 };

/* Field selection for lbm_read_fields (bit k selects out[k]). */
enum {
  LBM_F_PHI = 1u << 0,  /* order parameter phi, Eq. (22)                    */
  LBM_F_FS = 1u << 1,   /* solid fraction (pre-existing solid + ice)       */
  LBM_F_FL = 1u << 2,   /* liquid fraction of the material, Eq. (8)       */
  LBM_F_T = 1u << 3,    /* temperature, Eq. (8)                            */
  LBM_F_RHOH = 1u << 4, /* total enthalpy rho H, Eq. (28)                  */
  LBM_F_P = 1u << 5,    /* pressure, Eq. (17c)                             */
  LBM_F_UX = 1u << 6,   /* velocity x, Eq. (17b)                           */
  LBM_F_UY = 1u << 7,   /* velocity y, Eq. (17b)                           */
  LBM_F_RHO = 1u << 8,  /* density, Eq. (10)                               */
  LBM_F_MU = 1u << 9,   /* chemical potential mu_phi, Eq. (6)              */
  LBM_F_W = 1u << 10,   /* material (liquid-side) weight (1 - phi0 + phi)/2 */
  LBM_F_MDOT = 1u << 11 /* mass source (1 - rho_s/rho_l) dfs/dt, Eq. (1)   */
};
#define LBM_NUM_FIELDS 12

/* Problem statement (Secs. 2-4).  Densities, viscosities (dynamic),
 * conductivities and specific heats are given per phase: liquid l, solid s
 * (ice and the pre-existing solid Omega_0), gas g; each property is
 * interpolated by Eq. (10).  latent = L with Ste = Cp_l (T_m - T_w) / L,
 * Eq. (29).  rho_ref multiplies Cp_ref = 2 Cp_s Cp_l / (Cp_s + Cp_l) in the
 * enthalpy equilibrium Eq. (25) and in Eq. (26).  sigma, eps: surface
 * tension and interface width of Eq. (4); mobility = M of Eq. (21) with the
 * factor eta; theta_deg: contact angle on Omega_0, psi_deg: angle on the ice
 * (Eq. (4)).  (gx, gy): body force G = rho g.  T_cold: temperature imposed on
 * cold-mask nodes.  bc[k] for x-low, x-high, y-low, y-high; T_wall[k] used
 * where bc[k] == LBM_BC_DIRICHLET.  readings: bit 0 selects the variant of
 * the modified force that adds cs^2 S I to u Ft + Ft u in Eq. (16).
 * diag_every = k > 0 makes every k-th step also reduce the diagnostics of
 * its input state (0: only on request). */
typedef struct {
  int32_t nx, ny;
  int32_t precision; /* lbm_precision */
  uint32_t lattices; /* LBM_LAT_* bits */
  int32_t bc[4];
  double T_wall[4];
  double rho_l, rho_s, rho_g;
  double mu_l, mu_s, mu_g;
  double lambda_l, lambda_s, lambda_g;
  double cp_l, cp_s, cp_g;
  double rho_ref, latent;
  double sigma, eps, mobility, eta;
  double theta_deg, psi_deg;
  double gx, gy;
  double T_cold;
  uint32_t readings;
  int32_t diag_every;
  /* LBM_FP64_TANGENT only: the parameter direction s along which the state
   * is differentiated, as the rates dT_wall[k]/ds, dT_cold/ds,
   * dtheta_deg/ds and dlatent/ds (e.g. tan_T_cold = 1 for d/dT_cold;
   * tan_latent = -latent / Ste for d/dSte, since latent = Cp_l (T_m - T_w) /
   * Ste).  Ignored by the other precisions. */
  double tan_T_wall[4];
  double tan_T_cold, tan_theta_deg, tan_latent;
} lbm_params;

/* Global FP64 sums over the grid of one state (the conservation and
 * frozen-fraction monitors of Secs. 4.1-4.6). */
typedef struct {
  double mass;            /* sum rho                                        */
  double material_mass;   /* sum w (rho_s (1 - fl) + rho_l fl)              */
  double rhoH;            /* sum rho H                                      */
  double liquid_volume;   /* sum w fl                                       */
  double material_volume; /* sum w                                          */
  double frozen_volume;   /* sum w (1 - fl)                                 */
  double phi_sum;         /* sum phi                                        */
  double kinetic;         /* sum rho |u|^2 / 2                              */
  double nonfinite;       /* nodes whose population sums are not finite     */
  int64_t step;           /* index of the state these sums describe        */
} lbm_diag;

/* Validates *params, derives the relaxation times (Sec. 3: tau_f = nu/cs^2
 * + 1/2 per node, tau_g from Eq. (21), tau_a from Eq. (26), tau_s from
 * Eq. (27)) and allocates the device state on the current CUDA device.
 * Errors: LBM_ERR_ARG (null, grid < 2, unpaired periodic axis, a grid whose 27
 * population planes would pass 2^31 elements: about 79 million nodes),
 * LBM_ERR_PARAM (non-positive property, relaxation time <= 1/2 for any
 * phase), LBM_ERR_OOM, LBM_ERR_CUDA.  On success *out owns the memory until
 * lbm_destroy. */
int lbm_create(const lbm_params* params, lbm_ctx** out);

/* Sets the static solid field phi0 (1 in Omega_0, 0 in the fluid), the
 * optional cold mask (nonzero = enthalpy reset to T_cold each step; may be
 * NULL) and the initial phi, T and fl, then builds the initial populations:
 * f at rest (p = 0, u = 0), g = g_eq(phi, mu_phi, u = 0) (Eq. (19)),
 * h = h_eq(rho H, T, u = 0) (Eq. (25)); lag fields fl, w from the inputs,
 * p = phi u = Q = 0.  All five arrays are [ny][nx] doubles (mask: bytes) in
 * `where` memory.  Resets the step counter.  Synchronises `stream` when
 * where == LBM_HOST. */
int lbm_set_geometry(lbm_ctx* ctx, const double* phi0, const uint8_t* cold_mask,
                     const double* phi, const double* T, const double* fl, int where,
                     void* stream);

/* Enqueues nsteps >= 0 fused time steps on `stream` (enthalpy
 * inversion, order parameter and properties, finite-difference stencils and
 * chemical potential, velocity and pressure, three collisions, streaming
 * with wall conditions and cold mask, lag store; diagnostics every
 * diag_every steps).  Asynchronous.  Whole periods of the step sequence
 * (a multiple of 2 and of diag_every, at least 32 steps; none above 256)
 * are replayed from a CUDA graph captured once per context on a private
 * stream, so a long call costs one graph launch per period instead of one
 * kernel launch per step; the kernels and their order are those of single
 * steps, so results do not depend on how steps are grouped into calls.  No
 * graph is used when `stream` is itself being captured, or when the
 * environment sets LBM_STEP_GRAPHS=0 at lbm_create.  Errors: LBM_ERR_STATE
 * before lbm_set_geometry, LBM_ERR_ARG for nsteps < 0, LBM_ERR_CUDA on
 * launch or capture failure. */
int lbm_step(lbm_ctx* ctx, int64_t nsteps, void* stream);

/* Writes the fields selected by field_mask for the current state (the
 * values the next step would compute before its collisions), as [ny][nx] doubles,
 * into out[k] for every selected bit k (out[k] may be NULL otherwise).
 * where = LBM_HOST copies through a context-owned device staging buffer and
 * synchronises `stream`. */
int lbm_read_fields(lbm_ctx* ctx, uint32_t field_mask, double* const* out, int where,
                    void* stream);

/* Interface positions along one grid line of the current state, in node
 * coordinates along that line: out[0] = the largest coordinate at which phi
 * crosses 0 (the gas-liquid interface: the column height of the Stefan
 * problem of Sec. 4.2, the droplet tip height of Secs. 4.3-4.4 when the line
 * is the droplet axis), out[1] = the largest at which the frozen material
 * fraction w (1 - fl) crosses 1/2 (the ice front).  Between neighbouring
 * nodes k and k+1 with values a and b a crossing happens when exactly one of
 * a, b is <= the level, at k + a / (a - b) (linear interpolation); NaN where
 * the line has none.  axis 0: along x on row y = index; axis 1: along y on
 * column x = index; the line does not wrap across a periodic edge.
 * out: host memory for 2 doubles.  Runs the field read-out and a one-CTA
 * kernel on `stream` using the context's staging memory (allocated on first
 * use, as lbm_read_fields with LBM_HOST does) and synchronises `stream`.
 * Errors: LBM_ERR_ARG (null, bad axis, index outside the grid),
 * LBM_ERR_STATE before lbm_set_geometry, LBM_ERR_OOM/LBM_ERR_CUDA. */
int lbm_read_crossings(lbm_ctx* ctx, int axis, int index, double* out, void* stream);

/* LBM_FP64_TANGENT contexts: the derivatives of the fields selected by
 * field_mask along the context's parameter direction, laid out and copied as
 * lbm_read_fields does.  Errors: LBM_ERR_UNSUPPORTED for other precisions,
 * as lbm_read_fields otherwise. */
int lbm_read_tangent_fields(lbm_ctx* ctx, uint32_t field_mask, double* const* out, int where,
                            void* stream);

/* LBM_FP64_TANGENT contexts: out[0..1] as lbm_read_crossings, out[2..3] their
 * derivatives along the parameter direction (at a crossing between nodes k
 * and k+1 with values a, b and derivatives a', b': (a b' - b a') / (a - b)^2;
 * NaN where there is no crossing).  out: host memory for 4 doubles. */
int lbm_read_crossings_tangent(lbm_ctx* ctx, int axis, int index, double* out, void* stream);

/* Enqueues the diagnostic reduction of the current state (no time step). */
int lbm_compute_diagnostics(lbm_ctx* ctx, void* stream);

/* Synchronises the context's last stream and copies the most recent
 * diagnostics into *out.  Returns LBM_ERR_NONFINITE (with *out filled) when
 * any node's populations were not finite, LBM_ERR_STATE if no diagnostics
 * were ever computed. */
int lbm_read_diagnostics(lbm_ctx* ctx, lbm_diag* out);

/* LBM_FP64_TANGENT contexts: the derivatives of the nine sums of the most
 * recent diagnostics along the parameter direction (nonfinite: 0), with
 * out->step the state index they belong to.  Synchronises as
 * lbm_read_diagnostics.  Errors: LBM_ERR_UNSUPPORTED for other precisions,
 * LBM_ERR_STATE if no diagnostics were computed. */
int lbm_read_tangent_diagnostics(lbm_ctx* ctx, lbm_diag* out);

/* Bytes of a checkpoint (populations, lag fields, step counter, header). */
int lbm_state_size(const lbm_ctx* ctx, size_t* bytes);

/* Copies the current state into host_buf (capacity >= lbm_state_size).
 * Synchronises `stream`.  Restoring it with lbm_load_state into a context
 * with the same parameters and geometry reproduces later steps bit for bit. */
int lbm_save_state(lbm_ctx* ctx, void* host_buf, size_t capacity, void* stream);
int lbm_load_state(lbm_ctx* ctx, const void* host_buf, size_t size, void* stream);

/* Number of time steps taken since lbm_set_geometry (or restored). */
int64_t lbm_step_count(const lbm_ctx* ctx);

const char* lbm_last_error(const lbm_ctx* ctx);
const char* lbm_status_string(int status);

/* The source hash the library was built from: the first 16 hex digits of
 * the SHA-256 of every kernel and host source file, this header and the
 * compile flags (a static string, never NULL; "unknown" for a build that
 * did not define it).  No counterpart in the paper: it ties a loaded binary
 * to its sources. */
const char* lbm_source_hash(void);

/* Frees the context and all memory it owns (NULL is allowed). */
void lbm_destroy(lbm_ctx* ctx);

/* A batch groups `count` existing contexts of the same precision (grids of
 * any sizes, parameters and geometries, each stepped by Eqs. (11)-(25) as
 * lbm_step does) so that lbm_batch_step advances all of them together: one
 * launch per time step and per 64 grids covers the concatenated tile lists
 * of those grids, each tile evaluated by the same code as in lbm_step (the
 * results agree to the last bit where the compiler contracts both kernels'
 * copies of the arithmetic alike, as the FP64 build does, and otherwise to a
 * few roundings of the working precision).  This is how
 * many small problems fill the GPU.  LBM_FP32 batches run as the batched
 * TMA-staged tile kernel (each tile's inputs copied to shared memory by the
 * tensor copies of its own context, one CTA per 32 x 8 tile; a copy that
 * does not arrive within the bounded wait makes that context's next read
 * return LBM_ERR_TIMEOUT), LBM_FP64 batches, and LBM_FP32 batches under the
 * environment variable LBM_BATCH_KERNEL=fused, as the one-CTA-per-tile
 * kernel loading from global memory.  The batch holds the context pointers
 * only and allocates no device memory; the contexts stay usable on their own
 * (lbm_step, lbm_read_fields, diagnostics, checkpoints) and must outlive the
 * batch.
 * Errors: LBM_ERR_ARG (null, count < 1, mixed precision, a context twice),
 * LBM_ERR_OOM (host memory). */
typedef struct lbm_batch lbm_batch;
int lbm_batch_create(lbm_ctx* const* ctxs, int count, lbm_batch** out);

/* Enqueues nsteps time steps of every context of the batch on `stream`
 * (host-asynchronous; diagnostics every diag_every steps of the first
 * context, for all contexts).  Whole periods are replayed from a captured
 * CUDA graph as in lbm_step (recaptured when a context's parity, geometry
 * or state changed since).
 * Errors: LBM_ERR_ARG (null batch, nsteps < 0), LBM_ERR_STATE if a context
 * has no geometry, LBM_ERR_CUDA. */
int lbm_batch_step(lbm_batch* batch, int64_t nsteps, void* stream);

/* Frees the batch (not the contexts; NULL is allowed). */
void lbm_batch_destroy(lbm_batch* batch);

/* Testing hook for the failure paths (host-side fault injection): with
 * after >= 0, the (after + 1)-th device or pinned-host allocation that
 * lbm_create makes from now on fails as if the device were out of memory
 * (lbm_create then returns LBM_ERR_OOM and frees what it had allocated);
 * the hook disarms itself after firing.  after < 0 disarms it.  Process
 * wide; not for concurrent use with other lbm_create calls. */
void lbm_debug_fail_allocation(int after);

/* Testing hook for the bounded waits of the float step's TMA-staged tile
 * kernel (no device fault is involved): while on != 0, every such kernel
 * launched expects 16 bytes more than its tile copies deliver, so its first
 * wait runs out after about a second with nothing left in flight; the
 * kernel records it and the next lbm_read_fields or lbm_read_diagnostics of
 * the context returns LBM_ERR_TIMEOUT (the state is then undefined: set the
 * geometry again).  Process wide. */
void lbm_debug_tile_timeout(int on);

/* Reverse mode (adjoint) of the enthalpy-lattice step, Eqs. (8), (23)-(28)
 * with the fluid at rest: for a context with precision LBM_FP64 (a cold mask
 * allowed) and lattices == LBM_LAT_HEAT, or LBM_LAT_FLOW | LBM_LAT_HEAT with
 * rho_s == rho_l and no body force (then no mass source and no force ever
 * set the flow in motion, so its populations stay exactly zero: the
 * conduction-freezing column of Sec. 4.1), advances the state by nsteps
 * steps, as lbm_step
 * would, and returns the frozen fraction FF = sum w (1 - fl) / sum w of the
 * final state in *ff and its gradient in grad[0..5]: dFF/dT_wall[k] for the
 * four walls (zero where bc[k] is not LBM_BC_DIRICHLET), dFF/dlatent and
 * dFF/dT_cold (the cold-mask temperature; zero without a mask),
 * with the state at the start of the call held fixed, except that a call
 * right after lbm_set_geometry (step 0) includes the dependence of the
 * initial enthalpy populations on the latent heat (rho H = C T + w rho_l L
 * fl), so its gradient is that of the whole run from the initial fields.
 * The gradient comes from one reverse sweep of hand-written adjoint kernels
 * (the transposed step: pull through the push and the wall rules, then back
 * through the TRT collision and the enthalpy inversion, taking at its kinks
 * the branch the forward step took).  The forward pass keeps every
 * `every`-th state (checkpoints, 15 planes each); the sweep recomputes each
 * segment of `every` steps from its checkpoint before stepping back through
 * it, so memory is (nsteps / every + every) states.  Synchronises `stream`.
 * Errors: LBM_ERR_ARG (null output, nsteps < 1, every < 1), LBM_ERR_STATE
 * before lbm_set_geometry, LBM_ERR_UNSUPPORTED for other contexts,
 * LBM_ERR_OOM/LBM_ERR_CUDA (the context's state is then undefined). */
int lbm_adjoint_frozen_fraction(lbm_ctx* ctx, int64_t nsteps, int every, double* ff,
                                double* grad, void* stream);

/* Reverse mode (adjoint) of the phase-field step, Eqs. (6) and (18)-(21)
 * with the fluid at rest: for a context with precision LBM_FP64 and
 * lattices == LBM_LAT_PHASE (no velocity, no mass source: the modified
 * Cahn-Hilliard relaxation of a droplet on the solid phi0 with wetting),
 * advances the state by nsteps steps, as lbm_step would, and returns in
 * *pos the largest coordinate where phi crosses 0 along the grid line
 * (axis, index) of the final state, as out[0] of lbm_read_crossings (a
 * column: the tip height of a droplet; a row just above the substrate: its
 * contact line), and in grad[0..1] its derivatives with respect to the
 * contact angle theta (in degrees, through cos theta in Eq. (6)) and the
 * surface tension sigma.
 * The state at the start of the call is held fixed, except that a call
 * right after lbm_set_geometry (step 0) includes the dependence of the
 * initial phase populations on theta and sigma through their chemical
 * potential, so its gradient is that of the whole run from the initial
 * fields.  One reverse sweep of hand-written adjoint kernels: pull through
 * the push and bounce-back, back through the collision to mu_phi, and the
 * transposed Laplacian stencils (a gather in a fixed order: results are
 * deterministic) back to phi and fs; kinks of
 * the clamps take the branch the forward step took.  Checkpoints as in
 * lbm_adjoint_frozen_fraction.  *pos is NaN (and the gradient zero) when
 * phi does not cross 0 along the line.  Synchronises `stream`.
 * Errors: LBM_ERR_ARG (null output, nsteps < 1, every < 1, axis not 0 or 1,
 * index not a line of the grid), LBM_ERR_STATE before lbm_set_geometry,
 * LBM_ERR_UNSUPPORTED for other contexts or sigma == 0,
 * LBM_ERR_OOM/LBM_ERR_CUDA (the context's state is then undefined). */
int lbm_adjoint_crossing(lbm_ctx* ctx, int64_t nsteps, int every, int axis, int index,
                         double* pos, double* grad, void* stream);

/* Reverse mode (adjoint) of the coupled freezing step with the fluid at
 * rest: for a context with precision LBM_FP64, lattices == LBM_LAT_PHASE |
 * LBM_LAT_HEAT and sigma > 0 (a cold mask allowed), the phase field and the enthalpy
 * lattice coupled as in the full step (the mass source of Eq. (1) in the
 * order parameter, Eq. (22), and in the phase source, Eq. (20); w and
 * fs = phi0 + w (1 - fl) in the properties of Eq. (10) and in Eq. (6); the
 * lagged w in the inversion of Eq. (8)).  Advances the state by nsteps steps
 * as lbm_step would and returns in *value the observable of the final
 * state -- observable 0: the frozen fraction FF = sum w (1 - fl) / sum w;
 * observable 1: the last phi = 0 crossing along grid line (axis, index), as
 * out[0] of lbm_read_crossings -- and in grad[0..7] its derivatives with
 * respect to T_wall[0..3] (zero where bc[k] is not LBM_BC_DIRICHLET), the
 * latent heat L, the contact angle theta (degrees), sigma and the cold-mask
 * temperature T_cold (zero without a mask).  The state at
 * the start of the call is held fixed, except that a call right after
 * lbm_set_geometry (step 0) includes the initial populations' dependence on
 * L, theta and sigma.  Checkpoints and kinks as in
 * lbm_adjoint_frozen_fraction and lbm_adjoint_crossing.  Synchronises
 * `stream`.  Errors: LBM_ERR_ARG (null output, nsteps < 1, every < 1,
 * observable not 0 or 1, a bad line), LBM_ERR_STATE before
 * lbm_set_geometry, LBM_ERR_UNSUPPORTED for other contexts,
 * LBM_ERR_OOM/LBM_ERR_CUDA (the context's state is then undefined). */
int lbm_adjoint_freezing(lbm_ctx* ctx, int64_t nsteps, int every, int observable, int axis,
                         int index, double* value, double* grad, void* stream);

/* Reverse mode (adjoint) of the whole coupled step: as lbm_adjoint_freezing
 * for a context with precision LBM_FP64, all three lattices, readings == 0
 * and sigma > 0 (a cold mask allowed), with the flow lattice moving -- the velocity
 * of Eq. (17a,b) with the surface-tension, body and penalty forces, the
 * source S and the modified force of Eq. (16) (with the lagged pressure
 * gradient), the pressure of Eq. (17c), the flow collision, and phi u and u
 * in the phase and enthalpy equilibria all reversed, with the transposed
 * gradients of phi, rho and the lagged pressure.  grad[0..9]: d/dT_wall[0..3],
 * d/dL, d/dtheta_deg, d/dsigma, d/dgx, d/dgy, d/dT_cold (the cold-mask
 * temperature; zero without a mask).  dT0 (host memory for
 * [ny][nx] doubles, or NULL): the gradient with respect to the initial
 * temperature field of lbm_set_geometry, node by node (the call must then
 * start at step 0, else LBM_ERR_STATE).  Other errors as
 * lbm_adjoint_freezing. */
int lbm_adjoint_coupled(lbm_ctx* ctx, int64_t nsteps, int every, int observable, int axis,
                        int index, double* value, double* grad, double* dT0, void* stream);

/* Autotuner (the paper gives no implementation; a measuring aid of this
 * library): times the step forms the library has on the context's own grid
 * and state and keeps the fastest for later lbm_step calls.  Variant v is
 * kernel form v / 2 with captured periods of at least 32 steps (v even) or
 * 256 (v odd).  Kernel forms (form ids; a context times those it has):
 * 0 one CTA per 32 x 8 tile loading from global memory (every precision);
 * 1 LBM_FP32/LBM_FP16S: the TMA-staged tile kernel with one shared-memory
 * stage and one CTA per tile, LBM_FP64: the two-kernel split; 2 (float) the
 * TMA-staged kernel with two stages and two persistent CTAs per
 * multiprocessor (the copies of the next tile overlap the current one);
 * 3 (float) one stage and three persistent CTAs per multiprocessor; 4 one
 * CTA per 32 x 4 tile; 5 one CTA per 32 x 16 tile (4 and 5: LBM_FP32,
 * LBM_FP16S, LBM_FP64).  Tangent
 * contexts 0.  Each variant runs steps_per_trial steps twice from the same
 * saved state (the first run warms up and captures; the second is timed
 * with CUDA events on `stream`).  The fastest variant is kept, unless the
 * context's current one is within 2 % of it (then the current one stays).
 * The state, step counter and diagnostics
 * (including partial sums not yet read) are restored afterwards, so the
 * call does not advance the simulation.  out_us (12 doubles, may be NULL):
 * microseconds per step of each variant (-1 where not run); chosen (may be
 * NULL): the index kept.  The environment variable LBM_KERNEL_FORM=<form id>
 * read by lbm_create selects a form without timing (ignored where the
 * context does not have it).  Allocates a backup of the state (its population
 * and lag planes) for the duration of the call and synchronises `stream`.
 * Errors: LBM_ERR_ARG (steps_per_trial < 2), LBM_ERR_STATE before
 * lbm_set_geometry, LBM_ERR_OOM/LBM_ERR_CUDA. */
int lbm_autotune(lbm_ctx* ctx, int steps_per_trial, void* stream, double* out_us, int* chosen);

/* Largest grid lbm_diagnostics_noalloc accepts, in tiles of 32 x 8 nodes
 * (4096 tiles = 1,048,576 nodes, e.g. 1024 x 1024). */
#define LBM_NOALLOC_MAX_BLOCKS 4096

/* Diagnostics of a state the caller holds, without any device allocation.
 * The paper has no counterpart: this is a service of the library.
 *
 * Who needs it: callers that may not call cudaMalloc -- code that runs inside
 * a framework whose caching allocator or fixed memory pool owns all device
 * memory, latency-critical loops where the implicit synchronisation of an
 * allocation is not acceptable, and plug-ins that are handed device buffers
 * but are not allowed to create their own.  Everything else should use a
 * context and lbm_compute_diagnostics.
 *
 * Inputs (device memory of the current device, element type float for
 * LBM_FP32 and double for LBM_FP64 in params->precision): `pops`, 27 planes
 * in the order f0..f8, g0..g8, h0..h8; `lags`, 6 planes in the order fl, w,
 * p, phi ux, phi uy, Q (LBM_FP64) or 7 planes, the same and T (LBM_FP32,
 * whose populations are stored in the well-balanced form of LBM_FP32);
 * `phi0`, one plane; `cold_mask`, one plane of bytes or
 * NULL.  A plane holds ny rows of pitch elements, pitch = nx rounded up to a
 * multiple of 32, and planes start every `plane` elements, plane =
 * pitch * ny rounded up to a multiple of 64.  This is the layout that
 * lbm_save_state writes after its header.  Output: `out`, device memory for
 * 10 doubles, receives the nine sums of lbm_diag in declaration order and 0.
 *
 * Scratch: the per-tile partial sums live in one static device array of
 * LBM_NOALLOC_MAX_BLOCKS * 9 doubles (288 KB) that every device which loads
 * the library keeps until the process exits.  Each call overwrites the slots
 * it uses before a second kernel on `stream` sums them, so nothing needs
 * clearing, but all calls share the array: calls whose work overlaps on the
 * GPU (different streams without ordering) race and give wrong sums.  The
 * first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and keeps it for the life of the process (safe
 * against concurrent first calls), so make that first call before any
 * stream capture; after cudaDeviceReset of a device the kept address is
 * stale, and this entry point must not be called on that device again.
 * Enqueues on `stream`; does not synchronise.
 *
 * Errors: LBM_ERR_ARG for a null pointer or invalid grid, LBM_ERR_PARAM for
 * invalid parameters (the checks of lbm_create), LBM_ERR_UNSUPPORTED for a
 * grid of more than LBM_NOALLOC_MAX_BLOCKS tiles or a precision other than
 * LBM_FP32 and LBM_FP64 (message on stderr),
 * LBM_ERR_CUDA if the address lookup or the launch fails.  No call to
 * cudaMalloc, cudaFree or any allocating library routine is made. */
int lbm_diagnostics_noalloc(const lbm_params* params, const void* pops, const void* lags,
                            const void* phi0, const uint8_t* cold_mask, double* out,
                            void* stream);

/* Measures the fused multiply-add throughput of the current device in the
 * given precision (LBM_FP64 or LBM_FP32): 8 CTAs per SM run independent FMA
 * chains; the best of three timed launches (after one warm-up) gives
 * *flops_per_s = 2 * FMAs / time.  It is the arithmetic ceiling of the
 * double-precision step, which the FP64 pipe, not its HBM traffic, bounds
 * on this part (the paper gives no cost model; this is a measuring aid).
 * Runs on `stream` and synchronises it; allocates and frees a small output
 * buffer (8 x 256 x SMs elements).  Takes tens of milliseconds.
 * Errors: LBM_ERR_ARG (null output, other precision), LBM_ERR_OOM,
 * LBM_ERR_CUDA. */
int lbm_probe_fma_rate(int precision, double* flops_per_s, void* stream);

/* ------------------------------------------------------------------------
 * Three-dimensional contexts: the same coupled step on the D3Q19 lattice of
 * Sec. 3.1 (Eq. (13): weights 1/3, 1/18 for the six axes, 1/36 for the
 * twelve edge diagonals), as used for the rough-fracture case of Sec. 4.5.
 * Every lattice sum of Eqs. (11)-(28) runs over the 19 velocities, vectors
 * (velocity, forces, phi u, gradients) carry a z component, and the
 * isotropic stencils use the D3Q19 weights.  A link that leaves through an
 * edge or a corner of the grid is decided by the first wall it crosses in the
 * order x, y, z.  Grid arrays are [nz][ny][nx] with x fastest.  Precisions:
 * LBM_FP32, LBM_FP64 and LBM_FP64_TANGENT (FP64 values with their
 * derivatives along the direction of base.tan_* and tan_T_wall_z, read with
 * lbm3_read_tangent_fields and lbm3_read_tangent_diagnostics); LBM_FP16S:
 * LBM_ERR_UNSUPPORTED.  base.diag_every is ignored.  A step is two kernels (the per-node local
 * state, then stencils, collisions and streaming).  The conventions of the
 * 2-D calls apply (status codes, `where`, streams, ownership).
 * ---------------------------------------------------------------------- */
typedef struct lbm3_ctx lbm3_ctx;

typedef struct {
  lbm_params base;    /* nx, ny, precision, lattices, physics; base.bc and
                         base.T_wall give the x and y faces, (gx, gy) the
                         x and y components of the body force */
  int32_t nz;         /* >= 2 */
  int32_t bc_z[2];    /* z-low, z-high (LBM_BC_*; periodic in pairs) */
  double T_wall_z[2]; /* used where bc_z[k] == LBM_BC_DIRICHLET */
  double gz;          /* z component of the body force G = rho g */
  double tan_T_wall_z[2]; /* LBM_FP64_TANGENT: dT_wall_z[k]/ds (the x and y
                             faces' rates are base.tan_T_wall) */
} lbm3_params;

/* Fields of lbm3_read_fields: bit k selects out[k], in this order. */
enum {
  LBM3_F_PHI = 1u << 0, LBM3_F_FS = 1u << 1, LBM3_F_FL = 1u << 2, LBM3_F_T = 1u << 3,
  LBM3_F_RHOH = 1u << 4, LBM3_F_P = 1u << 5, LBM3_F_UX = 1u << 6, LBM3_F_UY = 1u << 7,
  LBM3_F_UZ = 1u << 8, LBM3_F_RHO = 1u << 9, LBM3_F_MU = 1u << 10, LBM3_F_W = 1u << 11,
  LBM3_F_MDOT = 1u << 12
};
#define LBM3_NUM_FIELDS 13

/* Validates *params as lbm_create does (plus nz, bc_z and the size limit:
 * a plane of nx rounded up to 32 times ny times nz nodes must stay below
 * 2^31; the device memory, about 550 B per node in FP32, is the practical
 * limit: some 500 million nodes on 280 GB) and allocates the device
 * state (two population buffers of 57 planes, two lag buffers of 7 planes,
 * 8 local planes, phi0, the mask, and a 13-plane FP64 read-out buffer).
 * Errors: LBM_ERR_ARG, LBM_ERR_PARAM, LBM_ERR_UNSUPPORTED (precision),
 * LBM_ERR_OOM, LBM_ERR_CUDA. */
int lbm3_create(const lbm3_params* params, lbm3_ctx** out);

/* As lbm_set_geometry, with [nz][ny][nx] arrays. */
int lbm3_set_geometry(lbm3_ctx* ctx, const double* phi0, const uint8_t* cold_mask,
                      const double* phi, const double* T, const double* fl, int where,
                      void* stream);

/* Enqueues nsteps >= 0 steps on `stream` (two kernel launches per step).
 * Errors: LBM_ERR_STATE before lbm3_set_geometry, LBM_ERR_ARG, LBM_ERR_CUDA. */
int lbm3_step(lbm3_ctx* ctx, int64_t nsteps, void* stream);

/* The fields selected by field_mask (LBM3_F_*) of the current state, as
 * [nz][ny][nx] doubles in out[k]; host outputs synchronise `stream`. */
int lbm3_read_fields(lbm3_ctx* ctx, uint32_t field_mask, double* const* out, int where,
                     void* stream);

/* The FP64 diagnostic sums of the current state (lbm_diag; the kinetic
 * energy with all three velocity components).  Synchronises `stream`. */
int lbm3_diagnostics(lbm3_ctx* ctx, lbm_diag* out, void* stream);

/* LBM_FP64_TANGENT contexts: the derivatives of the selected fields of the
 * current state (as lbm3_read_fields), and of the sums of the most recent
 * lbm3_diagnostics call (nonfinite: 0).  LBM_ERR_UNSUPPORTED for other
 * precisions, LBM_ERR_STATE before any diagnostics. */
int lbm3_read_tangent_fields(lbm3_ctx* ctx, uint32_t field_mask, double* const* out, int where,
                             void* stream);
int lbm3_read_tangent_diagnostics(lbm3_ctx* ctx, lbm_diag* out);

/* Checkpoint and resume, as lbm_state_size / lbm_save_state /
 * lbm_load_state (57 population planes and 7 lag planes after a header). */
int lbm3_state_size(const lbm3_ctx* ctx, size_t* bytes);
int lbm3_save_state(lbm3_ctx* ctx, void* host_buf, size_t capacity, void* stream);
int lbm3_load_state(lbm3_ctx* ctx, const void* host_buf, size_t size, void* stream);

int64_t lbm3_step_count(const lbm3_ctx* ctx);
const char* lbm3_last_error(const lbm3_ctx* ctx);
void lbm3_destroy(lbm3_ctx* ctx);

/* The lattice the kernels use: c[3 i + a] = component a of velocity i and
 * w[i] its weight, i = 0 ... 18 in the order of Eq. (13).  Host only; needs
 * no device. */
void lbm3_lattice(int32_t* c, double* w);

#ifdef __cplusplus
}
#endif

#endif /* LBM_GB300_H */

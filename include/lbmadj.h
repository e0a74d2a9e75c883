/*
 * lbmadj.h -- C-ABI of the GB300 (sm_103a) discrete adjoint lattice Boltzmann
 * solver.
 *
 * The calls follow the problem statement of the paper (arXiv 2501.02161):
 *   lattice + stencil            Sec. 2.1, Eq. 2-5 (D2Q9, D3Q19)
 *   node flags                   Sec. 2.1, Eq. 7-9 (fluid, wall, inlet, outlet)
 *   design field gamma           Sec. 2.2, Eq. 11-12 (relaxed to [0, 1])
 *   relaxation time tau          Eq. 3 (nu = (tau - 1/2)/3)
 *   objective                    Eq. 34 (inlet pressure, steady form) and a
 *                                mean-temperature term for heat sinks (Sec. 3.3)
 *   forward, adjoint, dJ/dgamma  Eq. 35-37, 53-56 / 59-61 / 64-65, 66
 *   temperature lattice          Eq. 71 (D3Q7, coupled through the frozen flow)
 *
 * Conventions shared by every call
 *   - Every function returns an lbm_status (0 = success, > 0 = warning with
 *     usable results, < 0 = error).  lbm_last_error() gives a message.
 *   - Lattice nodes are numbered n = x + nx*(y + ny*z), x fastest.
 *   - Inputs are copied into buffers the context owns; the caller keeps
 *     ownership of what it passes.  Outputs go to caller-owned buffers.
 *   - A pointer argument with on_device != 0 is a CUDA device pointer on the
 *     context's device (for example torch.Tensor.data_ptr()); with
 *     on_device == 0 it is ordinary host memory.
 *   - dtype codes: LBM_DTYPE_F64 (double) or LBM_DTYPE_F32 (float).
 *   - Work is ordered after all work already queued on the stream given to
 *     lbm_set_stream (default: the legacy default stream), and that stream
 *     waits for the call's work before the call returns control to it.  Calls
 *     that report numbers (solves, lbm_get_*) synchronise.
 *   - A context is not thread-safe; distinct contexts are independent.
 *
 * Node flag byte (bit-exact, identical in every call):
 *   bits 0-2  type: 0 FLUID, 1 WALL (full-way bounce-back, no collision,
 *             Eq. 9), 2 VEL (Zou-He velocity, Eq. 7), 3 PRES (Zou-He fixed
 *             density, Eq. 8)
 *   bits 3-5  inward normal of an open boundary or heated wall:
 *             0 +x, 1 -x, 2 +y, 3 -y, 4 +z, 5 -z
 *   bit 6     on a WALL node, HEAT: adds q_flux per step to the temperature
 *             population along its normal; on a PRES node, temperature inlet:
 *             the temperature is held at T_in (bc value 3) instead of the
 *             outflow condition (a pressure-driven inlet, Eq. 70)
 *   bit 7     must be 0
 *
 * Boundary values, 4 numbers per node, read only at VEL / PRES nodes:
 *   VEL: (ux, uy, uz, T_in)       PRES: (rho, unused, unused, T_in if bit 6)
 *
 * Faces of the lattice box: streaming wraps periodically across them, unless
 * lbm_set_symmetry makes an axis reflect (symmetry planes half a node beyond
 * both of its faces).
 *
 * Population order (for lbm_get_adjoint / state export):
 *   D2Q9  : 0 rest, 1 +x, 2 +y, 3 -x, 4 -y, 5 (+,+), 6 (-,+), 7 (-,-), 8 (+,-)
 *           (the order Eq. 7-8 use)
 *   D3Q19 : 0 rest, 1 +x, 2 -x, 3 +y, 4 -y, 5 +z, 6 -z, 7 (1,1,0), 8 (-1,-1,0),
 *           9 (1,-1,0), 10 (-1,1,0), 11 (1,0,1), 12 (-1,0,-1), 13 (1,0,-1),
 *           14 (-1,0,1), 15 (0,1,1), 16 (0,-1,-1), 17 (0,1,-1), 18 (0,-1,1)
 *   D3Q7  : 0 rest, 1 +x, 2 -x, 3 +y, 4 -y, 5 +z, 6 -z
 */
#ifndef LBMADJ_H
#define LBMADJ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LBM_OK = 0,
    LBM_NOT_CONVERGED = 1,   /* step cap reached above tolerance; results kept */
    LBM_ERR_ARG = -1,        /* bad argument (null, size, code, range) */
    LBM_ERR_OOM = -2,        /* device allocation failed / budget exceeded */
    LBM_ERR_CUDA = -3,       /* a CUDA call failed; see lbm_last_error */
    LBM_ERR_DIVERGED = -4,   /* non-finite residual or objective */
    LBM_ERR_ORDER = -5,      /* call made before the step it depends on */
    LBM_ERR_UNSUPPORTED = -6 /* combination not built (e.g. D2Q9 + thermal) */
} lbm_status;

typedef enum { LBM_D2Q9 = 0, LBM_D3Q19 = 1 } lbm_stencil;

/* Population storage.  Flow populations are always held as offsets
 * h_i = f_i - w_i rho0.  FP16_OFS / BF16_OFS store the flow populations h in
 * 16 bits and compute in FP32; in those modes the adjoint and temperature
 * populations stay FP32 (their slowly converging linear iterations would
 * accumulate 16-bit rounding into percent-level errors). */
typedef enum { LBM_FP64 = 0, LBM_FP32 = 1, LBM_FP16_OFS = 2, LBM_BF16_OFS = 3 } lbm_storage;

typedef enum { LBM_DTYPE_F64 = 0, LBM_DTYPE_F32 = 1 } lbm_dtype;

/* How gamma enters the equilibrium.  EQ12: u <- gamma u inside Eq. 4, as
 * Eq. 12 writes it.  LINEAR: f^eq = w (rho + gamma rho0 [...](u)), the model
 * whose gamma-derivative is the bracket printed in Eq. 66.  Both agree for
 * binary designs (Eq. 11) and both give the momentum drag (1-gamma)/tau. */
typedef enum { LBM_GAMMA_EQ12 = 0, LBM_GAMMA_LINEAR = 1 } lbm_gamma_model;

typedef struct {
    double tau;        /* flow relaxation time, > 0.5 (Eq. 2-3) */
    double rho0;       /* constant density of the incompressible model (Eq. 4) */
    int gamma_model;   /* lbm_gamma_model */
    double kappa_f;    /* fluid thermal diffusivity; tau_g = 1/2 + 4 kappa(gamma) */
    double k_ratio;    /* solid/fluid conductivity ratio: kappa = kappa_f (gamma + (1-gamma) k_ratio) */
    double q_flux;     /* heat per step added at HEAT wall nodes */
    double T0;         /* initial temperature (and 16-bit storage offset) */
    double beta_max;   /* heat generation in the solid, Q = beta_max (1 - gamma)(1 - T), added as
                          w_k Q in the temperature collision (Eq. 69, 71); 0 switches it off */
} lbm_params;

typedef struct {
    double w_pin;      /* weight of J_p = (1/(3 N_in)) sum_{VEL nodes} rho  (Eq. 34, steady) */
    double w_tmean;    /* weight of J_T = (1/N_nonwall) sum_{non-wall nodes} T */
    double w_qgen;     /* weight of J_Q = -sum_{non-wall nodes} Q (Eq. 72), Q of Eq. 69 */
} lbm_objective;

/* The problem in the paper's physical terms (Sec. 2.1, Eq. 3; Sec. 3.3):
 *   nu = U L / Re,  tau = 1/2 + 3 nu                      (Eq. 3, c_s^2 = 1/3)
 *   U  = u_ref, or sqrt(dp / rho0) when u_ref <= 0 and dp > 0: the velocity
 *        estimated from a pressure drop dp = p_in - p_out (Eq. 70, the
 *        pressure-driven heat sink)
 *   kappa_f = nu / Pr                                     (Pr = nu / kappa_f)
 * lbm_physics_to_params does the conversion (host only, no device needed);
 * lbm_set_physics converts and then behaves as lbm_set_params. */
typedef struct {
    double re;         /* Reynolds number, > 0 */
    double u_ref;      /* velocity scale U (lattice units), e.g. the inlet's peak speed */
    double l_ref;      /* length scale L (nodes), e.g. the inlet width; > 0 */
    double dp;         /* pressure drop defining U when u_ref <= 0 (Eq. 70) */
    double pr;         /* Prandtl number (> 0 with the thermal lattice; unused without) */
    double rho0;       /* as in lbm_params */
    int gamma_model;
    double k_ratio;
    double q_flux;
    double T0;
    double beta_max;
} lbm_physics;

/* tau and kappa_f from Re, U, L and Pr; the other fields are copied.
 * Errors: LBM_ERR_ARG (null, re <= 0, l_ref <= 0, no velocity scale,
 * rho0 <= 0, pr < 0, non-finite values). */
lbm_status lbm_physics_to_params(const lbm_physics* ph, lbm_params* out);

typedef struct {
    double tol;          /* stop when |I(t)-I(t-K)|/|I(t)| < tol; tol <= 0: run exactly max_steps */
    long long max_steps; /* step cap (or exact count when tol <= 0); >= 0 */
    int check_every;     /* K, steps between residual checks (> 0; the paper uses 1000) */
    int reset;           /* 1: restart from the initial state; 0: continue from the populations
                            left by the previous solve of this phase (a warm start that stays
                            valid across lbm_set_gamma / set_bc_values / set_params; lbm_set_flags
                            and a diverged solve discard it) */
} lbm_solve_opts;

typedef struct {
    long long steps;     /* steps taken in this call */
    double residual;     /* last |I(t)-I(t-K)|/|I(t)| */
    double I;            /* last residual quantity (mean |u|, mean T, mean sum |f*|) */
    double J;            /* objective at the last check (forward calls) */
    double ms;           /* wall time of the call in milliseconds */
    int status;          /* lbm_status of the phase */
} lbm_report;

typedef struct lbm_ctx lbm_ctx;

/* Create a context for an nx*ny*nz lattice (nz = 1 for D2Q9).  Allocates all
 * device state (populations double-buffered, adjoint, frozen fields).
 * thermal != 0 adds the D3Q7 temperature lattice (D3Q19 only).
 * Errors: LBM_ERR_ARG (sizes <= 0, nz != 1 for D2Q9, unknown codes),
 * LBM_ERR_UNSUPPORTED (thermal with D2Q9), LBM_ERR_OOM, LBM_ERR_CUDA. */
lbm_status lbm_create(lbm_ctx** out, int stencil, int nx, int ny, int nz, int storage,
                      int thermal);
/* Free every device buffer the context owns.  Null is accepted. */
void lbm_destroy(lbm_ctx* ctx);

/* Order the context's work after the given cudaStream_t (e.g.
 * torch.cuda.current_stream().cuda_stream; 0 = legacy default stream). */
lbm_status lbm_set_stream(lbm_ctx* ctx, void* cuda_stream);

/* Node flags, n = nx*ny*nz bytes, layout above.  Rejects bit 7, unknown
 * types, and open boundaries whose normal is not along an axis of the lattice
 * (LBM_ERR_ARG).  Invalidates forward and adjoint results. */
lbm_status lbm_set_flags(lbm_ctx* ctx, const uint8_t* flags, size_t n, int on_device);
/* Design field gamma in [0, 1], n values of dtype (Eq. 11-12). */
lbm_status lbm_set_gamma(lbm_ctx* ctx, const void* gamma, size_t n, int dtype, int on_device);
/* Boundary values, n = 4*nx*ny*nz values of dtype, layout above. */
lbm_status lbm_set_bc_values(lbm_ctx* ctx, const void* values, size_t n, int dtype,
                             int on_device);
/* Physical parameters.  tau <= 0.5, rho0 <= 0, kappa_f < 0 with thermal on,
 * k_ratio <= 0, beta_max < 0 (or != 0 without the thermal lattice) or an
 * unknown gamma model give LBM_ERR_ARG. */
lbm_status lbm_set_params(lbm_ctx* ctx, const lbm_params* p);
/* Parameters from Re, U, L and Pr (see lbm_physics); same errors as
 * lbm_physics_to_params and lbm_set_params (pr <= 0 with thermal on is
 * LBM_ERR_ARG). */
lbm_status lbm_set_physics(lbm_ctx* ctx, const lbm_physics* ph);
/* Objective weights.  Non-finite weights, or w_qgen != 0 without the
 * thermal lattice, give LBM_ERR_ARG. */
lbm_status lbm_set_objective(lbm_ctx* ctx, const lbm_objective* obj);

/* Which adjoint the flow-adjoint phase iterates.  DISCRETE (default) is the
 * paper's method (Eq. 53-65: the exact transpose of the forward step).
 * CONTINUOUS is the comparison the paper argues against (Sec. 2.3, Eq. 23-32):
 * adjoint collision, backward streaming (Eq. 30), then the boundary rows of
 * the continuous Lagrangian -- Eq. 27 at fixed-density outlets, Eq. 29 at
 * velocity inlets, where the objective enters with 2 w_pin / (3 N_in) -- on
 * any face, bounce-back at walls.  It stores the post-collision values
 * C^T f* (what lbm_get_adjoint returns); its dJ/dgamma is Eq. 32 (without
 * lambda) on the f* those values give, the boundary rows applied to the
 * backward-streamed store: the iterate one step after the last step counted
 * (the same f* once converged).
 * Built for D2Q9 flow lattices without symmetry planes (else
 * LBM_ERR_UNSUPPORTED, also from lbm_adjoint).  Switching discards the
 * adjoint state.  Errors: LBM_ERR_ARG (unknown scheme). */
typedef enum { LBM_ADJOINT_DISCRETE = 0, LBM_ADJOINT_CONTINUOUS = 1 } lbm_adjoint_scheme;
lbm_status lbm_set_adjoint_scheme(lbm_ctx* ctx, int scheme);

/* Symmetry planes (the quarter-domain heat sink of Sec. 3.3): bit a of axes
 * makes streaming along axis a reflect at both faces of the box instead of
 * wrapping: a pull that leaves the box reads the image node in the plane half
 * a node beyond the face, with that component of the population's direction
 * reversed.  Streaming stays a permutation, so the adjoint (Eq. 61) is the
 * same reflection.  A face that is not meant as a plane carries walls or open
 * boundaries (whose pulls from outside the box are overwritten or never
 * read).  Default 0 (all periodic).  Errors: LBM_ERR_ARG (bits above 2; bit 2
 * for D2Q9). */
lbm_status lbm_set_symmetry(lbm_ctx* ctx, int axes);

/* Boundary values of one face of the lattice box (the per-node form is
 * lbm_set_bc_values).  face: the inward normal code of the face (0: x = 0,
 * 1: x = nx-1, 2: y = 0, 3: y = ny-1, 4: z = 0, 5: z = nz-1).  kind:
 * LBM_VEL (Zou-He velocity inlet, Eq. 7) or LBM_PRES (fixed-density outlet,
 * Eq. 8).  Only the nodes of that face whose flag is that kind with that
 * normal are written: values holds 4 numbers per such node, in increasing
 * node order ((ux, uy, uz, T_in) or (rho_out, 0, 0, 0)), or just 4 numbers
 * applied to all of them (n = 4).  Other nodes keep their values.  Needs
 * lbm_set_flags (LBM_ERR_ORDER).  Errors: LBM_ERR_ARG (bad face, kind or
 * dtype, no such node on the face, n neither 4 nor 4 x their count). */
enum { LBM_VEL = 2, LBM_PRES = 3 };
lbm_status lbm_set_bc(lbm_ctx* ctx, int face, int kind, const void* values, size_t n, int dtype,
                      int on_device);

/* Forward solve (Eq. 35): the flow to its residual tolerance, then, with the
 * thermal lattice on, the temperature with the converged velocity frozen.
 * Stores the frozen u (and T) the adjoint needs.  Returns LBM_NOT_CONVERGED
 * when a phase hits max_steps above tol, LBM_ERR_DIVERGED on non-finite
 * values.  rep may be null; rep->steps counts flow + thermal steps. */
lbm_status lbm_forward(lbm_ctx* ctx, const lbm_solve_opts* opts, lbm_report* rep);

/* Adjoint solve (Eq. 53-56 iterated to a fixed point from f*_C = 0): the
 * temperature adjoint first (thermal on), then the flow adjoint with the
 * thermal coupling term.  Needs a completed lbm_forward (else LBM_ERR_ORDER). */
lbm_status lbm_adjoint(lbm_ctx* ctx, const lbm_solve_opts* opts, lbm_report* rep);

/* The solve sequence phase by phase.  lbm_forward runs LBM_PHASE_FLOW then
 * (thermal on) LBM_PHASE_TEMPERATURE; lbm_adjoint runs (thermal on)
 * LBM_PHASE_TEMPERATURE_ADJOINT, the thermal-to-flow coupling, then
 * LBM_PHASE_FLOW_ADJOINT.  lbm_solve_phase runs one of them with its own
 * tolerance and step cap, so a caller can stop each phase where it wants (for
 * example: replay another solver's step counts phase by phase).  Order: the
 * temperature phase needs a completed flow phase (Eq. 71 runs on the frozen
 * converged flow); the temperature adjoint needs a completed forward; the
 * flow adjoint needs a completed forward and, thermal on, a completed
 * temperature adjoint (the coupling term of its source) -- else
 * LBM_ERR_ORDER.  opts->reset restarts the phase's populations; restarting the
 * flow phase also restarts the temperature populations, restarting the
 * temperature adjoint also restarts the flow adjoint.  A completed phase
 * invalidates the results of the phases after it.  rep (may be null) gets
 * this phase's steps, residual and I; rep->J is the objective so far.
 * Errors: LBM_ERR_ARG (unknown phase, temperature phase without the thermal
 * lattice), LBM_ERR_ORDER, LBM_ERR_DIVERGED; LBM_NOT_CONVERGED as lbm_forward. */
typedef enum {
    LBM_PHASE_FLOW = 0,
    LBM_PHASE_TEMPERATURE = 1,
    LBM_PHASE_FLOW_ADJOINT = 2,
    LBM_PHASE_TEMPERATURE_ADJOINT = 3
} lbm_phase;
lbm_status lbm_solve_phase(lbm_ctx* ctx, int phase, const lbm_solve_opts* opts, lbm_report* rep);

/* dJ/dgamma per node (Eq. 66 without the volume multiplier lambda, plus the
 * temperature terms when thermal is on), n = nx*ny*nz values of dtype into
 * caller memory.  Zero at WALL nodes.  Needs lbm_adjoint (LBM_ERR_ORDER). */
lbm_status lbm_sensitivity(lbm_ctx* ctx, void* out, int dtype, int on_device);

/* Macroscopic fields of the converged forward state, each n (rho, T) or 3n
 * (u, component-major: u[a*n + node]) values of dtype; any may be null.
 * T needs thermal on.  Needs lbm_forward (LBM_ERR_ORDER). */
lbm_status lbm_get_fields(lbm_ctx* ctx, void* rho, void* u, void* T, int dtype,
                          int on_device);

/* Objective J of the converged forward state (host double). */
lbm_status lbm_get_objective(lbm_ctx* ctx, double* J);

/* Adjoint populations after the adjoint boundary step (f* = B^T f*_C, the
 * stored iterate), Q*n values, population-major: fstar[i*n + node]; gstar:
 * 7*n values.  Either may be null. */
lbm_status lbm_get_adjoint(lbm_ctx* ctx, void* fstar, void* gstar, int dtype, int on_device);

/* Time plain fused steps of one phase: n steps (rounded up to even) are
 * captured as a CUDA graph, replayed once untimed, then replayed between two
 * CUDA events recorded on the context's stream; writes the mean milliseconds
 * per step of the timed replay (kernel time plus the gaps between graph
 * nodes).  phase: 0 flow forward, 1 temperature forward, 2 flow adjoint,
 * 3 temperature adjoint.  The 2n steps advance that phase's state as a solve
 * would; no reduction runs.  Needs the inputs set (LBM_ERR_ORDER) and, for
 * phases 1-3, a completed lbm_forward. */
lbm_status lbm_time_steps(lbm_ctx* ctx, int phase, int n, double* ms_per_step);

/* ---------------------------------------------------------------------------
 * Checkpoint / resume of a context's solver state (no counterpart in the
 * paper).  The state is the current forward and adjoint populations (and the
 * temperature ones), the frozen fields the adjoint reads, and the solve
 * bookkeeping (which phases completed, the last residual quantities, J); the
 * inputs (flags, gamma, BC values, parameters) are not part of it.  A state
 * imported into a context of the same shape, stencil, storage and thermal
 * setting, whose flags and parameters were set to the same values, continues
 * exactly as the exporting context would: a warm-started lbm_forward /
 * lbm_adjoint, lbm_sensitivity and lbm_get_fields give bit-identical results.
 * Use it to move a design's state off the device and back, or to checkpoint
 * a long solve.
 * --------------------------------------------------------------------------- */

/* Bytes lbm_export_state writes for this context (0 for a null context). */
size_t lbm_state_bytes(lbm_ctx* ctx);

/* Copy the state to dst (host memory, pinned or pageable, or device memory;
 * at least lbm_state_bytes(ctx) bytes, owned by the caller).  Synchronises.
 * Errors: LBM_ERR_ARG (null pointer, buffer too small), LBM_ERR_CUDA. */
lbm_status lbm_export_state(lbm_ctx* ctx, void* dst, size_t bytes);

/* Replace the context's state with one written by lbm_export_state.  The
 * flags and parameters must already be set to the values the state was
 * computed with (LBM_ERR_ARG otherwise, or when the shape, stencil, storage
 * or thermal setting differ, or the buffer is short); gamma may differ (a
 * warm start after a design update).  Synchronises.  Errors: LBM_ERR_ARG,
 * LBM_ERR_CUDA. */
lbm_status lbm_import_state(lbm_ctx* ctx, const void* src, size_t bytes);

/* ---------------------------------------------------------------------------
 * Batched solves (serving)
 *
 * A batch advances many resident contexts together: every call of
 * lbm_batch_step runs check_every steps of each admitted context's current
 * phase (flow, temperature, temperature adjoint, flow adjoint), then checks
 * each context's residual exactly as lbm_forward / lbm_adjoint do (same step
 * counts, same FP64 sums), so a context's results are bit-identical alone, in
 * any mix, and through the single-context calls.  A lattice at or above the
 * solo threshold (lbm_batch_set_solo_tiles; by default every lattice) runs its
 * K steps as its own single-lattice graph on its context's stream, all of
 * them concurrently; lattices below it are packed into one CUDA graph replay
 * of persistent kernels that walk the tiles of all packed lattices (each tile
 * one block of that lattice's single-lattice launch).  Contexts may be
 * admitted and retired between steps (continuous batching); admission never
 * re-captures the packed graph.  Built for D3Q19 with FP32, FP16_OFS or
 * BF16_OFS storage.
 * --------------------------------------------------------------------------- */
typedef struct lbm_batch lbm_batch;

/* Bytes of device memory lbm_create allocates for a context of this shape
 * (for admission by HBM footprint). */
size_t lbm_footprint_bytes(int stencil, int nx, int ny, int nz, int storage, int thermal);

/* storage: the storage every admitted context must use; check_every: K, even,
 * the residual-check interval (and graph length); max_slots: resident contexts
 * at most; hbm_budget_bytes: device memory the batch's contexts may hold
 * together (0: no limit).  A context counts against the budget, with its
 * lbm_footprint_bytes, from its first admission until lbm_batch_release or
 * lbm_destroy, so finished contexts kept for a warm start keep counting.
 * Errors: LBM_ERR_ARG, LBM_ERR_UNSUPPORTED (FP64), LBM_ERR_OOM. */
lbm_status lbm_batch_create(lbm_batch** out, int storage, int check_every, int max_slots,
                            size_t hbm_budget_bytes);
void lbm_batch_destroy(lbm_batch* b);

/* Stop counting a context against the batch's budget (it must not be
 * running in the batch: LBM_ERR_ORDER; unknown contexts: LBM_ERR_ARG).
 * lbm_destroy of a counted context releases it. */
lbm_status lbm_batch_release(lbm_batch* b, lbm_ctx* ctx);

/* The budget and the bytes counted against it now. */
lbm_status lbm_batch_memory(lbm_batch* b, size_t* budget, size_t* held);

/* Queue a context (inputs set, D3Q19, the batch's storage) for a forward +
 * adjoint solve with opts->tol and opts->max_steps per phase (opts->check_every
 * is ignored: the batch's K applies; opts->reset = 0 warm-starts from the
 * context's previous populations).  The context must not be used by other
 * calls until it is returned by lbm_batch_poll.  *slot receives its slot id.
 * Errors: LBM_ERR_ARG (wrong storage/stencil, batch full), LBM_ERR_ORDER
 * (inputs missing), LBM_ERR_OOM (a context not yet counted does not fit the
 * budget now: nothing changes; admit it after releasing others). */
lbm_status lbm_batch_admit(lbm_batch* b, lbm_ctx* ctx, const lbm_solve_opts* opts, int* slot);

/* Advance every admitted context by K steps of its current phase and move
 * contexts whose phase converged (or hit its cap, or diverged) on; *n_active
 * receives the contexts still running.  Synchronises. */
lbm_status lbm_batch_step(lbm_batch* b, int* n_active);

/* Contexts admitted from now on whose lattice has at least min_tiles tiles
 * (256-node blocks of its single-lattice launch) run solo; the others are
 * packed into the persistent launch; 0 packs every lattice.  The default is
 * 1: every lattice solo (concurrent single-lattice graphs measured faster
 * than the packed launch for every mix tried).  Errors: LBM_ERR_ARG. */
lbm_status lbm_batch_set_solo_tiles(lbm_batch* b, long long min_tiles);

/* Contexts that finished since the last poll: up to max (slot, context,
 * report) triples; *n receives the count.  A finished context is released
 * from the batch; lbm_sensitivity / lbm_get_fields on it work as after
 * lbm_adjoint (report->status < 0: the solve failed, e.g. diverged). */
lbm_status lbm_batch_poll(lbm_batch* b, int* slots, lbm_ctx** ctxs, lbm_report* reports, int max,
                          int* n);

/* ---------------------------------------------------------------------------
 * Allocation-free single step (no counterpart in the paper).
 *
 * For callers that cannot allocate device memory: code running inside a
 * framework that owns every device allocation (a custom allocator or a memory
 * pool it must not bypass), or code that runs where cudaMalloc is forbidden.
 * The call runs one fused forward step with the residual / objective
 * reduction on caller-owned buffers and allocates nothing: its reduction
 * scratch is a static device array inside the library (512 KiB per GPU that
 * loads the library, held until the process exits).
 *
 * Populations are the offset populations h_i = f_i - w_i rho0, population-
 * major with `stride` elements between planes (stride >= nx*ny*nz); the rest
 * state is h = 0.  gamma, bc, rho and u are double for LBM_FP64 storage and
 * float otherwise; u has 3 planes of `stride`.  sums receives two doubles:
 * the sum of |u| over non-wall nodes and the sum of rho over VEL nodes, both
 * of the post-boundary state (the quantities the solver's residual and
 * objective use).  All pointers are device pointers.
 *
 * The lattice may need at most 32768 reduction blocks (about 8.3 million
 * nodes of 256-node tiles); larger lattices give LBM_ERR_ARG.  The first call
 * on a device looks up the scratch array's device address, so make that first
 * call before any stream capture.  The address is kept for the life of the
 * process: after cudaDeviceReset (or any teardown of the device's primary
 * context) the library's device code is loaded again and the kept address is
 * stale, so this entry point must not be used on that device again in the
 * same process.  Every call shares the one scratch array, so calls that
 * overlap on the GPU (different streams, no ordering) race.
 * --------------------------------------------------------------------------- */
typedef struct {
    int stencil;         /* lbm_stencil */
    int storage;         /* lbm_storage (D2Q9: FP64 or FP32) */
    int nx, ny, nz;
    long long stride;    /* elements between population planes, >= nx*ny*nz */
    const void* f_in;    /* Q planes, read */
    void* f_out;         /* Q planes, written (must not alias f_in) */
    const uint8_t* flags;
    const void* gamma;
    const void* bc;      /* 4 values per node, layout above */
    void* rho;           /* out, nx*ny*nz values */
    void* u;             /* out, 3 planes of stride */
    double* sums;        /* out, 2 doubles */
    double tau, rho0;
    int gamma_model;
} lbm_step_desc;

lbm_status lbm_flow_step_noalloc(const lbm_step_desc* d, void* cuda_stream);

/* Message for the last error on this thread (static storage, valid until the
 * next call on this thread). */
const char* lbm_last_error(void);

/* Library version string. */
/* Host-side check of the kernels' pull addressing (no counterpart in the
 * paper; a stand-in for a memory checker, which this GPU pool does not run).
 * Runs, on the CPU and without a GPU, the same neighbour-offset code the
 * kernels use for every node and every direction e_i, both ways (x - e_i for
 * the forward pull, x + e_i for the adjoint pull), and stores in *mismatches
 * how many computed sources differ from the periodic wrap of x -/+ e_i or fall
 * outside the lattice.  stencil: 0 D2Q9, 1 D3Q19, 2 D3Q7 (temperature).
 * Errors: LBM_ERR_ARG (null pointer, bad sizes, more than 2^24 nodes). */
lbm_status lbm_check_addressing(int stencil, int nx, int ny, int nz, long long* mismatches);

const char* lbm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LBMADJ_H */

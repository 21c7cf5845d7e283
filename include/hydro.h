/*
 * hydro.h -- C ABI of the GB300 (sm_103a) FP64 WENO5/WENO7 + RK3 solver for
 * 3+1D ideal relativistic hydrodynamics, after Sikorski et al.,
 * "Relativistic hydrodynamics on graphics processing units" (arXiv:1604.03360).
 *
 * The operation (paper, Sec. 1):
 *   Eq. 1   du/dt + sum_i d f_i(u)/dx_i = 0 with u = (E, M_x, M_y, M_z, R):
 *           energy density T^00, momentum densities T^0i and the conserved
 *           charge density n*gamma of an ideal fluid with p = cs2 * e.
 *   Eq. 2   L(u) = sum_i (F_i(x - e_i/2) - F_i(x + e_i/2)) / |e_i| on a
 *           Cartesian grid; F at the half-cell faces from finite-difference
 *           WENO of order 5 or 7 (Sec. 1.2) on Lax-Friedrichs split fluxes.
 *   Sec. 1  third-order Runge-Kutta in time (SSP / Shu-Osher form).
 * Readings where the paper is silent (each switchable in hydro_config: local
 * Lax-Friedrichs, characteristic-wise WENO, several charges, the general EOS
 * p = cs2 (e - eos_mass n_1)): component-wise WENO on f^+- =
 * (f +- alpha_d u)/2 with alpha_d the largest characteristic speed over the
 * grid (recomputed from every stage's input); epsilon = weno_eps in
 * omega_k ~ d_k / (eps + beta_k)^2; dt = cfl * min_d dx_d / max_d alpha_d over
 * directions with more than one cell, clipped so that t lands on t_end;
 * outflow = copy of the edge cell into the ghost cells; periodic = wrap;
 * directions with one cell contribute no flux difference.
 *
 * Conventions for every entry point:
 *   - Fields are FP64 structure-of-arrays: field f (0..4, or 0..3+nq with
 *     several charges) of a state starts at
 *     ptr + f * field_stride and holds nz*ny*nx values, x fastest.
 *     field_stride >= nx*ny*nz (elements, not bytes).
 *   - mem = HYDRO_MEM_HOST: ptr is host memory (pageable or pinned);
 *     mem = HYDRO_MEM_DEVICE: ptr is device memory on the handle's device.
 *     The caller keeps ownership of every pointer it passes.
 *   - All work is ordered on the CUDA stream given at creation (NULL = the
 *     legacy default stream).  Calls that return data to the host synchronise
 *     that stream; all others are asynchronous.
 *   - Every call returns a hydro_status; no C++ exception crosses the ABI and
 *     no kernel traps.  Device-side problems (an unphysical state such as
 *     E <= 0 or |M| >= E, or a NaN) are recorded on the device and reported
 *     by the next synchronising call (hydro_get_state, hydro_sync), which
 *     then returns HYDRO_ERR_UNPHYSICAL.  Every wait inside a kernel is
 *     bounded (the TMA-staged launch variants wait for their tile loads);
 *     one that runs out of time (about a second) is reported the same way
 *     as HYDRO_ERR_TIMEOUT, and that step's results are invalid.
 *     hydro_last_error() describes the most recent failure of a handle.
 *   - A handle is not thread-safe: one host thread at a time.
 */
#ifndef HYDRO_H
#define HYDRO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HYDRO_OK = 0,
    HYDRO_ERR_INVALID_ARG = 1,
    HYDRO_ERR_CUDA = 2,
    HYDRO_ERR_OOM = 3,
    HYDRO_ERR_UNPHYSICAL = 4,
    HYDRO_ERR_TIMEOUT = 5,
    HYDRO_ERR_STATE = 6
} hydro_status;

/* WENO5 / WENO7: finite-difference WENO of Sec. 1.2 (the hot path).
 * MUSTA_FORCE: the second-order scheme of Sec. 1.1 -- MUSCL linear
 * reconstruction with a slope limiter and the multi-stage (MUSTA) centred
 * FORCE flux; see hydro_config.limiter / musta_stages. */
typedef enum { HYDRO_MUSTA_FORCE = 2, HYDRO_WENO5 = 5, HYDRO_WENO7 = 7 } hydro_scheme;
/* HYDRO_BC_HALO (z only): the grid is one z-slab of a larger grid.  The
 * handle stores G = r planes (WENO5 3, WENO7 4, MUSTA-FORCE 2) of ghost cells
 * below and above its nz interior planes, and its stage kernels read them as
 * they are; the caller fills them before every RK stage (hydro_halo_*) and
 * drives the step one stage at a time (hydro_stage).  See the slab-domain
 * entry points below. */
typedef enum { HYDRO_BC_OUTFLOW = 0, HYDRO_BC_PERIODIC = 1, HYDRO_BC_HALO = 2 } hydro_bc;
typedef enum { HYDRO_MEM_HOST = 0, HYDRO_MEM_DEVICE = 1 } hydro_mem;

/* Problem definition (Eq. 2 grid, Sec. 1.2 scheme, boundary rule). */
typedef struct {
    int32_t n[3];       /* interior cells nx, ny, nz (>= 1; a direction with
                           n = 1 is inactive; a periodic active direction
                           needs n >= 4 for WENO7, >= 3 for WENO5) */
    int32_t scheme;     /* HYDRO_WENO5, HYDRO_WENO7 or HYDRO_MUSTA_FORCE */
    int32_t bc[3];      /* hydro_bc per direction */
    int32_t split;      /* flux splitting: 0 = global Lax-Friedrichs (alpha_d
                           = max speed over the grid), 1 = local Lax-Friedrichs
                           (each face j+1/2 uses the max speed over the 2r
                           cells of its two stencils); dt uses the global
                           speeds either way.  Local LF is not supported by
                           hydro_forward_record/hydro_adjoint or
                           hydro_step_noalloc (HYDRO_ERR_INVALID_ARG) */
    int32_t nq;         /* conserved charge densities: 0 or 1 = one (R), up to
                           3 (R_1, R_2, R_3; Sec. 1 names charge densities in the plural).
                           Each is passive (p = cs2 e) and advected like R; a
                           state then has 4 + nq fields (E, M_x, M_y, M_z,
                           R_1..R_nq) and primitives (e, v, n_1..n_nq).  nq > 1
                           is supported by the single-grid path only */
    int32_t limiter;    /* MUSTA-FORCE: MUSCL slope limiter on the conserved
                           variables, component-wise: 0 minmod, 1 monotonized
                           central, 2 van Leer, 3 superbee.  A reconstructed
                           state with E <= 0 or |M| >= E falls back to the
                           cell value.  Ignored by WENO */
    int32_t musta_stages; /* MUSTA-FORCE: stages K of the centred FORCE flux on
                           the local states (0 = default 2; 1 = plain FORCE),
                           local ratio dt/dx = 0.9 / max|lambda| of the local
                           states.  Ignored by WENO.  MUSTA-FORCE runs on the
                           single-grid path with split = 0, nq <= 1 */
    int32_t charwise;   /* WENO reconstruction: 0 = component-wise (on each
                           field of the split fluxes), 1 = characteristic-wise:
                           at each face the split fluxes are projected on the
                           characteristic fields of df_d/du at the mean of the
                           two neighbouring states, reconstructed there and
                           mapped back (Sec. 1.2 leaves this choice open).
                           1 needs WENO with split = 0; it runs on the
                           single-grid and z-slab paths, not the adjoint, the
                           batch or hydro_step_noalloc */
    double dx[3];       /* cell sizes |e_i| > 0 */
    double origin[3];   /* lower corner of the box (informational) */
    double cs2;         /* EOS p = cs2 * e, 0 < cs2 < 1 (1/3 in the paper's tests) */
    double cfl;         /* dt = cfl * min dx / max alpha when dt_fixed <= 0 */
    double dt_fixed;    /* > 0: constant time step */
    double weno_eps;    /* WENO epsilon, 1e-40 <= weno_eps <= 1e30 (1e-6).
                           Range of the data: split-flux differences up to
                           about 1e24 (WENO7) or 1e37 (WENO5) in magnitude;
                           beyond that the products of the smoothness terms
                           overflow and the result is NaN, reported as
                           HYDRO_ERR_UNPHYSICAL */
    double eos_mass;    /* equation of state p = cs2 (e - eos_mass n_1): 0 (the
                           default) is p = cs2 e; > 0 is the ideal gas of
                           adiabatic index 1 + cs2 whose rest mass is eos_mass
                           per unit of the first charge (Sec. 1 leaves the EOS
                           open).  The first charge then enters the pressure, the
                           primitive recovery iterates (bracketed Newton on p)
                           and states with e <= eos_mass n_1 are unphysical.
                           > 0 needs component-wise WENO (either splitting) and
                           runs on the single-grid and z-slab paths only */
} hydro_config;

typedef struct hydro_s hydro_t;

/* Create a solver for one grid.  The library allocates and owns all device
 * buffers (three conserved states, three primitive scratch states and a small
 * control block, about 27 doubles per cell).  stream: a cudaStream_t (may be
 * NULL).  Errors: INVALID_ARG for a bad config or NULL out, OOM, CUDA. */
hydro_status hydro_create(const hydro_config* cfg, void* stream, hydro_t** out);

/* Release every resource of h (NULL is a no-op). */
hydro_status hydro_destroy(hydro_t* h);

/* Load the conserved state u = (E, M_x, M_y, M_z, R) (Eq. 1) at time t and
 * reset the step counter.  Also recovers the primitives and the characteristic
 * speeds of the new state on the device.  Asynchronous. */
hydro_status hydro_set_state(hydro_t* h, const double* u, int64_t field_stride, int32_t mem, double t);

/* Load primitives (e, v_x, v_y, v_z, n) and convert them to the conserved
 * state on the device: E = (e+p) g^2 - p, M = (e+p) g^2 v, R = n g, with
 * g^2 = 1/(1 - v^2), p = cs2 e.  Requires |v| < 1, e > 0. */
hydro_status hydro_set_primitive(hydro_t* h, const double* w, int64_t field_stride, int32_t mem, double t);

/* Advance by up to nsteps RK3 steps (Sec. 1).  If t_end >= 0 the last step is
 * shortened so that t lands on t_end and later steps do nothing.  Each step is
 * one replay of a captured CUDA graph: a 1-thread step-begin kernel (dt from
 * the current characteristic speeds), then per RK3 stage either one fused
 * stage kernel (Eq. 2 + RK combine + speeds of the new state), or in the
 * z-pass launch variants a z-face pass followed by the stage kernel, or in
 * the three-pass variants (the default for WENO with global or local
 * Lax-Friedrichs, any number of charges, component- or characteristic-wise)
 * an x-, a y- and a z-face pass followed by a per-cell combination kernel,
 * and a 1-thread step-end kernel (hydro_kernels_per_step counts them).
 * Asynchronous; no host synchronisation. */
hydro_status hydro_step(hydro_t* h, int32_t nsteps, double t_end);

/* Copy the current conserved state out (synchronises the stream).  t and
 * step (either may be NULL) receive the simulation time and the number of
 * steps taken since the last set_state.  Returns HYDRO_ERR_UNPHYSICAL if a
 * kernel met an unphysical state since the last set_state (the state is still
 * copied). */
hydro_status hydro_get_state(hydro_t* h, double* u, int64_t field_stride, int32_t mem, double* t, int64_t* step);

/* Copy the primitives (e, v_x, v_y, v_z, n) of the current state out
 * (synchronises the stream). */
hydro_status hydro_get_primitive(hydro_t* h, double* w, int64_t field_stride, int32_t mem);

/* Synchronise the stream and report deferred device errors. */
hydro_status hydro_sync(hydro_t* h);

/* Event-by-event stream on one grid (the many independent initial conditions
 * that motivate the paper's GPU code, Sec. 1): for each of n_items initial
 * states u_in[i] (conserved fields in host memory, layout as hydro_set_state
 * with mem = HYDRO_MEM_HOST), load it at time t0, advance nsteps RK3 steps
 * (t_end as in hydro_step) and write the final state to u_out[i] (host
 * memory, same layout).  Each item's result is bit for bit what
 * hydro_set_state + hydro_step + hydro_get_state give.  The copies are
 * double-buffered: item i+1 is copied in and item i-1 out on two copy
 * streams of the handle while item i steps on the handle's stream, with
 * device-to-device moves between the staging buffers and the state.  The
 * first call allocates the staging buffers (three states) and the copy
 * streams; they live until hydro_destroy.  Host buffers should be page-locked
 * (cudaMallocHost or pinned torch tensors): pageable ones work, but their
 * copies do not overlap.  u_in[i] and u_out[j] may be the same buffer only
 * if j >= i + 2 never reuses it before item i's copy-in ends (simplest:
 * distinct buffers, or the same input buffer for every item).  Synchronises
 * before returning; returns the first error of any item
 * (HYDRO_ERR_UNPHYSICAL names the item and the cell in hydro_last_error).
 * Afterwards the handle holds the last item's final state.  Whole grids only
 * (not z-slab handles). */
hydro_status hydro_run_many(hydro_t* h, int32_t n_items, const double* const* u_in, double* const* u_out,
                            int64_t field_stride, int32_t nsteps, double t0, double t_end);

/* Largest characteristic speed per direction of the current state (alpha_d
 * of the global Lax-Friedrichs splitting) and the last time step taken.
 * Synchronises. */
hydro_status hydro_get_speeds(hydro_t* h, double alpha[3], double* last_dt);

/* Text of the last error of h (never NULL; "" if none).  Valid until the next
 * call on h.  hydro_last_error(NULL) describes the last failed hydro_create. */
const char* hydro_last_error(hydro_t* h);

/* Advance like hydro_step, but launch the five kernels of every step directly
 * (no graph) with CUDA events between them on the handle's stream, and
 * return in kernel_ms[5] the summed device time of: step-begin, stage 1,
 * stage 2, stage 3, step-end.  Synchronises once per step.  For measurement
 * only; the numerical result equals hydro_step's bit for bit. */
hydro_status hydro_profile_step(hydro_t* h, int32_t nsteps, double t_end, double kernel_ms[5]);

/* Launch configuration of the stage kernel.  Several CTA tile shapes and
 * face orders are compiled per scheme (a new handle starts on the fastest for
 * the 256^3 workload); the z-chunk (planes per CTA) sets how many CTAs share a
 * column.  Some variants compute the z-face fluxes in a separate z pass that
 * runs before each stage kernel; some of those stage the raw cells of each
 * z plane in shared memory with tensor-map (TMA) tile loads, which needs an
 * even nx (rows of a multiple of 16 bytes).  hydro_set_launch forces a variant
 * (0 <= variant < hydro_launch_variants(scheme, split, nq)) and z-chunk (zc <= 0: the
 * built-in wave-count heuristic), rebuilding the step graph; a TMA-staged
 * variant is refused (HYDRO_ERR_INVALID_ARG) for an odd nx (the autotuner
 * skips it there).  Results do
 * not depend on the choice beyond FMA-level rounding of the same formulas. */
int32_t hydro_launch_variants(int32_t scheme, int32_t split, int32_t nq);
/* The same count for a full configuration (characteristic-wise WENO has its
 * own tile shapes); 0 for an invalid configuration. */
int32_t hydro_launch_variants_cfg(const hydro_config* cfg);
hydro_status hydro_set_launch(hydro_t* h, int32_t variant, int32_t zc);
hydro_status hydro_get_launch(hydro_t* h, int32_t* variant, int32_t* tile_x, int32_t* tile_y, int32_t* zc);
/* Kernels one hydro_step step launches with the current launch configuration
 * (step-begin, per RK3 stage the z pass if any and the stage kernel,
 * step-end); 0 for a NULL handle.  No GPU work. */
int32_t hydro_kernels_per_step(hydro_t* h);

/* Autotuner: with a state loaded, time one stage launch for every compiled
 * tile shape and a few z-chunks around the heuristic choice on this grid, keep
 * the fastest and rebuild the step graph (synchronises; the loaded state is
 * left unchanged).  If the environment variable HYDRO_TUNE_CACHE names a file,
 * the choice is looked up there first (key: scheme and grid size) and stored
 * there after tuning.  best_ms (may be NULL) receives the chosen stage time. */
hydro_status hydro_autotune(hydro_t* h, double* best_ms);

/* Device pointer of the current conserved state (5 fields, stride
 * hydro_field_stride()) for zero-copy readers; owned by h. */
const double* hydro_state_device_ptr(hydro_t* h);
int64_t hydro_field_stride(hydro_t* h);

/* ---- z-slab domain decomposition ----------------------------------------
 * L(u) of Eq. 2 at a cell depends on the r (= G) neighbouring cells along
 * each axis (Sec. 1, after Eq. 2), and the global Lax-Friedrichs speeds of
 * Sec. 1.2 are maxima over the whole grid.  A grid split into z-slabs, each
 * a handle with bc[2] = HYDRO_BC_HALO holding nz >= G interior planes,
 * therefore advances exactly like the whole grid if, before each RK stage,
 * every slab's G ghost planes on each side hold the neighbouring slab's
 * planes of that stage's input (or the boundary rule's values at the ends of
 * the grid), and every speed slot is the maximum over all slabs.  A step is
 *     hydro_stage(h, 0, t_end)            dt from speed slot 0 (must already
 *                                         be the global max), clear slots 1-3
 *     for s in 1, 2, 3:
 *         fill ghost planes of level s-1  (hydro_halo_pack / _unpack /
 *                                          _fill_outflow)
 *         hydro_stage(h, s, t_end)        RK stage s; local max speeds of its
 *                                         output into slot s
 *         max-reduce slot s over slabs    (hydro_speed_slot read, reduce, write)
 *     hydro_stage(h, 4, t_end)            commit: slot 3 becomes slot 0, t += dt
 * After hydro_set_state/_set_primitive slot 0 holds the slab's own speeds
 * and must be max-reduced before the first step.  Levels: 0 = u^n (also the
 * stage-3 output), 1 and 2 = the stage-1 and stage-2 outputs.  Every call is
 * stream-ordered on the handle's stream and returns without synchronising
 * unless a host buffer is involved.  hydro_step/_profile_step, the adjoint
 * and hydro_autotune reject halo handles. */

/* Doubles in one side's ghost block: (nf + 4 [+ 3 with local LF]) fields x
 * G planes x nx x ny, laid out field by field, each field's planes in
 * ascending z (the layout of hydro_halo_pack's output). */
int64_t hydro_halo_doubles(hydro_t* h);
/* Copy the G interior planes next to `side` (0 = low z, 1 = high z) of every
 * field of `level` into buf (hydro_halo_doubles() doubles, host or device per
 * mem, owned by the caller; a host copy synchronises the stream). */
hydro_status hydro_halo_pack(hydro_t* h, int32_t level, int32_t side, double* buf, int32_t mem);
/* Copy buf (layout of hydro_halo_pack) into the G ghost planes on `side` of
 * `level`: the low ghost planes take the lower neighbour's high pack, the
 * high ghost planes the upper neighbour's low pack. */
hydro_status hydro_halo_unpack(hydro_t* h, int32_t level, int32_t side, const double* buf, int32_t mem);
/* Outflow boundary at the end of the grid: every ghost plane on `side` of
 * `level` becomes a copy of the nearest interior plane (the zero-gradient
 * rule of the whole-grid kernels). */
hydro_status hydro_halo_fill_outflow(hydro_t* h, int32_t level, int32_t side);
/* One part of a step on a halo handle: which = 0 step begin (dt, clipped to
 * t_end when t_end >= 0), 1..3 RK stage, 4 step commit.  Any other value or
 * a handle without HYDRO_BC_HALO -> HYDRO_ERR_INVALID_ARG. */
hydro_status hydro_stage(hydro_t* h, int32_t which, double t_end);
/* Read (io = 0) or write (io = 1) speed slot `slot` (0 = speeds of u^n,
 * 1..3 = of the stage-s output): 3 non-negative doubles (max |lambda| along
 * x, y, z), host or device per mem.  A host read synchronises the stream. */
hydro_status hydro_speed_slot(hydro_t* h, int32_t slot, int32_t io, double* speeds, int32_t mem);

/* Measurement helper, not part of the paper's method: times a kernel of
 * independent FP64 FMA chains on every SM (on `stream`, synchronising it) and
 * returns the FP64 FMA issue rate in FMA/s -- the roofline denominator of the
 * FP64-bound stage kernel.  Allocates and frees a small scratch buffer. */
hydro_status hydro_measure_fp64_peak(void* stream, double* fma_per_second);

/* Self-check helper, not part of the paper's method: y[i] = the kernels'
 * reciprocal of x[i] for i < n (x, y device pointers owned by the caller,
 * n >= 0; asynchronous on `stream`).  The kernels divide by taking a MUFU
 * seed and one cubically convergent Newton correction instead of IEEE
 * division; this entry point lets a test bound that reciprocal's error
 * against 1/x.  Valid for 2^-1022 <= |x| <= 2^1022 (the seed flushes
 * subnormal inputs and results to zero).  INVALID_ARG for n < 0 or a NULL
 * pointer with n > 0; CUDA if the launch fails. */
hydro_status hydro_eval_rcp(const double* x, double* y, int64_t n, void* stream);

/* ---- Reverse mode (adjoint) --------------------------------------------
 * Gradients of a final-state observable with respect to the initial state.
 * The Lax-Friedrichs speeds and time steps are frozen at their forward values
 * (they are maxima over the grid and not differentiable); the WENO weights
 * (epsilon > 0) are smooth, so every other ingredient is differentiated
 * exactly.  The paper's scheme (Sec. 1, Eq. 2, Sec. 1.2) is the function
 * being differentiated; the adjoint itself is not in the paper.
 *
 * hydro_forward_record: advance the current state by nsteps RK3 steps (no
 *   t_end), recording each step's speeds and dt and checkpointing the state
 *   every ckpt_every steps (device workspace owned by h, about
 *   99 + 5 * ceil(nsteps/ckpt_every) + 27 * ckpt_every doubles per cell:
 *   the reverse sweep keeps every stage input of one segment; allocated on
 *   the first call and kept by later calls with the same nsteps and
 *   ckpt_every, so only a call that changes them allocates).
 *   Asynchronous.
 * hydro_adjoint: grad_u0 = (d u_N / d u_0)^T lambda_final for the recorded
 *   run: segment by segment, the step-start states are recomputed from the
 *   checkpoint with frozen stages, then each step's three stage adjoints run
 *   in reverse.  lambda_final and grad_u0: 5 fields with field_stride, in
 *   `mem`.  Synchronises.  HYDRO_ERR_STATE if nothing was recorded.  The
 *   environment variable HYDRO_ADJ_PENCIL=<0..5>, read at each call, selects
 *   a variant of the reverse-WENO pencil kernel (integer-pipe products, CTAs
 *   per SM) for timing; all give the same bits, and other values select the
 *   default.
 * hydro_recorded_steps: number of recorded steps and (either may be NULL)
 *   the speeds alpha[n][stage][axis] (9 per step) and dt[n].  Synchronises.
 * hydro_eps2: momentum anisotropy eps_2 = sum(T^xx - T^yy) / sum(T^xx + T^yy)
 *   of state u (NULL: the current state) and, if grad != NULL, its gradient
 *   with respect to the conserved fields (5 fields, R component zero).
 *   Synchronises. */
hydro_status hydro_forward_record(hydro_t* h, int32_t nsteps, int32_t ckpt_every);
hydro_status hydro_adjoint(hydro_t* h, const double* lambda_final, double* grad_u0, int64_t field_stride, int32_t mem);
hydro_status hydro_recorded_steps(hydro_t* h, int32_t* nsteps, double* alpha, double* dt);
hydro_status hydro_eps2(hydro_t* h, const double* u, int64_t field_stride, int32_t mem, double* eps2, double* grad,
                        int64_t grad_stride, int32_t grad_mem);

/* ---- Event-by-event ensembles ------------------------------------------
 * Many independent grids ("events", possibly of different sizes and cell
 * spacings, one scheme for all) advanced together; the paper motivates GPU
 * hydro with event-by-event studies (Sec. 1).  Each RK3 stage of ALL events is
 * one persistent launch of sms x (CTAs per SM) CTAs that pop (event, tile,
 * z chunk) items from a precomputed work-list with one atomicAdd each and run
 * the same per-item stage code as hydro_step, so every event's result equals
 * its single-grid result.  Each event keeps its own speeds, dt and time; a
 * step is one replay of a captured CUDA graph.  Events are indexed 0..n-1 in
 * the order of cfgs.  Semantics of set/get/step/sync as for a single grid
 * (t_end is not supported: steps are always taken). */
typedef struct hydro_batch_s hydro_batch_t;
hydro_status hydro_batch_create(const hydro_config* cfgs, int32_t n_events, void* stream, hydro_batch_t** out);
hydro_status hydro_batch_destroy(hydro_batch_t* b);
hydro_status hydro_batch_set_state(hydro_batch_t* b, int32_t event, const double* u, int64_t field_stride, int32_t mem,
                                   double t);
hydro_status hydro_batch_set_primitive(hydro_batch_t* b, int32_t event, const double* w, int64_t field_stride,
                                       int32_t mem, double t);
hydro_status hydro_batch_step(hydro_batch_t* b, int32_t nsteps);
hydro_status hydro_batch_get_state(hydro_batch_t* b, int32_t event, double* u, int64_t field_stride, int32_t mem,
                                   double* t, int64_t* step);
hydro_status hydro_batch_sync(hydro_batch_t* b);
int32_t hydro_batch_size(hydro_batch_t* b);
const char* hydro_batch_last_error(hydro_batch_t* b);
/* As hydro_profile_step, for the whole batch (kernel_ms: step-begin, the three
 * persistent stages, step-end). */
hydro_status hydro_batch_profile_step(hydro_batch_t* b, int32_t nsteps, double kernel_ms[5]);
/* Tile shape / z chunk of the persistent kernel (variants as for a single
 * grid); n_items is the work-list length.  hydro_batch_autotune times a
 * stage-1 launch per candidate (states, speeds and times are unchanged) and
 * keeps the fastest. */
hydro_status hydro_batch_set_launch(hydro_batch_t* b, int32_t variant, int32_t zc);
/* Kernels one hydro_batch_step step launches (as hydro_kernels_per_step, for
 * the whole batch); 0 for a NULL handle.  No GPU work. */
int32_t hydro_batch_kernels_per_step(hydro_batch_t* b);
hydro_status hydro_batch_get_launch(hydro_batch_t* b, int32_t* variant, int32_t* tile_x, int32_t* tile_y, int32_t* zc,
                                    int32_t* n_items);
hydro_status hydro_batch_autotune(hydro_batch_t* b, double* best_ms);

/* ---- Stepping without device allocation -------------------------------
 * The paper has no counterpart of this entry point; it exists for callers
 * that cannot call cudaMalloc -- for example a host application whose device
 * memory belongs to its own pool allocator, or a loop with a fixed footprint
 * that must not pay cudaMalloc's implicit synchronisation.  It advances the
 * conserved state by up to nsteps RK3 steps exactly like hydro_step (the same
 * scheme and the same result bit for bit, computed by the fused stage kernel,
 * which needs no z-face buffer), but keeps all intermediate data in one static
 * device array of the library (HYDRO_NOALLOC_MAX_CELLS * 176 bytes + 256
 * bytes, about 23 MB) that every GPU which loads the library holds until the
 * process exits.  It calls no cudaMalloc, cudaFree or allocating library
 * routine.
 *   cfg          grid and scheme, as for hydro_create.
 *   u_in, u_out  device pointers: 5 fields (E, M_x, M_y, M_z, R) with stride
 *                field_stride; u_out receives the result (u_out == u_in is
 *                allowed: the update is then in place).  Owned by the caller.
 *   field_stride cell count <= field_stride <= HYDRO_NOALLOC_MAX_CELLS, else
 *                HYDRO_ERR_INVALID_ARG with a message saying so.
 *   t0, t_end    start time; t_end < 0 for no limit (as in hydro_step).
 *   stream       cudaStream_t for all work (NULL: legacy default stream).
 *   t_out        NULL: fully asynchronous, device errors are not reported.
 *                Non-NULL: the call synchronises the stream, stores the final
 *                time and returns HYDRO_ERR_UNPHYSICAL if a stage met an
 *                unphysical state.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) and configures the kernels, with that device
 * current; make that first call before any stream capture.  All calls share
 * the array and it keeps the previous call's contents (each call resets what
 * it reads): calls whose GPU work overlaps race on it and must be serialised.
 * hydro_noalloc_last_error() describes the calling thread's last failure. */
#define HYDRO_NOALLOC_MAX_CELLS 131072
hydro_status hydro_step_noalloc(const hydro_config* cfg, const double* u_in, double* u_out, int64_t field_stride,
                                double t0, int32_t nsteps, double t_end, void* stream, double* t_out);
const char* hydro_noalloc_last_error(void);

/* Library version string. */
const char* hydro_version(void);

#ifdef __cplusplus
}
#endif
#endif /* HYDRO_H */

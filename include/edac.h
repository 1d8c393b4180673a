/*
 * edac.h -- C ABI of the GB300 (sm_103a) EDAC weakly-compressible SPH library
 * with an inlet and the hybrid non-reflecting outlet of Negi, Ramachandran &
 * Haftu, arXiv 1907.04034.
 *
 * One context = one 2D particle system on one GPU.  A time step is the paper's
 * per-step particle pass: cell-list neighbour search, summation density
 * (Eq. summation-density) with the quintic spline (Eq. quintic-spline), solid
 * wall projection (Sec. 2), mirrored inlet pressure (Sec. 3.2, Eqs. matform and
 * taylor2), the EDAC-TVF momentum and pressure rates (Eqs. tvf-momentum, pavg,
 * tvf-p-ij-basa, p-edac, transport-vel), a midpoint predictor-corrector
 * integrator, the hybrid outlet (Sec. 3.4, Eqs. timeevg, acouinten, acou with the
 * characteristic variables of Eq. characteristic-vars), particle recycling (end
 * of Sec. 3.4) and the solid force (Eq. tvf-momentum_solid).
 *
 * Conventions
 *   - Every function returns an edac_status; nothing throws across the ABI.
 *   - Host pointers ("h_") are caller-owned and only read or written during the
 *     call; device pointers ("d_") are caller-owned device memory.
 *   - The library never allocates device memory: the caller supplies one
 *     device workspace of edac_workspace_bytes() bytes (256-byte aligned) that
 *     the context owns the layout of until edac_destroy().
 *   - All GPU work is issued on params.cuda_stream (a cudaStream_t; NULL means
 *     the legacy default stream, which disables CUDA-graph replay).
 *   - Device-side faults (capacity overflow, non-finite values, particles that
 *     left the domain box, event-list overflow) set a sticky device error word.
 *     It is read at every edac_get_* / edac_read_* call; once set, the call
 *     returns the matching code and edac_step() returns EDAC_E_STATE until the
 *     context is re-initialised with edac_set_particles().
 *   - Not thread-safe per context; distinct contexts are independent.
 */
#ifndef EDAC_H
#define EDAC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct edac_ctx edac_ctx;

typedef enum {
    EDAC_OK = 0,
    EDAC_E_INVALID = 1,   /* bad argument or parameter (host-side check)        */
    EDAC_E_CAPACITY = 2,  /* particle capacity or an event list exceeded       */
    EDAC_E_CUDA = 3,      /* a CUDA runtime call failed; see edac_last_error() */
    EDAC_E_NONFINITE = 4, /* a NaN/Inf appeared in the integrated fields       */
    EDAC_E_TIMEOUT = 5,   /* a bounded device wait gave up                     */
    EDAC_E_STATE = 6,     /* call out of order, or the context is in error     */
    EDAC_E_DOMAIN = 7     /* a particle left the domain box of the cell grid   */
} edac_status;

/* arithmetic of the pair sums */
enum { EDAC_FP64 = 0, EDAC_MIXED = 1 };

/* particle tags (uint8) */
enum { EDAC_FLUID = 0, EDAC_INLET = 1, EDAC_OUTLET = 2, EDAC_WALL = 3, EDAC_SLIPWALL = 4 };

/* field ids for edac_read_state() (all returned as fp64) */
enum {
    EDAC_F_X = 0, EDAC_F_Y, EDAC_F_U, EDAC_F_V, EDAC_F_UT, EDAC_F_VT, EDAC_F_P, EDAC_F_M,
    EDAC_F_RHO, EDAC_F_VOL, EDAC_F_AU, EDAC_F_AV, EDAC_F_AP, EDAC_F_ABU, EDAC_F_ABV,
    EDAC_F_FX, EDAC_F_FY, EDAC_F_NNB, EDAC_F_UBAR, EDAC_F_VBAR, EDAC_F_PBAR, EDAC_F_J2,
    EDAC_F_J2P, EDAC_F_ADVP, EDAC_F_REDP, EDAC_F_RPOS, EDAC_NUM_FIELDS
};

/* kernels that edac_profile() can time with CUDA events */
enum { EDAC_K_PASS_A = 0, EDAC_K_PASS_B = 1, EDAC_K_REBUILD = 2, EDAC_K_BOUNDARY = 3,
       EDAC_K_STAGE = 4, EDAC_K_RECYCLE = 5, EDAC_NUM_KERNELS = 6 };

/*
 * Run parameters, SI units.  h = hdx * dx, support radius r_c = 3h.
 * The cell grid covers the box [x_min, x_max) x [y_min, y_max) with cells of
 * at least r_c; a periodic axis needs at least 3 cells.  Particles must stay
 * inside the box (EDAC_E_DOMAIN otherwise).
 */
typedef struct {
    double x_min, x_max, y_min, y_max;
    int periodic_x, periodic_y;
    double dx;       /* initial particle spacing                                  */
    double hdx;      /* h / dx (1.2 in the paper)                                 */
    double rho0;     /* reference density                                          */
    double U;        /* inlet / reference speed                                    */
    double nu;       /* kinematic viscosity                                        */
    double cs;       /* artificial speed of sound c_s (10 u_max, Sec. 2)           */
    double alpha;    /* EDAC damping coefficient of Eq. edac-nu (0.5)             */
    double pb;       /* background pressure of Eq. transport-vel                   */
    double eta_reg;  /* regulariser eta of Eqs. tvf-momentum / p-edac (0.01)       */
    double gx, gy;   /* body force                                                  */
    double dt;       /* time step (> 0)                                             */
    int use_pavg;    /* 1: subtract p_avg (Eq. pavg); 0: plain p_ij average        */
    int precision;   /* EDAC_FP64 or EDAC_MIXED                                     */
    int capacity;    /* maximum live particles, recycling headroom included         */
    int max_history; /* per-step history records kept on the device (ring)          */
    int use_graphs;  /* 1: capture one step in a CUDA graph and replay it          */
    void *cuda_stream;
} edac_params;

/* Bytes of device workspace a context with these parameters needs. */
edac_status edac_workspace_bytes(const edac_params *params, size_t *bytes);

/* Create a context on the current CUDA device.  d_workspace: caller-owned
 * device memory of at least edac_workspace_bytes() bytes, 256-byte aligned,
 * kept alive until edac_destroy().  No GPU work is issued. */
edac_status edac_create(const edac_params *params, void *d_workspace, size_t bytes,
                        edac_ctx **out);

/* Inlet zone (Sec. 3): inlet particles sit in [x_in - n_layers dx, x_in) and move
 * with u(y) = U + sum_{k=1..n_modes} a_k sin(k pi (y - y0) / H), v = 0; their
 * pressure is mirrored from the fluid (Sec. 3.2).  n_modes <= 16.  Call before
 * edac_set_particles(). */
edac_status edac_set_inlet(edac_ctx *ctx, double x_in, int n_layers, int n_modes,
                           const double *h_modes, double y0, double H);

/* Inlet velocity in time (the outlet test problems of Sec. 4; default: the steady
 * modes of edac_set_inlet).  With t the time of the state (steps done x dt; an
 * inlet particle takes the value at the end of each integrator stage, a new one
 * the value at the end of the step), y0 and H those of edac_set_inlet:
 *   EDAC_INLET_MODES  (nprm 0): the steady u(y) of edac_set_inlet, v = 0;
 *   EDAC_INLET_PULSE  (nprm 4, prm = A, t0, t1, delta; Eq. velfunc2, read with a
 *     decaying exponent): u = U + A cos(pi (y - y0)/12) exp(-(t - t0)^2/delta)
 *     for t0 < t < t1, else U; v = 0;
 *   EDAC_INLET_RAMP   (nprm 1, prm = T; Sec. 4.3): u = U min(t/T, 1), v = 0;
 *   EDAC_INLET_VORTEX (nprm 4, prm = G, c, d0, y_c; Eqs. vortex, vortexx): a
 *     vortex whose centre starts d0 upstream and moves at U: x_r = U (d0 - t),
 *     y_r = y - y_c, u = U + G y_r/(x_r^2 + y_r^2 + c), v = -G x_r/(...).
 * Inlet particles move in x only, with u.  EDAC_E_INVALID for a bad kind,
 * parameter count or range (delta, T, c > 0, t1 > t0).  Drops the step graph. */
#define EDAC_INLET_MODES 0
#define EDAC_INLET_PULSE 1
#define EDAC_INLET_RAMP 2
#define EDAC_INLET_VORTEX 3
edac_status edac_set_inlet_transient(edac_ctx *ctx, int kind, int nprm, const double *prm);

/* Outlet zone: outlet particles sit in [x_out, x_out + n_layers dx) and move in x
 * only; a fluid particle past x_out becomes an outlet particle, one past
 * x_out + n_layers dx is deleted.  kind selects the treatment of Sec. 3:
 *   EDAC_OUTLET_HYBRID (Sec. 3.4): frozen time averages plus the acoustic part
 *     carried by J2 with J3 = 0; n_avg is the length of the time average
 *     (Eq. timeevg; 6 in the paper, at most 8) and i_thresh < 0 selects
 *     I = (rho0 U^2/2)^2/(2 rho0 c_s) of Eq. acouinten;
 *   EDAC_OUTLET_DONOTHING (Sec. 3.1): u, v, p frozen at the crossing, advected
 *     with that u;
 *   EDAC_OUTLET_MOD_DONOTHING (Sec. 3.1.1): values frozen, advected with the
 *     Shepard velocity of the fluid (Eq. shepard0);
 *   EDAC_OUTLET_CHARACTERISTIC (Sec. 3.3): p = J2/2, u = U + J2/(2 rho0 c_s)
 *     from the fluid's J2 against the free stream, v frozen;
 *   EDAC_OUTLET_MIRROR (Sec. 3.2): p, u, v by the mirrored Taylor extrapolation
 *     (Eqs. matform, taylor2) about (2 x_out - x, y).
 * Call before edac_set_particles(). */
#define EDAC_OUTLET_HYBRID 0
#define EDAC_OUTLET_DONOTHING 1
#define EDAC_OUTLET_MOD_DONOTHING 2
#define EDAC_OUTLET_CHARACTERISTIC 3
#define EDAC_OUTLET_MIRROR 4

/* Reference state (u_ref, p_ref) of EDAC_OUTLET_CHARACTERISTIC (Sec. 3.3): the
 * fluid's J2 = rho0 c (u - u_ref) + (p - p_ref), the outlet's u = u_ref +
 * J2/(2 rho0 c), p = p_ref + J2/2.  Default (U, 0). */
edac_status edac_set_outlet_reference(edac_ctx *ctx, double u_ref, double p_ref);
edac_status edac_set_outlet(edac_ctx *ctx, double x_out, int n_layers, int kind, int n_avg,
                            double i_thresh);

/* Solid-wall behaviour of tag EDAC_WALL or EDAC_SLIPWALL (Sec. 2 cites Adami et
 * al. 2012): slip = 0 gives the ghost velocity 2 u_wall - <u_fluid>, slip = 1
 * (normal along y) gives (<u>, -<v>).  count_in_drag adds the particles' force
 * (Eq. tvf-momentum_solid) to the drag/lift history: 0 not counted; 1 summed
 * over fluid neighbours with p~_ij the interpolated pressure (rho_j p_i + rho_i
 * p_j)/(rho_i + rho_j) (the solid-solid pairs of that antisymmetric form cancel
 * in the body's total); 2 the equation as printed, summed over every neighbour
 * with the solid particle's own p_avg,i (Eq. pavg) in p~_ij when p_avg is on.
 * The tangent model and the adjoint take 1 only (EDAC_E_STATE otherwise).
 * Other values: EDAC_E_INVALID.  Defaults: WALL no-slip counted (1), SLIPWALL
 * slip not counted. */
edac_status edac_set_wall(edac_ctx *ctx, int tag, int slip, double uw, double vw,
                          int count_in_drag);

/* Upload n particles from host arrays (copied) and evaluate the rates at t = 0.
 * ids must be unique; tags in [0, 4]; all particles inside the domain box;
 * n <= capacity.  n = 0 is allowed (an empty system).  Resets the step counter,
 * the history and the error word. */
edac_status edac_set_particles(edac_ctx *ctx, int n, const double *h_x, const double *h_y,
                               const double *h_u, const double *h_v, const double *h_p,
                               const double *h_m, const uint8_t *h_tag, const uint64_t *h_id);

/* Advance nsteps time steps.  Asynchronous on the context's stream: no host
 * synchronisation; the live-particle count stays on the device. */
edac_status edac_step(edac_ctx *ctx, int nsteps);

/* Re-evaluate the rates (density, volume, accelerations, pressure rate, wall
 * forces) at the current state without advancing time (asynchronous). */
edac_status edac_evaluate(edac_ctx *ctx);

/* Synchronise and return the live-particle count. */
edac_status edac_get_count(edac_ctx *ctx, int *n_active);

/* Synchronise and copy the live particles to host arrays in ascending id order:
 * h_id and h_tag (either may be NULL) and nfields fields (ids in field_ids,
 * EDAC_F_*) into h_out[f][0..n).  cap: length of every output array.  The
 * columns are permuted into id order on the device (kernels on the context's
 * stream, with the integrator's per-step base-state arrays as scratch, which no
 * result depends on between steps) and copied straight into the outputs. */
edac_status edac_read_state(edac_ctx *ctx, int cap, uint64_t *h_id, uint8_t *h_tag,
                            int nfields, const int *field_ids, double *const *h_out, int *n);

/* Synchronise and copy the per-step history (most recent min(steps, max_steps,
 * max_history) records, oldest first): force on the drag walls (fx, fy), mass
 * flux into the outlet (mass of fluid->outlet conversions / dt), live count,
 * and the numbers of spawned, deleted and fluid->outlet particles.  Any output
 * pointer may be NULL. */
edac_status edac_read_history(edac_ctx *ctx, int max_steps, double *h_fx, double *h_fy,
                              double *h_mass_flux, int *h_n_active, int *h_n_spawn,
                              int *h_n_delete, int *h_n_to_outlet, int *nsteps);

/* Recycling event log: the transitions of Sec. 3.4 taken at the end of each step,
 * one record per event with the step (the step counter after it: 1 for the first
 * step after edac_set_particles), the kind, the particle id and a second id:
 *   EDAC_EVENT_DELETE     an outlet particle past x_out + L_out was removed (other 0)
 *   EDAC_EVENT_TO_OUTLET  a fluid particle past x_out became an outlet particle
 *                         (other 0)
 *   EDAC_EVENT_SPAWN      an inlet particle past x_in became fluid (other: its id)
 *                         and the new inlet particle id was created upstream of it
 * Within a step: deletions, then conversions to outlet, then spawns, each kind in
 * ascending id (spawns in ascending parent id, which is ascending new id).
 * edac_events_bytes: device bytes of a log of max_events records.
 * edac_events_enable: caller-owned device memory, 256-byte aligned, kept alive while
 *   it is set (d_log NULL switches the log off); synchronises the stream and empties
 *   the log.  A step whose events do not all fit is not logged; its events are
 *   counted as dropped.  A batch member logs into the log set before
 *   edac_batch_create.  The forward steps of edac_adjoint_run are logged once.
 * edac_read_events: synchronises, copies the records oldest first into the host
 *   arrays (each may be NULL; cap: their length), sets *n to their number and
 *   *n_dropped (may be NULL) to the events not logged, then empties the log.  cap
 *   below the logged count: EDAC_E_INVALID with *n = that count, log kept.  No log
 *   set: EDAC_E_STATE. */
#define EDAC_EVENT_DELETE 0
#define EDAC_EVENT_TO_OUTLET 1
#define EDAC_EVENT_SPAWN 2
edac_status edac_events_bytes(int max_events, size_t *bytes);
edac_status edac_events_enable(edac_ctx *ctx, void *d_log, size_t bytes);
edac_status edac_read_events(edac_ctx *ctx, int cap, int *h_step, int *h_kind, uint64_t *h_id,
                             uint64_t *h_other, int *n, int64_t *n_dropped);

/* Debug: bytes of caller-owned device scratch that edac_read_neighbors() needs at
 * the current positions (rebuilds the cell list and re-counts neighbours;
 * synchronises; does not change the trajectory). */
edac_status edac_neighbor_scratch_bytes(edac_ctx *ctx, size_t *bytes);

/* Debug: neighbour lists at the current positions, built with the same
 * membership test the pair kernels use.  d_scratch: caller-owned device memory of
 * at least edac_neighbor_scratch_bytes() bytes.  Writes, in ascending id order of
 * i, h_start[0..n] (CSR offsets) and h_nbr_ids[start[i]..start[i+1]) (neighbour
 * ids of i, ascending, i itself included).  cap_n >= n, cap_ids >= total.
 * Synchronises. */
edac_status edac_read_neighbors(edac_ctx *ctx, void *d_scratch, size_t scratch_bytes, int cap_n,
                                int64_t *h_start, int64_t cap_ids, uint64_t *h_nbr_ids, int *n,
                                int64_t *total);

/* Timing: enable (1) or disable (0) CUDA-event timing of one kernel group
 * (EDAC_K_*).  While any group is enabled, edac_step() launches eagerly
 * (no graph) and brackets each launch of the enabled groups with events. */
edac_status edac_profile(edac_ctx *ctx, int kernel, int enable);

/* Synchronise and return the summed device time (ms) and launch count of a
 * timed kernel group since the last reset; reset = 1 clears them. */
edac_status edac_read_profile(edac_ctx *ctx, int kernel, double *ms, int64_t *launches,
                              int reset);

/* Number of kernel launches (and memset nodes) issued by this context so far,
 * graph replays included. */
edac_status edac_launch_count(edac_ctx *ctx, int64_t *count);

/* ---------------------------------------------------------------------------
 * Allocation-free summation density.  The paper has no counterpart: this is a
 * service for callers that cannot allocate device memory at the time they need
 * the result -- code whose framework has handed all device memory to its own
 * pool allocator (a raw allocation would fail or fragment that pool), plug-ins
 * hosted by an application that owns the device memory and gives them none of
 * their own, and real-time code that forbids allocation on its hot path
 * (cudaMalloc and cudaFree can block and synchronise the device).
 * Neither this call nor the library allocates anything for it: the cell-list
 * scratch is a fixed static device array of the library (about 3.7 MB, held on
 * every GPU that loads the library until the process exits).
 *
 * For n particles at d_x, d_y with masses d_m (caller-owned device arrays, fp64,
 * any order) it writes, in the same order, rho_i = sum_j m_j W_ij, the volume
 * 1 / sum_j W_ij and the neighbour count N_i (self included), fp64, with the
 * membership test and quintic spline of edac_step's fp64 path.  Only the domain
 * box, periodic flags, dx, hdx and cuda_stream of params are used.
 * Limits: n <= EDAC_STATIC_MAX_PARTICLES and at most EDAC_STATIC_MAX_CELLS cells
 * (EDAC_E_INVALID / EDAC_E_CAPACITY beyond them); a particle outside the box
 * gives EDAC_E_DOMAIN.  The first call on a device (with that device current)
 * looks up the scratch address; make it before any stream capture.  All calls
 * share the scratch, so calls whose GPU work overlaps (other streams, other
 * host threads on the same device) race.  The particles of a cell are visited in
 * the order the counting atomics give, so the fp64 sums of two calls on the same
 * input may differ in the last bits (edac_step's cell build ranks them instead).
 * Synchronises params->cuda_stream. */
#define EDAC_STATIC_MAX_PARTICLES 262144
#define EDAC_STATIC_MAX_CELLS 65536
edac_status edac_density_static(const edac_params *params, int n, const double *d_x,
                                const double *d_y, const double *d_m, double *d_rho,
                                double *d_vol, int *d_nnb);

/* ---------------------------------------------------------------------------
 * FMA-pipe peak of the current device, measured.  The paper has no counterpart:
 * this is the denominator of the pair passes' roofline (their binding resource
 * is the FP32 pipe on the mixed path and the FP64 pipe on the fp64 path), taken
 * on the device at the clocks it runs under load rather than from a data sheet.
 * kind: EDAC_PEAK_FP32 (the larger of scalar and paired FP32 FMA) or
 * EDAC_PEAK_FP64.  Runs FMA-chain kernels filling every SM for about 0.1 s on
 * cuda_stream (NULL: default stream) and writes the best rate of three timed
 * launches to *tflops, in TFLOP/s with 2 flops per FMA.  Allocates nothing;
 * synchronises the stream.  EDAC_E_INVALID for a bad kind or NULL tflops,
 * EDAC_E_CUDA if a launch or event call fails. */
#define EDAC_PEAK_FP32 0
#define EDAC_PEAK_FP64 1
edac_status edac_fma_peak(int kind, void *cuda_stream, double *tflops);

/* ---------------------------------------------------------------------------
 * Self-check of the library's fp32 <-> fp64 conversions.  The paper has no
 * counterpart: on GB300 the hardware conversions between fp32 and fp64 issue
 * to the fp64 pipe (1/64 of the fp32 rate), so the kernels convert on the
 * integer pipe instead (IEEE 754 widening, and narrowing with round to
 * nearest, ties to even); this compares those conversions with the hardware's
 * on the device.  all_floats != 0: every one of the 2^32 float bit patterns
 * is widened; n_doubles: that many sampled double bit patterns are narrowed
 * (uniform bit patterns, values whose dropped bits sit at or next to a
 * rounding tie, values near the float range's overflow and underflow edges).
 * Writes the mismatch counts (0 when the conversions agree; NaNs compare
 * equal whatever their payload).  Runs on cuda_stream (NULL: default stream)
 * and synchronises it; allocates nothing (the counters are static device
 * variables, so overlapping calls race).  EDAC_E_INVALID for NULL outputs,
 * EDAC_E_CUDA if a copy or launch fails. */
edac_status edac_conversion_check(void *cuda_stream, int all_floats, uint64_t n_doubles,
                                  uint64_t *float_mismatches, uint64_t *double_mismatches);

/* ---------------------------------------------------------------------------
 * Tiling of the mixed path's pair passes (no effect on the fp64 path): a tile
 * is a row segment of tile_cells cells (1..EDAC_TILE_MAX_CELLS) whose block has
 * `threads` threads (a multiple of 32 from 64 to EDAC_TILE_MAX_THREADS).  The
 * default, 11 cells and 160 threads, suits large systems; small ones fill the
 * GPU better with smaller tiles.  Results differ only in the rounding of the
 * fp32 sums (the candidate order changes).  EDAC_E_INVALID outside those
 * values.  Drops the captured step graph. */
#define EDAC_TILE_MAX_CELLS 16
#define EDAC_TILE_MAX_THREADS 256
edac_status edac_set_tiling(edac_ctx *ctx, int tile_cells, int threads);

/* Autotuner of that tiling: times `trials` evaluations (edac_evaluate, which
 * recomputes the rates of the current state: positions, velocities and
 * pressures stay as they are) for each candidate tiling on the context's
 * stream, keeps the fastest, evaluates once more with it and returns it
 * (tile_cells, threads, ms per evaluation; any of them may be NULL).  On the
 * fp64 path it only times the one configuration.  Synchronises the stream. */
edac_status edac_autotune(edac_ctx *ctx, int trials, int *tile_cells, int *threads, double *ms);

/* ---------------------------------------------------------------------------
 * Batches of independent systems (uneven channels, parameter sweeps): one call
 * advances every member one step per graph launch.  The paper has no
 * counterpart; this is the throughput mode for many small systems, which one
 * at a time cannot fill the GPU.  edac_batch_create captures one step of each
 * member, each on its own stream (a non-default stream other than cuda_stream,
 * the batch's own; members that share a stream run one after the other), into
 * one CUDA graph whose branches run concurrently.  Configure the members (inlet, outlet, walls,
 * tiling, particles) first: a member changed afterwards needs a new batch.
 * Members must outlive the batch.  The members' results are bitwise those of
 * stepping each alone.  Errors: EDAC_E_INVALID (NULL, repeated members, a
 * member on the default or the batch stream), EDAC_E_STATE (a member without particles, in error or
 * profiling), EDAC_E_CUDA (capture failed).  Errors of the calls without a
 * context are read with edac_last_error(NULL). */
typedef struct edac_batch edac_batch;
edac_status edac_batch_create(edac_ctx *const *ctxs, int n, void *cuda_stream, edac_batch **out);

/* Fused batch: the step of every member, as with edac_batch_create, but each kernel of
 * the step is launched once over the blocks of all members, so that one step of the whole
 * batch is one graph of about 21 kernel nodes instead of about 20 per member.  The paper
 * has no counterpart (as for edac_batch_create).  Each block of such a launch looks up its
 * member in a block-offset table and runs the single-system kernel body on that member's
 * data, so every member keeps its own cell grid, parameters, time step, tiling and outlet.
 * Its results are bitwise those of stepping it alone on the fp64 path; on the mixed path
 * they agree to fp32 rounding (the batched kernels are separate compilations of the same
 * bodies, in which the compiler may fuse a multiply and an add differently), and runs
 * stay bitwise reproducible.  The tables (the members' device
 * parameters and one offset table per kernel shape) live in caller-owned device memory of
 * edac_batch_workspace_bytes(n) bytes, 256-byte aligned, kept alive while the batch exists;
 * the library allocates nothing.  The members must share the precision; the mixed pair
 * passes run with the largest thread count of the members' tilings.  Stepped, counted and
 * released with edac_batch_step, edac_batch_launch_count and edac_batch_destroy; as for
 * edac_batch_create, configure the members first and keep them alive.  Errors: those of
 * edac_batch_create, and EDAC_E_INVALID for a missing, small or misaligned workspace or
 * members of different precision.  Synchronises cuda_stream once (the table upload). */
edac_status edac_batch_workspace_bytes(int n, size_t *bytes);
edac_status edac_batch_create_fused(edac_ctx *const *ctxs, int n, void *cuda_stream,
                                    void *d_workspace, size_t bytes, edac_batch **out);

/* nsteps steps of every member: nsteps graph launches on the batch stream, which
 * first waits for the work queued on the members' streams; the members' streams
 * then wait for the batch.  Asynchronous. */
edac_status edac_batch_step(edac_batch *batch, int nsteps);

/* Kernels launched per batch step (all members). */
edac_status edac_batch_launch_count(edac_batch *batch, int64_t *kernels_per_step);

/* Release the batch (synchronises its stream); the members stay valid. */
void edac_batch_destroy(edac_batch *batch);

/* Probes (the measurement points of Sec. 4's test problems): at n points (1..
 * EDAC_MAX_PROBES, host arrays h_x, h_y) the Shepard averages sum f W / sum W of
 * the fluid p, u, v over the fluid particles within 3h of the point (the exact
 * membership test of the passes), in fp64 on both paths, and the fluid count:
 * h_out[4 i + 0..3] = (p, u, v, count).  All weights zero: the plain means;
 * no fluid in reach: zeros.  Uses the state after the last step (tags after
 * recycling).  Synchronises the stream. */
#define EDAC_MAX_PROBES 8
edac_status edac_probe(edac_ctx *ctx, int n, const double *h_x, const double *h_y, double *h_out);

/* ---------------------------------------------------------------------------
 * Tangent-linear model (fp64 path, steady inlet modes, hybrid outlet): the
 * derivatives of the step with respect to the inlet modes a_1..a_8 of
 * u(y) = U + sum_k a_k sin(k pi (y - y0)/H) (edac_set_inlet), carried forward
 * next to the values, with the neighbour sets, the gate decisions, the outlet
 * classes and the recycling events the values produce held fixed.  Gives the
 * gradient of any functional of the force history, such as the time-averaged
 * drag, with respect to the modes.  It is forward-mode (no checkpoints); the
 * pair-pass tangents run in fp32 (relative rounding ~1e-7, against the fp64
 * step's derivatives), the boundary parts in fp64: a tangent step costs a few
 * fp64 steps (2.8x on a 98k-particle cylinder).
 *   edac_tangent_workspace_bytes: device bytes the tangents need (caller-owned,
 *     256-byte aligned, kept alive while tangents are stepped);
 *   edac_tangent_enable: set the tangents of the current state (zero except the
 *     inlet velocities, whose derivatives are the mode shapes) and of its rates;
 *     EDAC_E_STATE on the mixed path or with other inlet/outlet kinds;
 *   edac_step_tangent: nsteps steps of values and tangents (no graph);
 *   edac_read_tangent_history: for the last steps (at most max_steps, and not
 *     before the enable) d F_x / d a_k into h_dfx[step * 8 + k] and d F_y / d a_k
 *     into h_dfy, aligned with edac_read_history; synchronises the stream. */
#define EDAC_TANGENT_DIRECTIONS 8
edac_status edac_tangent_workspace_bytes(edac_ctx *ctx, size_t *bytes);
edac_status edac_tangent_enable(edac_ctx *ctx, void *d_workspace, size_t bytes);
edac_status edac_step_tangent(edac_ctx *ctx, int nsteps);
edac_status edac_read_tangent_history(edac_ctx *ctx, int max_steps, double *h_dfx,
                                      double *h_dfy, int *nsteps);

/* ---------------------------------------------------------------------------
 * Reverse-mode adjoint (fp64 path, steady inlet modes, hybrid outlet or none):
 * the gradient with respect to the inlet modes a_1..a_8 (edac_set_inlet) of
 *   L = sum_n [ w_fx[n] F_x^n + w_fy[n] F_y^n
 *               + w_pe[n] sum_{fluid i} omega(x_i) p_i^2 at the end of step n ]
 * over nsteps steps from the current state (F: the force on the drag walls of
 * each step, as in edac_read_history; the last term is the pressure energy of
 * the fluid in an x-window, e.g. the layer in front of the outlet where waves
 * the outlet reflects stay, with the weight omega = sin^2(pi (x - pe_x0) /
 * (pe_x1 - pe_x0)) on [pe_x0, pe_x1) and 0 outside, which vanishes smoothly at
 * both edges so that particles crossing them change L continuously).  The paper has no counterpart (it states the
 * method, not its derivatives).  The adjoint of every operation of a step is
 * taken in reverse order with the neighbour sets, the acoustic-gate decisions,
 * the red/blue outlet classes and the recycling events of the forward run held
 * fixed, as in the tangent model; the forward run keeps a checkpoint of the
 * context's workspace every checkpoint_every steps and the reverse sweep
 * recomputes each segment from its checkpoint once (storing its steps), then
 * each step from its snapshot.  Its cost is that of a few fp64 forward runs
 * for any number of parameters.  The context must be freshly uploaded (no steps
 * taken since edac_set_particles) and is left in the state after nsteps steps
 * (as edac_step would leave it, history included).
 *   edac_adjoint_workspace_bytes: device bytes edac_adjoint_run needs for these
 *     nsteps and checkpoint_every (the adjoint fields and (nsteps /
 *     checkpoint_every + 1 + checkpoint_every) copies of the context's workspace);
 *   edac_adjoint_run: d_workspace caller-owned, 256-byte aligned, at least that
 *     many bytes; any weight array may be NULL (zeros), else nsteps values;
 *     writes L to *h_loss (may be NULL) and dL/da_k, k = 1..8, to h_grad[0..7]
 *     (zero for modes beyond those edac_set_inlet set).  nsteps <= max_history.
 *     Synchronises the stream.  EDAC_E_STATE on the mixed path, with other inlet
 *     or outlet kinds, after steps, or in error; EDAC_E_INVALID for bad sizes. */
edac_status edac_adjoint_workspace_bytes(edac_ctx *ctx, int nsteps, int checkpoint_every,
                                         size_t *bytes);
edac_status edac_adjoint_run(edac_ctx *ctx, void *d_workspace, size_t bytes, int nsteps,
                             int checkpoint_every, const double *h_w_fx, const double *h_w_fy,
                             const double *h_w_pe, double pe_x0, double pe_x1, double *h_loss,
                             double *h_grad);

/* Text of the last error of this context (valid until the next call); with
 * ctx = NULL, the last error of a context-less call (edac_workspace_bytes,
 * edac_create) made on this host thread. */
const char *edac_last_error(edac_ctx *ctx);

/* Release the context (host memory, events, graphs).  The workspace stays the
 * caller's.  Synchronises the stream first. */
void edac_destroy(edac_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* EDAC_H */

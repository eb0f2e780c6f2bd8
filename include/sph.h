/*
 * sph.h -- C ABI of the GB300 two-phase weakly compressible SPH particle loop.
 *
 * Method: Wei et al., "Behavior of Oil under Breaking Waves by a Two-phase SPH
 * Model", Sec. II.  One time step evaluates, for every particle, the per-phase
 * density renormalisation (Eq. ct_dist_3), the equation of state (Eqs. state
 * and beta), the colour-index gradient (Eq. cd) and surface stress tensor
 * (Eq. csf), the symmetric pressure gradient (Eq. dist_p_1), the harmonic-mean
 * two-phase viscosity (Eq. visc_2, or Eq. visc_1), the surface-tension force
 * (F_s/rho, Sec. II-C), gravity, and the two-phase continuity equation
 * (Eq. ct_dist_2), and advances the state with an explicit midpoint
 * predictor-corrector.  Dynamic boundary particles (Sec. III) are water
 * particles whose position and velocity stay fixed while their density
 * integrates.
 *
 * Conventions for every entry point:
 *   - Return value: SPH_OK (0) or a negative SPH_E* code; the message of the
 *     last failure on the calling thread is available from sph_last_error().
 *     The library never aborts the process.
 *   - Host arrays are owned by the caller and only read (or, for sph_read,
 *     written) during the call.  Device memory belongs to the handle from
 *     sph_create until sph_destroy.
 *   - All GPU work is issued on the CUDA stream given to sph_create, in call
 *     order.  sph_step and sph_run return once the work is queued; errors
 *     raised on the device (non-finite values, a particle leaving the box, a
 *     step too large for the neighbour-search skin) are reported by the next
 *     call that waits for the stream: sph_run, sph_sync, sph_read,
 *     sph_neighbours, sph_diag.
 *   - Particle order: arrays passed in and read out are in the caller's
 *     original order (particle id = index in the arrays given to sph_create).
 */
#ifndef SPH_H
#define SPH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Error codes */
#define SPH_OK          0
#define SPH_EINVAL     -1  /* invalid argument or parameter */
#define SPH_ENOMEM     -2  /* device or host allocation failed */
#define SPH_ECUDA      -3  /* a CUDA runtime call failed */
#define SPH_ENONFINITE -4  /* a NaN or Inf appeared in the state */
#define SPH_ECFL       -5  /* a particle moved farther in a step than the cell skin allows */
#define SPH_EDOMAIN    -6  /* a particle left the box of the cell grid */
#define SPH_ECAPACITY  -7  /* a particle has more neighbours than max_neighbours */
#define SPH_ETIMEOUT   -8  /* a grid barrier of the persistent kernel gave up after one second */
#define SPH_EFALLBACK  -9  /* the judge rejected a surrogate jump; the state holds the plain
                              method's result (sph_surrogate_advance_judged), not a failure */
#define SPH_EBOUNDS   -10  /* an index read from device data was out of range (reported by the
                              bounds-checked build only; the access was skipped) */

/* Viscous term forms (Sec. II-C) */
#define SPH_VISC_DYNAMIC   0  /* Eq. visc_2: (1/rho_i) sum 2 mu_ij (m_j/rho_j) (r.gradW)/(r^2+delta^2) u_ij */
#define SPH_VISC_KINEMATIC 1  /* Eq. visc_1: sum 2 nu_ij (m_j/rho_j) (r.gradW)/(r^2+delta^2) u_ij, nu = mu/rho0 */

/* Fields for sph_read.  Floating fields are written as double, integer fields
 * as int32.  "eval" fields hold the last rates evaluation (sph_eval_rates, or
 * stage 2 of the last sph_step). */
#define SPH_FIELD_POS        0  /* n*dim  position x (state) */
#define SPH_FIELD_VEL        1  /* n*dim  velocity u (state) */
#define SPH_FIELD_RHO        2  /* n      density rho (state) */
#define SPH_FIELD_RHO_EVAL   3  /* n      density after renormalisation, Eq. ct_dist_3 (eval) */
#define SPH_FIELD_PRESSURE   4  /* n      pressure P, Eq. state (eval) */
#define SPH_FIELD_ACC        5  /* n*dim  acceleration Du/Dt, zero on walls (eval) */
#define SPH_FIELD_DRHO       6  /* n      density rate Drho/Dt, Eq. ct_dist_2 (eval) */
#define SPH_FIELD_TENSOR     7  /* n*dim*dim surface stress tensor T, Eq. csf (eval) */
#define SPH_FIELD_CELL       8  /* n      int32 cell id of the last cell-list build */
#define SPH_FIELD_ORDER      9  /* n      int32 particle id at each sorted position:
                                   the stable order by (cell id, particle id) */

/* Physical and numerical parameters.  The layout is fixed; unused 3-D
 * entries are ignored when dim == 2. */
typedef struct sph_params {
    int32_t dim;           /* 2 or 3 */
    int32_t visc_form;     /* SPH_VISC_DYNAMIC or SPH_VISC_KINEMATIC */
    int32_t renorm_every;  /* Eq. ct_dist_3 at stage 1 of steps with step % renorm_every == 0; 0 = never */
    int32_t max_neighbours;/* capacity of the per-particle neighbour list (pairs closer
                              than 2h + 2 skin), rounded up to a multiple of 4; 0 selects
                              48 in 2-D and 128 in 3-D */
    int32_t rebuild_every; /* 0: the cell and neighbour lists are rebuilt when a particle
                              may move farther than skin from where it was at the last
                              build; k > 0: rebuilt every k steps */
    int32_t periodic;      /* bit a set: axis a is periodic with period box_hi[a] - box_lo[a]
                              (the cross-tank boundary of the flume runs, Sec. "Laboratory
                              experiment & numerical setup").  The period must hold a whole
                              number of super-cells, at least three: cell_size when
                              cell_size >= 2h + 2 skin, else 2 cell_size.  Positions are read
                              back wrapped into the box.  Not allowed in a batch. */
    int32_t renorm_walls;  /* 1: dynamic boundary particles are renormalised (Eq. ct_dist_3)
                              like water particles, the paper's reading: Sec. III gives them
                              the fluid's equations of continuity and state, and Eq. ct_dist_3
                              is part of the discretised continuity equation (Sec. II-B).
                              0: they keep the density continuity gives them (a stabilisation
                              of long runs, not the paper's); they still enter the water's
                              sums either way. */
    int32_t reserved;      /* must be 0 */
    double h;              /* smoothing length; the Wendland C2 kernel has support 2h */
    double c0;             /* reference speed of sound C_s0 (Eq. beta) */
    double gamma;          /* exponent of Eq. state; must be 7 (the paper's value) */
    double delta;          /* regulariser of the viscous term (the paper uses 0.1 h) */
    double alpha_s;        /* interfacial surface tension coefficient (Eq. csf) */
    double cell_size;      /* edge of the cell grid used for hashing, sorting and the
                              neighbour search; >= h + skin (half the list radius) */
    double skin;           /* the neighbour list holds the pairs closer than 2h + 2 skin,
                              so it stays complete while no particle has moved farther
                              than skin since the list was built */
    double g[3];           /* gravitational acceleration */
    double rho0[2];        /* reference density per phase: [0] water, [1] oil */
    double mu[2];          /* dynamic viscosity per phase */
    double mass[2];        /* particle mass per phase */
    double box_lo[3];      /* lower corner of the domain covered by the cell grid */
    double box_hi[3];      /* upper corner */
} sph_params;

typedef struct sph_sim *sph_handle;

/* Creates a simulation of n particles and copies the initial state to the GPU.
 *   x, u   : n*dim doubles, row-major (particle-major), positions and velocities
 *   rho    : n doubles, densities
 *   phase  : n bytes, 0 = water, 1 = oil
 *   wall   : n bytes, 0 = fluid, 1 = dynamic boundary particle, 2 = piston
 *            particle (a boundary particle moved by sph_set_piston); boundary
 *            and piston particles must be phase 0.  Boundary particles keep
 *            the position and velocity they are given (Sec. III); while every
 *            wall == 1 particle has zero velocity (the intended use) the force
 *            sweep skips their mutual pairs, whose terms are zero, and a state
 *            in which one moves is computed in full (same results)
 *   stream : a cudaStream_t, or NULL for the default stream
 * Every position must lie inside [box_lo, box_hi].  On success *out holds the
 * handle; on failure *out is NULL and nothing is leaked. */
int sph_create(const sph_params *params, int64_t n, const double *x, const double *u,
               const double *rho, const uint8_t *phase, const uint8_t *wall,
               void *stream, sph_handle *out);

/* Creates ONE handle over k >= 1 independent instances (a batch of separate
 * problems advanced together by every launch; the paper runs one problem at
 * a time, so this packing is this library's).  params[q] holds instance q's
 * parameters; all instances must share dim, h, gamma, delta, g, cell_size,
 * skin, visc_form, renorm_every, rebuild_every and max_neighbours, and may
 * differ in c0, alpha_s, rho0, mu, mass and box.  counts[q] particles belong
 * to instance q; x, u, rho, phase and wall hold the instances one after
 * another (instance 0's particles first), each in its own frame and box.
 * The boxes are packed side by side in one cell grid (a shelf packing in the
 * x-y plane) with gaps of 2h + 2 skin + 2 cell_size, so no two instances
 * interact; every read returns positions in each instance's own frame.
 * Particle ids run over the whole batch.  k <= 65535, total n <= 2^26.  A
 * particle that leaves its own box but not the packed grid is not reported
 * as SPH_EDOMAIN: walls keep particles inside in the intended use. */
int sph_create_batch(int k, const sph_params *params, const int64_t *counts, const double *x,
                     const double *u, const double *rho, const uint8_t *phase, const uint8_t *wall,
                     void *stream, sph_handle *out);

/* As sph_create, with x, u, rho, phase and wall in device memory (e.g. torch
 * tensors); they are copied, so the caller keeps them.  Waits for `stream`. */
int sph_create_dev(const sph_params *params, int64_t n, const double *x_dev, const double *u_dev,
                   const double *rho_dev, const uint8_t *phase_dev, const uint8_t *wall_dev, void *stream,
                   sph_handle *out);

/* Prescribed motion of the piston particles (wall == 2), the piston-type wave
 * maker of Sec. "Laboratory experiment & numerical setup": they move rigidly
 * along `axis` with displacement, for t <= t_end,
 *   X(t) = sum_{c < ncomp} amp[c] (sin(omega[c] t + phase[c]) - sin(phase[c]))
 * and velocity X'(t); after t_end they rest at X(t_end) (t_end may be
 * infinite).  The paper's stroke x(t) = S/2 - S/2 cos(2 pi f t), 0 <= t <=
 * 1/(2f), is ncomp = 1, amp = S/2, omega = 2 pi f, phase = -pi/2, t_end =
 * 1/(2f).  A step from time t puts them at X(t + dt/2) - X(t) from where they
 * are, velocity X'(t + dt/2), for the second stage, and at X(t + dt) - X(t),
 * velocity X'(t + dt), at its end; their density integrates like a fixed
 * boundary particle's.  The state's velocity of a piston particle should be
 * X'(t) along the axis at the current time.  ncomp = 0 stops the motion
 * (pistons then stay where they are).  Single-instance handles only; at most
 * 8 components.  The time is the handle's clock (sph_get_time). */
int sph_set_piston(sph_handle h, int axis, int ncomp, const double *amp, const double *omega, const double *phase,
                   double t_end);

/* The handle's clock: 0 at creation, advanced by dt by every step (by
 * repeated addition).  Reading waits for the stream. */
int sph_get_time(sph_handle h, double *t);
int sph_set_time(sph_handle h, double t);

/* A time step for the current state: the smallest over instances q of
 *   min(0.25 h / c0, 0.125 h^2 / nu_max, 0.25 sqrt(rho0_min h^3 / (2 pi alpha_s)),
 *       0.25 sqrt(h / |a|_max)) / dt_scale[q],
 * nu_max = max over phases of mu / rho0, rho0_min the smaller reference
 * density, |a|_max the largest acceleration of a fluid particle in the last
 * rates evaluation (that term is left out before the first one; the tension
 * term when alpha_s = 0).  The paper fixes only c0 >= 10 u_max (Sec. II-A);
 * the four bounds are the usual acoustic, viscous, capillary and body-force
 * limits of weakly compressible SPH.  Waits for the stream. */
int sph_suggest_dt(sph_handle h, double *dt);

/* Perturbs the state in place (no counterpart in the paper: training-data
 * augmentation for the learned surrogate, and robustness tests): every
 * velocity component of a fluid particle gets N(0, sigma_u^2) added, its
 * density a factor 1 + N(0, sigma_rho^2).  The variates come from a
 * counter-based generator (SplitMix64, Box-Muller) keyed on seed, the
 * original particle id and the channel, so they do not depend on the
 * particle order.  The next step or evaluation rebuilds the lists.
 * Queued on the stream. */
int sph_perturb_state(sph_handle h, double sigma_u, double sigma_rho, uint64_t seed);

/* Interface error between the oil of two handles (e.g. a variant of a run and
 * the plain run): with O the set of cells of a grid of spacing
 * d_p = (m_oil / rho0_oil)^(1/dim) from box_lo that hold at least one oil
 * particle, *err = |O_a xor O_b| / |O_b| (0 for identical oil layouts; 1e30
 * if b has no oil and a has).  Both handles must have the same cell grid and
 * oil particle volume (SPH_EINVAL otherwise).  Waits for both streams. */
int sph_oil_occupancy_diff(sph_handle a, sph_handle b, double *err);

/* Per-instance step sizes: instance q advances by dt * scales[q] whenever the
 * handle advances by dt (each scale in (0, 1]).  Default 1. */
int sph_set_dt_scales(sph_handle h, const double *scales);

/* Replaces the state (x, u, rho; same layout as sph_create) of an existing
 * handle with host data, keeping its parameters, phases and walls (device or
 * managed memory is also accepted and read in place).  The step
 * counter is left as it is.  After a step has run (and with rebuild_every ==
 * 0) the cell order and neighbour list are kept when every particle of the
 * new state is within the corrector's skin test of its position at the last
 * list build (now and half a step of the last dt ahead); otherwise, or with a
 * non-finite position, the next step rebuilds them.  Either way the result
 * of the following steps is that of a handle created at the new state, up to
 * the particle order in which the sums are taken.  Synchronises the stream. */
int sph_set_state(sph_handle h, const double *x, const double *u, const double *rho);

/* Builds the cell list at the current positions: cell hash, stable sort by
 * (cell id, particle id), reorder of every per-particle array, cellStart and
 * cellEnd (the neighbour search; the paper inherits it from the GPU code
 * base named at the end of Sec. II-C and does not describe it). */
int sph_build_cells(sph_handle h);

/* One evaluation of the rates at the current state, on a fresh cell list,
 * renormalising the density when the current step index calls for it.  Does
 * not advance the state; the results are read with the *_EVAL fields,
 * SPH_FIELD_PRESSURE, SPH_FIELD_ACC, SPH_FIELD_DRHO and SPH_FIELD_TENSOR. */
int sph_eval_rates(sph_handle h);

/* One predictor-corrector step of size dt > 0 (cell build, two rates
 * evaluations, two integrations).  Queues the work and returns. */
int sph_step(sph_handle h, double dt);

/* nsteps steps of size dt, then waits for the stream and reports any device
 * error.  With graph != 0 one step is captured once into a CUDA graph and
 * replayed: a one-thread kernel copies the device rebuild flag into the
 * condition of a conditional (IF) node whose body is the cell-list chain, so
 * steps without a list build launch five kernels instead of fourteen.  The
 * eager form (graph == 0) launches all fourteen, the cell-list kernels
 * returning at once without a build; both compute the same bits. */
int sph_run(sph_handle h, double dt, int64_t nsteps, int graph);

/* The same nsteps steps as sph_run in ONE cooperative kernel launch: every
 * phase of the step (cell build when due, both sweeps of both stages) is a
 * grid-stride loop over the particles, phases separated by a grid-wide
 * barrier.  The results are bit-identical to sph_run's (same per-particle
 * arithmetic and summation order).  Every barrier wait gives up after one
 * second; the launch then returns early, the state is left partly advanced
 * and the call returns SPH_ETIMEOUT.  The launch uses the shape set by
 * sph_set_launch_shape or chosen by sph_autotune (default: 256 threads, as
 * many blocks per SM as fit).  With graph != 0 the launch is captured into a
 * CUDA graph (re-captured when dt, nsteps or the shape changes).  Waits for
 * the stream.  nsteps < 2^31. */
int sph_run_persistent(sph_handle h, double dt, int64_t nsteps, int graph);

/* Launch shape of sph_run_persistent: block in {128, 256, 512} threads,
 * grid_blocks blocks (clamped to what can be co-resident; 0 = as many as
 * can), and how each phase's particles are shared out: dynamic_chunks = 1
 * hands chunks of consecutive particles to warps from a grid-wide counter,
 * 0 gives each thread a fixed grid-stride share.  Shapes of at most 512
 * threads per SM run a build of the kernel with up to 128 registers a
 * thread, the others one with 64.  sph_get_launch_shape returns the shape
 * with the grid it gives on the current device.  Default: 256, 0, 1. */
int sph_set_launch_shape(sph_handle h, int block, int grid_blocks, int dynamic_chunks);
int sph_get_launch_shape(sph_handle h, int *block, int *grid_blocks, int *dynamic_chunks);

/* Times sph_run_persistent over trial_steps steps of size dt for every block
 * size in {128, 256, 512} with grids of every co-resident multiple of the SM
 * count, and, where the particles are fewer than twice such a grid's
 * threads, of 1/2, 1/4, 1/8 and 1/19 of the SM count, each with both ways of
 * sharing out particles; keeps the fastest shape and writes it and its
 * milliseconds per step to the non-NULL outputs.
 * Each trial starts from the state at entry; afterwards the state, the step
 * counter and the build counter are put back as they were (the next step
 * rebuilds the lists). */
int sph_autotune(sph_handle h, double dt, int trial_steps, int *best_block, int *best_grid_blocks,
                 int *best_dynamic_chunks, double *best_ms_per_step);

/* Waits for the stream and reports any device-side error flag. */
int sph_sync(sph_handle h);

/* Test support for the barrier time-out (no counterpart in the paper): puts
 * the persistent kernel's grid barrier in a state that no arrival completes,
 * so that the next sph_run_persistent waits out its one-second limit in every
 * block and returns SPH_ETIMEOUT, after which the barrier is reset and runs
 * work again.  The state advanced by that call is undefined. */
int sph_test_stall_barrier(sph_handle h);

/* Copies a field (SPH_FIELD_*) into host memory in original particle order.
 * bytes must be at least the field's size (see the field list).  Device or
 * managed memory is written in place by the kernel that unpermutes the
 * field; host memory (pinned is fastest) through a staging copy.  Waits for
 * the stream. */
int sph_read(sph_handle h, int field, void *host_out, int64_t bytes);

/* x, u (n*dim) and rho (n) in one call with one wait: the state as sph_read
 * gives it, and the argument sph_set_state takes.  Reports device error
 * flags like sph_sync. */
int sph_read_state(sph_handle h, double *x, double *u, double *rho);

/* Advances a state held by the caller: loads (x, u, rho) as sph_set_state
 * does, runs nsteps graph-replayed steps of dt as sph_run does, and writes
 * the resulting state to (x_out, u_out, rho_out) as sph_read_state does — all
 * queued on the handle's stream with one wait at the end instead of one per
 * call.  Layouts are those of sph_create (original particle order, x and u
 * n*dim, rho n); host memory (pinned is fastest) goes through the staging
 * copies, device or managed memory is used in place.  The outputs may be the
 * inputs.  Returns SPH_EINVAL for a NULL array, a non-positive or non-finite
 * dt or a negative nsteps, and reports device error flags like sph_sync. */
int sph_advance_host(sph_handle h, double dt, int64_t nsteps, const double *x, const double *u, const double *rho,
                     double *x_out, double *u_out, double *rho_out);

/* Neighbour sets at the current positions (rebuilds the cell list, which
 * invalidates the eval fields) as computed by the GPU's own
 * candidate test (j != i and |r_ij|^2 < (2h)^2 in the kernels' arithmetic),
 * in CSR form over original particle ids, each row ascending.  start has n+1
 * entries.  Returns the number of pairs (>= 0), or SPH_EINVAL when cap is too
 * small (start is filled in that case, so a second call can size list). */
int64_t sph_neighbours(sph_handle h, int64_t *start, int32_t *list, int64_t cap);

/* Neighbour statistics at the current positions (rebuilds the cell list):
 * out[0] = number of ordered pairs (i, j), j != i, with |r_ij| < 2h;
 * out[1] = how many of them join particles of different phase.  These are
 * the pair counts the interaction sweeps evaluate. */
int sph_pair_stats(sph_handle h, int64_t out[2]);

/* The same count by classes (rebuilds the cell list): out[0] and out[1] as
 * in sph_pair_stats; out[2] = ordered pairs of two static boundary particles
 * (wall flag 1); out[3] = ordered pairs (i, j) of a static boundary particle
 * i with a particle j that is not one.  While every static boundary particle
 * is at rest the force sweep (Eq. dist_p_1, visc_2, ct_dist_2) leaves out the
 * out[2] pairs, whose terms are zero (u_ij = 0 in the continuity term; a
 * boundary particle's acceleration is not used), and of the out[3] pairs only
 * the continuity term is needed.  Errors: SPH_EINVAL for a NULL argument. */
int sph_pair_classes(sph_handle h, int64_t out[4]);

/* FP64 diagnostics over the fluid particles (walls excluded):
 *   out[0] mass, out[1..3] momentum sum m u, out[4] kinetic energy,
 *   out[5] potential energy -sum m g.x, out[6..8] oil centroid,
 *   out[9] oil sphericity sqrt(lambda_min/lambda_max) of the covariance of
 *   oil positions, out[10] max |u|, out[11] number of oil particles. */
int sph_diag(sph_handle h, double out[12]);

/* sph_diag for every instance of a batch: out holds 12 doubles per instance
 * (instance q at out[12 q], same layout as sph_diag, positions in the
 * instance's own frame).  sph_diag on a batch reports instance 0. */
int sph_diag_instances(sph_handle h, double *out);

/* Per-kernel timing with CUDA events on the simulation's stream.  While
 * enabled, every launch is bracketed by events; sph_timing_read returns, for
 * kernel index k (0 <= k < sph_timing_count()), its name, launch count and
 * total milliseconds since the last reset. */
int sph_timing_enable(sph_handle h, int enable);
int sph_timing_reset(sph_handle h);
int sph_timing_count(void);
int sph_timing_read(sph_handle h, int k, const char **name, int64_t *launches, double *total_ms);

/* Number of cell and neighbour-list builds performed so far (waits for the
 * stream), or a negative error code. */
int64_t sph_list_builds(sph_handle h);

/* Number of particles (all instances), step counter, grid cells. */
int64_t sph_num_particles(sph_handle h);
int64_t sph_step_index(sph_handle h);
int64_t sph_num_cells(sph_handle h);
/* Number of instances (1 unless created by sph_create_batch). */
int64_t sph_num_instances(sph_handle h);

void sph_destroy(sph_handle h);

/* Allocation-free cell sort (no counterpart in the paper).  It serves callers
 * that cannot allocate device memory: a host application whose device memory
 * belongs to its own pool or allocator (a cudaMalloc from inside it would
 * fail or fragment that pool), or a deployment whose device memory is fixed
 * in advance.  Computes, for n particles whose positions x_dev are a device
 * array of n * dim doubles (particle-major), the cell id of each particle on
 * the grid of params (cell_size, box_lo, box_hi) into cell_dev (n int32,
 * device) and the particle ids in the stable order by (cell id, particle id)
 * into order_dev (n int32, device): the same values as SPH_FIELD_CELL and
 * SPH_FIELD_ORDER after sph_build_cells.  The caller owns all three arrays.
 * No device memory is allocated: the scratch is one file-scope device array
 * of about 21 MB that every GPU loading the library holds until the process
 * exits, limiting n to 2^20 particles and the grid to 2^20 cells (larger
 * sizes return SPH_EINVAL).  The first call on a device looks up that
 * array's device address (once per device, with the device current) and
 * caches it, so make the first call before any stream capture; a device
 * reset (cudaDeviceReset) invalidates the cached address, so do not call
 * this again in the same process after one.  Every call on a device shares
 * the array and keeps the last call's contents (the parts that must start at
 * zero are cleared by each call); calls that overlap on the GPU race.  Before
 * returning, the call copies a one-word out-of-box flag to the host and waits
 * for the stream; it returns SPH_EDOMAIN when a particle lies outside the
 * box (the cell ids of such a particle are then clamped into the grid). */
int sph_cell_sort_noalloc(const sph_params *params, int64_t n, const double *x_dev, int32_t *cell_dev,
                          int32_t *order_dev, void *stream);

/* FP32 fused multiply-add throughput of the current device (no counterpart
 * in the paper: the measured denominator of the force sweeps' roofline).
 * Launches blocks_per_sm (1..8) resident blocks of 256 threads on every SM,
 * each thread running 16 independent FMA chains of iters (1..2^20) steps,
 * once to warm up and once timed with CUDA events on stream (NULL: the
 * default stream); waits for the stream.  Writes the achieved rate in
 * TFLOP/s (2 flops per FMA) to *tflops and the timed launch's duration to
 * *ms.  Allocates nothing; reads no memory. */
int sph_fp32_peak(int blocks_per_sm, int iters, void *stream, double *tflops, double *ms);

/* Message of the last failure on the calling thread ("" if none). */
const char *sph_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SPH_H */

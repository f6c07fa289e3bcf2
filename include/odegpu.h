/*
 * odegpu.h -- C ABI of the GB300 (sm_103a) library that integrates very many
 * independent, identical, low-order ODE systems, one system per GPU thread,
 * after F. Hegedus, "Modular, general purpose ODE integration package to solve
 * large number of independent ODE systems on GPUs" (arXiv:1810.03931).
 *
 * Conventions shared by every call
 * --------------------------------
 * Return value: int status, ODE_OK (0) on success, a negative ODE_ERR_* code
 *   otherwise.  The message of the last failure is returned by
 *   ode_last_error(solver) (or ode_last_error(NULL) for failures that have no
 *   solver, e.g. ode_create).  A failed call leaves the solver usable unless
 *   the CUDA context itself was lost (ODE_ERR_CUDA with a sticky CUDA error).
 * Layout: every per-system array is structure-of-arrays, component-major:
 *   value[component * stride + system], as the problem pool of Sec. 6.1 of the
 *   paper prescribes (Fig. "problem pool"; the index idx + i*NoT of Sec. 6.5).
 *   All floating-point data are IEEE binary64 (double).
 * Ownership: the solver owns all of its device buffers (allocated by
 *   ode_create, freed by ode_destroy).  Caller buffers are only read or
 *   written during the call (or, for calls that take a stream, by work
 *   enqueued on that stream); no call keeps a caller pointer after it returns.
 * Pointer kind: calls that take caller arrays have a ptr_kind argument,
 *   ODE_PTR_HOST (host memory, pageable or pinned) or ODE_PTR_DEVICE (device
 *   memory of the solver's device, e.g. a torch CUDA tensor's data_ptr()).
 * Streams: a `void *stream` argument is a cudaStream_t (NULL = the legacy
 *   default stream).  Calls with ODE_PTR_HOST arrays synchronize that stream
 *   before returning; calls with device arrays only enqueue work.
 * Threads: a solver may be used from one host thread at a time.
 * Nothing on this interface falls back to the CPU: with no usable GPU,
 *   ode_create fails with ODE_ERR_CUDA.
 */
#ifndef ODEGPU_H
#define ODEGPU_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ode_solver ode_solver; /* opaque; the ParametricODESolver object of Sec. 6.2 */

/* Models: the pre-declared device hooks of Sec. 6.5-6.8 are compiled into
 * the library per model (Sec. 6.9: hooks in the kernels' translation unit).
 *  ODE_DUFFING        Eqs. (1)-(2): n=2, P=2 (k, B), A=7, E=1 (F0 = y2)
 *                     solver constants (delta, c3, omega), default (-1, 1, 1)
 *                     i.e. x'' + k x' + x + x^3 = B cos(omega t);
 *                     c3 = 0 gives the linear damped forced oscillator.
 *  ODE_KELLER_MIKSIS  Eqs. (12)-(28): n=2, P=13 (C0..C12), A=4, E=1 (F0 = y2)
 *  ODE_VALVE          Eqs. (29)-(34): n=3, P=5 (kappa, delta, beta, q, r),
 *                     A=5, E=2 (F0 = y2, F1 = y1 with impact y2 <- -r y2)
 *  ODE_BOUNCE         bouncing ball (closed-form checks): n=2, P=2 (g, r),
 *                     A=6, E=1 (F0 = y1 with impact y2 <- -r y2)
 *  ODE_DUFFING_LYAPUNOV  Eqs. (1)-(6): the Duffing model with its
 *                     linearisation in polar coordinates attached (y3 =
 *                     radius, y4 = angle of a tangent vector): n=4, P=2
 *                     (k, B), A=5, E=1 (F0 = y2), constants as ODE_DUFFING.
 *                     Finalization (Sec. 6.8, Eq. (7)) stores a4 = ln y3,
 *                     resets y3 = 1 and reduces y4 modulo 2 pi to [-pi, pi]
 *                     at every slice end, so the largest
 *                     Lyapunov exponent is the mean of a4 over slices divided
 *                     by the slice length (Eq. (7) as printed averages y3
 *                     itself; the logarithm is read).  Binary64 only.
 * Accessories (Sec. 5, Sec. 6.7), all models: a0 = max y1, a1 = its time,
 *   a2 = min y1, a3 = its time (over accepted points of one slice);
 *   Duffing a4, a5 = y1 and t at the first detection of event 0, a6 = count
 *   of event-0 detections; valve a4 = number of impacts; ball a4 = time of the
 *   last impact, a5 = velocity just before it.  Initialization (Sec. 6.8)
 *   sets a0..a5 from the state at the slice start and counts to zero. */
enum ode_model {
  ODE_DUFFING = 0,
  ODE_KELLER_MIKSIS = 1,
  ODE_VALVE = 2,
  ODE_BOUNCE = 3,
  ODE_DUFFING_LYAPUNOV = 4
};

/* Schemes (Sec. 3, Sec. 6.4): classic fixed-step RK4 and the adaptive
 * Runge-Kutta-Cash-Karp 4(5) pair (fifth-order solution propagated). */
enum ode_scheme { ODE_RK4 = 0, ODE_RKCK45 = 1 };

/* Precision: ODE_FP64 evaluates everything in binary64.  ODE_FP32_RHS
 * evaluates the right-hand-side stages in binary32 (stage states, f, and the
 * weighted stage sums of the update and of the embedded error estimate) and
 * keeps the state, time, the state update y + h * sum, the error estimate's
 * scaling and norm, the step-size controller and event location in binary64.
 * Available for ODE_DUFFING, ODE_VALVE and ODE_BOUNCE (not Keller-Miksis). */
enum ode_prec { ODE_FP64 = 0, ODE_FP32_RHS = 1 };

/* CopyModePossibilities of Sec. 6.3, as bit flags. */
enum ode_copy { ODE_TIMEDOMAIN = 1, ODE_STATE = 2, ODE_PARAM = 4, ODE_ACC = 8, ODE_ALL = 15 };

enum ode_ptr { ODE_PTR_HOST = 0, ODE_PTR_DEVICE = 1 };

/* Time-domain update done by the Finalization hook at the end of a slice
 * (Sec. 6.8):  KEEP leaves (t0, t1) unchanged (the next slice starts again at
 * t0, as the Duffing Poincare loop of Sec. 7.1.1 does); T0_TO_T sets t0 to
 * the end time (the listing of Sec. 6.8); SHIFT sets t0 to the end time and
 * t1 = t0 + (old t1 - old t0). */
enum ode_td_mode { ODE_TD_KEEP = 0, ODE_TD_T0_TO_T = 1, ODE_TD_SHIFT = 2 };

/* Why the last slice of a system ended. */
enum ode_sys_status {
    ODE_ST_NONE = 0,        /* not integrated yet */
    ODE_ST_TEND = 1,        /* reached t1 */
    ODE_ST_EVENT_STOP = 2,  /* EventStopCondition reached (Sec. 6.6) */
    ODE_ST_EQUILIBRIUM = 3, /* MaximumIterationForEquilibrium steps inside a zone (Sec. 4) */
    ODE_ST_HMIN_NAN = 4,    /* non-finite step at the minimum step size (Sec. 6.5) */
    ODE_ST_STEP_BUDGET = 5, /* per-slice step budget exhausted */
    ODE_ST_TIMEOUT = 6      /* stopped by the launch watchdog (ode_set_time_limit) */
};

enum ode_error {
    ODE_OK = 0,
    ODE_ERR_INVALID_ARG = -1,
    ODE_ERR_OUT_OF_MEMORY = -2,
    ODE_ERR_CUDA = -3,
    ODE_ERR_NOT_READY = -4,
    ODE_ERR_TIMEOUT = -5,
    ODE_ERR_UNSUPPORTED = -6
};

/* ---- solver object (Sec. 6.2) ------------------------------------------ */

/* Create a solver for `n_systems` (N_T, >= 1) systems of `model`, integrated
 * with `scheme` in precision `prec`, on CUDA device `device`.  Allocates the
 * device arrays (time domain 2N, state nN, parameters PN, accessories AN,
 * status, event counters EN and step counters) and zero-fills them.  The
 * dimensions n, P, A, E are fixed by the model (Sec. 6.2's configuration).
 * Errors: INVALID_ARG (bad enum, N < 1, FP32_RHS with Keller-Miksis),
 * OUT_OF_MEMORY, CUDA.  *out is NULL on failure. */
int ode_create(ode_solver **out, int model, int scheme, int prec, int n_systems, int device);

/* Free the solver and its device memory (waits for its outstanding work).
 * NULL is accepted. */
int ode_destroy(ode_solver *s);

/* Dimensions: state n (N_sys), parameters P (N_par), events E (N_E),
 * accessories A (N_A) per system; any pointer may be NULL. */
int ode_query_dims(const ode_solver *s, int *n_sys, int *n_par, int *n_evt, int *n_acc);
int ode_num_systems(const ode_solver *s, int *n_systems);

/* ---- properties (Sec. 6.5, 6.6) ----------------------------------------- */

/* OdeProperties: per-component relative and absolute tolerances (host arrays
 * of n doubles), maximum and minimum step, TimeStepGrowLimit and
 * TimeStepShrinkLimit.  Defaults are those printed in Sec. 6.5: 1e-10, 1e-10,
 * 1e6, 1e-12, 5, 0.1.  Requires 0 < h_min <= h_max < inf,
 * 1 <= grow <= 1e4, 1e-4 <= shrink <= 1, tolerances finite and >= 0 with
 * atol_i + rtol_i > 0.  Ignored by RK4. */
int ode_set_tolerances(ode_solver *s, const double *rtol, const double *atol, double h_max,
                       double h_min, double grow_limit, double shrink_limit);

/* EventProperties: enable (1) or disable (0) the model's event functions; per
 * event (host arrays of E) the direction (-1, 0, +1, MATLAB rule), the
 * absolute tolerance of the event zone (>= 0) and the stop count (0 = never,
 * n = stop at the n-th detection in a slice); MaximumIterationForEquilibrium
 * (0 = off).  Arrays may be NULL when enabled = 0.  Defaults: disabled, dir
 * -1, tol 1e-6, stop 0 (valve: stop (1, 0), equilibrium 50, Sec. 6.6). */
int ode_set_events(ode_solver *s, int enabled, const int *direction, const double *tolerance,
                   const int *stop_count, int max_steps_in_zone);

/* Solver-wide model constants (host array, nc <= 8 doubles).  Duffing and
 * Duffing-Lyapunov: (delta, c3, omega).  Other models take none (nc = 0). */
int ode_set_model_constants(ode_solver *s, const double *c, int nc);

/* Finalization time-domain update (enum ode_td_mode). */
int ode_set_time_domain_mode(ode_solver *s, int mode);

/* Per-slice step budget (accepted + rejected trial steps); default 1e9. */
int ode_set_step_budget(ode_solver *s, long long max_steps_per_slice);

/* Watchdog: a thread that runs longer than `seconds` within one launch stops
 * its system with status ODE_ST_TIMEOUT and takes no further work, and the
 * next synchronizing call (ode_synchronize, ode_run_periods with host
 * records, ode_get_status with host arrays) returns ODE_ERR_TIMEOUT.
 * Default 600 s; 0 disables it.  It bounds the run time of every launch. */
int ode_set_time_limit(ode_solver *s, double seconds);

/* Launch shape: block_size (multiple of 32 in [32, 256], 0 = automatic) and
 * persistent: 0 = one thread per system, grid ceil(N / block_size), the
 * launch of Sec. 6.4; 1 or 2 = a persistent grid (resident blocks x SMs)
 * whose threads refill their slot from a device work queue the moment their
 * system finishes.  Queue order 1: warp-aggregated pops of 32 consecutive
 * systems, chunks handed out in a stride order that spreads consecutive pops
 * over the index range (a warp holds neighbouring systems, SMs get a mix of
 * the sweep); order 2: each thread takes the next system in index order.
 * Results do not depend on the shape. */
int ode_set_launch(ode_solver *s, int block_size, int persistent);

/* Work split of a launch (no counterpart in the paper, whose launch gives
 * every thread one system and runs one Solve per launch, Sec. 6.4):
 * systems_per_thread in [1, 64] for the per-sweep launch (thread g of G takes
 * systems g, g + G, g + 2G, ... one after another; the persistent launches
 * ignore it), slices_per_launch >= 0 for ode_run_periods (the run is split
 * into launches of that many slices, each launch storing and reloading the
 * whole state; 0 = all slices in one launch), and warp_sync 0 or 1 (1: a
 * thread whose slice has ended waits until every thread of its warp has
 * ended its slice, and they start the next one together, so that the threads
 * of a warp do not drift apart over many slices).  Results do not depend on
 * any of them.  Defaults 1, 0, 0. */
int ode_set_schedule(ode_solver *s, int systems_per_thread, int slices_per_launch, int warp_sync);

/* ---- filling and reading the object (Sec. 6.3, 6.10) --------------------- */

/* LinearSet: copy `count` consecutive systems from a pool of `pool_size`
 * systems, pool index start_pool + i -> object index start_obj + i, for the
 * arrays selected by copy_mode (ODE_TIMEDOMAIN: td[2][pool_size], ODE_STATE:
 * y[n][pool_size], ODE_PARAM: p[P][pool_size], ODE_ACC: acc[A][pool_size]).
 * Unselected arrays may be NULL.  Errors: INVALID_ARG for ranges outside
 * [0, N) or [0, pool_size), NULL selected arrays; CUDA. */
int ode_linear_set(ode_solver *s, int start_obj, int start_pool, int pool_size, int count,
                   const double *td, const double *y, const double *p, const double *acc,
                   int copy_mode, int ptr_kind, void *stream);

/* RandomSet: as ode_linear_set for scattered systems: idx_obj[i] <- idx_pool[i]
 * for i < count.  The index arrays live in the same memory kind as the data.
 * Indices are checked on the host for ODE_PTR_HOST; device indices must be
 * in range (out-of-range device indices are skipped by the copy kernel). */
int ode_random_set(ode_solver *s, const int *idx_obj, const int *idx_pool, int pool_size, int count,
                   const double *td, const double *y, const double *p, const double *acc,
                   int copy_mode, int ptr_kind, void *stream);

/* LinearGet / RandomGet: the reverse copies, object -> pool (the read-back
 * that Sec. 6.10 does through the public h_* arrays). */
int ode_linear_get(ode_solver *s, int start_obj, int start_pool, int pool_size, int count,
                   double *td, double *y, double *p, double *acc, int copy_mode, int ptr_kind,
                   void *stream);
int ode_random_get(ode_solver *s, const int *idx_obj, const int *idx_pool, int pool_size, int count,
                   double *td, double *y, double *p, double *acc, int copy_mode, int ptr_kind,
                   void *stream);

/* ---- integration (Sec. 6.4, Sec. 7.1.1) ---------------------------------- */

/* Solve: integrate every system over its own time domain [t0, t1] once (one
 * slice), starting with step h0 (RKCK45) or with the fixed step
 * (t1 - t0) / ceil((t1 - t0) / h0) (RK4).  Asynchronous on `stream`.
 * h0 > 0 required. */
int ode_solve(ode_solver *s, double h0, void *stream);

/* The iterated Solve of Sec. 7.1.1 in ONE kernel: n_transient + n_record
 * consecutive slices per system, each slice starting with step h0 and ending
 * with the Finalization time-domain update; after each of the last n_record
 * slices a record of R = A + n + 1 doubles per system is written:
 *   records[((r * R) + c) * N + i], c < A: accessories, c = A .. A+n-1: the
 *   state at the slice end (the Poincare point), c = A + n: the end time.
 * records may be NULL (no record written); with ODE_PTR_HOST the records are
 * staged in a solver-owned device buffer and copied back before return.
 * Step counters (accepted, rejected) accumulate; status and event counters
 * describe the last slice. */
int ode_run_periods(ode_solver *s, double h0, int n_transient, int n_record, double *records,
                    int ptr_kind, void *stream);

/* Autotuner: integrate n_slices slices from the current state with every
 * launch shape of a fixed candidate list -- block size 64, 96, 128, 160,
 * 192, 256 for each of four forms: per-sweep with 1 and with 2 systems per
 * thread, persistent with queue order 1 and 2 (shapes the kernel cannot
 * launch are skipped) -- then every form at its fastest block size with
 * warp-synchronous slices, and the fastest shape of the first search with
 * the slices split into launches of 1 and of ceil(n_slices / 2) slices; every
 * trial is timed with CUDA events on `stream` and starts from the same saved
 * state, which is restored at the end (state, status and counters).  The
 * fastest of all trials is kept (as ode_set_launch and ode_set_schedule would
 * set it).  Outputs (may be NULL): block size, persistent value, systems per
 * thread, slices per launch (0 = all), warp_sync, and trial_ms[32] =
 * milliseconds per trial: [form][block] for the 4 x 6 shapes in the order
 * above; then for the fastest of those: [1 slice per launch, ceil(n_slices /
 * 2) per launch, all in one launch, all with warp-synchronous slices]; then
 * [form] with warp-synchronous slices at that form's fastest block (-1 for
 * skipped trials).  Allocates a temporary copy of the state.  Synchronous. */
int ode_autotune(ode_solver *s, double h0, int n_slices, void *stream, int *block_size,
                 int *persistent, int *systems_per_thread, int *slices_per_launch, int *warp_sync,
                 double *trial_ms);

/* Wait for all work this solver enqueued. */
int ode_synchronize(ode_solver *s);

/* Per-system results: status (N ints), accepted and rejected step counts
 * (N long long each), event counters of the last slice (E*N ints,
 * [event][system]).  Any pointer may be NULL.  Synchronous for host arrays. */
int ode_get_status(ode_solver *s, int *status, long long *accepted, long long *rejected,
                   int *event_counts, int ptr_kind, void *stream);

/* Reset accepted / rejected step counters to zero. */
int ode_reset_counters(ode_solver *s, void *stream);

const char *ode_last_error(const ode_solver *s);

/* ---- helpers ------------------------------------------------------------- */

/* Keller-Miksis coefficients C0..C12, Eqs. (16)-(28), from physical
 * parameters in SI units (omega in rad/s); C must hold 13 doubles.  C8 uses
 * omega_2 (Eq. (24) prints omega_1, but the derivative of P_A2 sin(omega_2 t)
 * gives omega_2; only omega_2 agrees with the dimensional equation).  Pure
 * host computation. */
int ode_km_coefficients(double PA1, double PA2, double omega1, double omega2, double theta,
                        double RE, double Pinf, double pV, double sigma, double mu, double rho,
                        double cL, double gamma, double *C);

/* Clustering order (Sec. 7.2: threads of a warp should integrate systems of
 * similar parameters, which need similar numbers of steps).  keys: host array
 * [K][N] (component-major, K in 1..8) of the quantities that govern the step
 * counts, e.g. the swept parameters.  perm: host array of N ints that
 * receives a permutation of 0..N-1 visiting the systems along a Z-order
 * (Morton) curve of the keys, each scaled to [0, 1] over its finite range
 * and quantized to floor(63 / K) bits (at most 31); keys with no spread are
 * ignored, systems with a non-finite key come last, ties keep index order.
 * Load system perm[i] into slot i (e.g. ode_random_set) so that neighbouring
 * slots -- one warp, and consecutive pops of the persistent work queue --
 * hold neighbouring parameter points.  Pure host computation; the paper has
 * no such call (it leaves the ordering to the user). */
int ode_cluster_order(const double *keys, int K, int N, int *perm);

/* Kernel resources of one (model, scheme, prec, persistent) instantiation:
 * registers per thread, local (spill) bytes per thread, and the resident
 * blocks per SM at the given block size.  Any output may be NULL. */
int ode_kernel_info(int model, int scheme, int prec, int persistent, int block_size, int device,
                    int *regs, int *local_bytes, int *blocks_per_sm);

/* Measured FMA throughput of the device: dependent-chain DFMA and FFMA
 * microkernels over every SM (FMA per second; one FMA = 2 flops).  Used as
 * the roofline peak of the arithmetic-bound integrators. */
int ode_probe_fma_peak(int device, double *dfma_per_s, double *ffma_per_s);

/* Measured cost of one binary64 cos(), pow() and sqrt() call, in DFMA
 * equivalents (call throughput relative to the DFMA issue rate, with the loop
 * overhead subtracted).  Used to count the transcendental calls of an
 * algorithm in the FMA-peak roofline.  Any output may be NULL. */
int ode_probe_call_cost(int device, double *cos_dfma, double *pow_dfma, double *sqrt_dfma);

/* Settings of ode_run_periods_noalloc (host memory, read during the call).
 * rtol / atol: first n entries used; direction / tolerance / stop_count:
 * first E entries used (E, n of the model, see enum ode_model); the meaning
 * and limits of every field are those of ode_set_tolerances, ode_set_events,
 * ode_set_model_constants (unused entries 0), ode_set_time_domain_mode,
 * ode_set_step_budget and ode_set_time_limit. */
typedef struct ode_noalloc_settings {
    int model, scheme, prec;
    double rtol[4], atol[4];
    double h_max, h_min, grow_limit, shrink_limit;
    int events_enabled;
    int direction[2];
    double tolerance[2];
    int stop_count[2];
    int max_steps_in_zone;
    int time_domain_mode;
    long long max_steps_per_slice;
    double time_limit_s;
    double model_constants[8];
} ode_noalloc_settings;

/* ---- serving: continuous batching of sweep requests (not in the paper) ---- */

/* A request loop for parameter-sweep requests of uneven size, model and
 * horizon.  Each served model has a resident pool of `capacity` system slots
 * in HBM (the pools together must fit in the server's HBM budget: admission
 * by footprint).  A request of n systems and n_periods periods waits (FIFO per
 * model) until a contiguous range of n free slots exists, is then copied into
 * it and stays resident there.  Its systems are merged into ONE persistent
 * launch per model (a resident serving kernel whose threads take systems from
 * a ring of slot indices that the host keeps filling while the kernel runs):
 * a thread that finishes a system takes the next one at once, whatever
 * request it belongs to, so requests that arrive while others run share the
 * same launch.  Systems of different requests are published to the ring in
 * round-robin chunks, so a small request is not queued behind a large one.
 * The GPU is split between models with work (max-min fair shares of the SMs);
 * a model that gets work while others hold the GPU has them stop at their
 * next slice boundary and relaunch with the new split.  When all n systems of
 * a request are done its results are copied out asynchronously; its slots
 * are reused once that copy has completed.  A request's results are those of
 * ode_run_periods with n_transient = n_periods - 1, n_record = 1 (same
 * per-system arithmetic, restarted per slice), alone or in any mix.
 * The caller drives the loop with ode_server_progress (non-blocking). */
typedef struct ode_server ode_server;

/* device, HBM budget for the pools (bytes), and the residency quantum
 * slice_periods: 0 = a thread keeps a system for its whole horizon; k >= 1 =
 * a system goes back to the ring after k slices (time slicing between the
 * systems waiting for threads; results are the same either way). */
int ode_server_create(ode_server **out, int device, long long hbm_budget_bytes, int slice_periods);

/* Serve a model with the settings of ode_run_periods_noalloc (the settings'
 * model / scheme / precision select the kernel), initial step h0 and a pool of
 * `capacity` slots.  Errors: INVALID_ARG, OUT_OF_MEMORY (pool beyond the
 * budget), CUDA. */
int ode_server_add_model(ode_server *s, const ode_noalloc_settings *settings, double h0, int capacity);

/* Queue a request: host arrays td [2][n], y0 [n_sys][n], p [P][n] (copied
 * before return).  *ticket identifies it.  n must not exceed the pool. */
int ode_server_submit(ode_server *s, int model, int n_systems, int n_periods, const double *td,
                      const double *y0, const double *p, long long *ticket);

/* One non-blocking pass of the loop: read the last snapshot of the done
 * counters and yielded systems (finished requests are copied out), admit
 * waiting requests, publish systems to the rings, start, grow or rebalance the
 * serving kernels, and start the next snapshot.  Outputs the numbers of
 * resident and waiting requests (may be NULL). */
int ode_server_progress(ode_server *s, int *n_running, int *n_waiting);

/* State of a request: 0 waiting, 1 running, 2 done. */
int ode_server_poll(ode_server *s, long long ticket, int *state);

/* Results of a finished request (host arrays, any may be NULL): td [2][n],
 * y [n_sys][n], accessories of its last period [A][n], status [n], accepted
 * steps [n], and its latency (submit to results on the host, seconds).
 * Releases the ticket.  NOT_READY if the request has not finished. */
int ode_server_result(ode_server *s, long long ticket, double *td, double *y, double *acc,
                      int *status, long long *accepted, double *latency_s);

/* Counters of one served model (out[8]): serving-kernel instances started,
 * stop requests (rebalancing), systems taken back from the yield list,
 * snapshots read, ring entries published, requests copied out, flags seen
 * (1 watchdog stop, 2 an entry outside the pool), systems not yet counted. */
int ode_server_stats(const ode_server *s, int model, long long *out);

/* Stop the serving kernels at their next slice boundary, wait for them and
 * free everything (unfinished requests are dropped). */
int ode_server_destroy(ode_server *s);
const char *ode_server_last_error(const ode_server *s);

/* ---- integration without allocation ---------------------------------------- */

/* The paper has no counterpart to this call; it exists for callers that
 * cannot allocate device memory themselves or through the library: code whose
 * device memory is owned by another allocator's pool (a framework caching
 * allocator, where a raw cudaMalloc beside the pool fragments memory and may
 * fail unpredictably), and latency-bound loops that cannot afford the implicit
 * device synchronisation of cudaMalloc / cudaFree.
 *
 * It does what ode_run_periods does on a persistent launch -- n_transient +
 * n_record consecutive slices of every system in one kernel, records written
 * after each of the last n_record slices -- without a solver object and
 * without allocating: td [2][N], y [n][N], p [P][N], acc [A][N] (read and
 * updated in place) and records [n_record][A+n+1][N] (may be NULL) are the
 * caller's DEVICE arrays on `device`, laid out as in ode_run_periods.  The
 * kernel's other global memory (work-queue head, watchdog flag, per-system
 * stop status, event counters and step counters) is a fixed array inside the
 * library, reserved on every GPU that loads the library's device code and
 * kept until the process exits (1 835 264 bytes: a 256-byte header, then the
 * step counters, the status and the event counters, each section starting on
 * a 256-byte boundary so that every one is aligned for its type whatever
 * n_systems is); it holds at most 65536 systems, and larger n_systems are
 * rejected with ODE_ERR_INVALID_ARG, as are arrays not aligned for their
 * element type.  status [N] (int) and
 * accepted [N] (long long), device arrays or NULL, receive the stop status
 * and the accepted-step count of this call.
 *
 * The call only enqueues work on `stream` and calls no cudaMalloc, cudaFree
 * or other allocating routine.  Its first call on a device looks up the
 * array's device address (once per device); make that first call before any
 * stream capture.  Every call reuses the same array, which keeps the last
 * call's contents; the call clears what must start at zero.  Calls whose work
 * overlaps on the GPU (other streams, other host threads) race on the array
 * and must be serialised by the caller.  A watchdog stop shows as
 * ODE_ST_TIMEOUT in `status`.  Returns ODE_OK or an ODE_ERR_* code; *message
 * (if message is not NULL) points to a thread-local description of the last
 * failure of this call. */
int ode_run_periods_noalloc(const ode_noalloc_settings *settings, int n_systems, int device,
                            double h0, int n_transient, int n_record, double *td, double *y,
                            const double *p, double *acc, double *records, int *status,
                            long long *accepted, void *stream, const char **message);

#ifdef __cplusplus
}
#endif
#endif /* ODEGPU_H */

/*
 * ah.h -- C ABI of the GB300 lattice Abelian-Higgs library.
 *
 * The library evolves a periodic N^3 lattice of the U(1) Abelian-Higgs model
 * in conformal time with the staggered leapfrog of Correia & Martins,
 * arXiv:1809.00995 (Sec. 2, Eqs. up_pi, up_E, up_phi, up_A, with the
 * s-dependent couplings of Eq. 7 and the random-phase initial state), and
 * computes the network diagnostics of the same section (xi_L and <v^2>_X of
 * Eqs. defXiV2/defR, the winding length xi_W of Eq. 9, <v^2>_omega of
 * Eq. defEoS) plus the Gauss-law residual.  All compute runs in CUDA kernels
 * on one GPU (sm_103a); there is no CPU fallback.
 *
 * Conventions (all entry points):
 *  - Every call returns an ah_status (AH_OK = 0) and never aborts the
 *    process; ah_last_error() gives a thread-local message for the last
 *    failure on the calling thread.
 *  - Pointers are host pointers unless stated otherwise.  Output structs and
 *    buffers are owned by the caller; the library owns all device memory of a
 *    simulation and frees it in ah_destroy.
 *  - Lattice site (x, y, z), 0 <= x, y, z < N, has linear index
 *    x + N*(y + N*z) (x fastest); boundaries are periodic.
 *  - Field components, in this order wherever 10 of them are packed:
 *    0 phi.re, 1 phi.im, 2 Pi.re, 3 Pi.im, 4..6 theta_1..3, 7..9 E_1..3,
 *    where theta_i = e dx A_i is the phase of the link x -> x + k_i (Eq. 3)
 *    and E_i = d theta_i / d eta its conjugate.  At integer step n the state
 *    holds phi^n, theta^n, Pi^{n-1/2}, E^{n-1/2}.
 *  - Background: a(tau) = (tau / tau_ref)^alpha with alpha = 0, 1, 2 for
 *    Minkowski, radiation, matter; e = e0 a^(s-1), lambda = lambda0 a^(2(s-1))
 *    (Eq. 7); tau_n = tau0 + n dt.
 */
#ifndef AH_H
#define AH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum ah_status {
    AH_OK = 0,
    AH_ERR_ARG = 1,        /* invalid argument or configuration          */
    AH_ERR_OOM = 2,        /* device or host allocation failed           */
    AH_ERR_CUDA = 3,       /* a CUDA runtime call or launch failed       */
    AH_ERR_UNSTABLE = 4,   /* configuration violates leapfrog stability  */
    AH_ERR_NONFINITE = 5,  /* diagnostics found Inf/NaN in the state     */
    AH_ERR_TIMEOUT = 6,    /* a bounded device or host wait gave up      */
    AH_ERR_BUSY = 7,       /* resource in use (server full, call pending)*/
    AH_ERR_CANCELLED = 8,  /* request was cancelled                      */
    AH_ERR_NOTFOUND = 9    /* unknown request id                         */
} ah_status;

enum { AH_MINKOWSKI = 0, AH_RADIATION = 1, AH_MATTER = 2 };
enum { AH_FP32 = 0, AH_FP64 = 1 };
/* Kernel family for the leapfrog step.
 *  PLAIN: the paper's three-kernel structure (Pi kick, E kick, drift),
 *         one thread per site, all loads from global memory.
 *  FUSED: one z-marching kernel per step: both kicks and both drifts fused,
 *         shared-memory XY tiles, link exponentials computed once per site,
 *         ping-pong phi/theta buffers.
 *  AUTO:  FUSED. */
enum { AH_KERNEL_AUTO = 0, AH_KERNEL_PLAIN = 1, AH_KERNEL_FUSED = 2 };
/* Configuration flags.
 *  EXACT_DIAG: evaluate every diagnostic per site in FP64 with arctangent
 *  windings (slow).  By default per-site energies are evaluated in the state
 *  precision (accumulated in FP64), the Gauss residual in FP64, and windings by
 *  sign carries that equal the FP64 arctangent formula, with the plaquettes
 *  near a branch cut re-evaluated in FP64. */
enum { AH_FLAG_EXACT_DIAG = 1, AH_FLAG_AUTOTUNE = 2, AH_FLAG_WRAP_THETA = 4, AH_FLAG_CORE_GROWTH = 8,
       AH_FLAG_TWO_STEP = 16, AH_FLAG_FUSED_DIAG = 32 };
/* AUTOTUNE: at creation, time every compile-time shape of the fused step on
 * the initial state (then re-initialise it) and keep the fastest; results are
 * cached per (device, N, precision, two-step mode) for the life of the process.
 * WRAP_THETA: after every drift (Eq. up_A) a link phase with |theta| > pi is
 * replaced by theta - 2 pi k, k the nearest integer to theta / 2 pi, so that
 * theta stays in [-pi, pi] (to one rounding) and an FP32 state keeps its
 * absolute resolution on theta at late times.  U = e^{i theta}, the
 * plaquettes and every observable except max |theta| are unchanged up to
 * rounding; ah_get_fields returns the wrapped phases.  Without the flag theta
 * is non-compact (never wrapped), as in Eq. up_A.
 * CORE_GROWTH: the schedule of Sec. 2 that grows the comoving string width
 * first and then evolves the true equations: the exponent of Eq. 7 is s for
 * tau < tau_ref (s < 0 grows the width) and 1 from tau_ref on.  Since
 * a(tau_ref) = 1, e and lambda equal e0 and lambda0 on both sides of the
 * switch, so the couplings are continuous there.  Every coupling of a step
 * (at tau_n and tau_n +- dt/2) takes the exponent of its own time.
 * TWO_STEP (FP32, fused kernel only): ah_step advances pairs of steps with
 * one kernel pass each (temporal blocking: the state is read and written once
 * per two steps, 40 B per site-update instead of 80), and an odd last step
 * with the single-step kernel.  Each step evaluates the same formulas as a
 * single step; results agree to FP32 rounding (multiply-adds may be fused
 * differently).  Pi and E are then kept in two buffer sets (one read, one
 * written), so the state takes 20 instead of 15 arrays of N^3 reals; in this
 * mode ah_set_variant, ah_autotune and ah_info.variant / n_variants /
 * variant_name refer to the two-step shapes, and the TMA-fed single-step
 * shapes are not available.  Refused (AH_ERR_ARG) for FP64 and for
 * AH_KERNEL_PLAIN.
 * In this mode, while the last whole-lattice observables of the simulation
 * found max |theta| <= 2^-7 (weak gauge fields: early times, small scale
 * factors), the pairs run a kernel whose link exponentials take two-term
 * sine/cosine forms in warps whose phases are all within 2^-6 (within an ulp
 * of the general forms; ah_info.weak_field_launches counts those launches).
 * FUSED_DIAG (with TWO_STEP only, else AH_ERR_ARG): an asynchronous
 * observables pass (ah_observables_start) is always taken by the next
 * two-step launch, which reads the state of the pass for its first step
 * anyway (see ah_observables_start).  Without the flag a two-step simulation
 * chooses by the last whole-lattice observables it returned: the fused launch
 * when fewer than 1e-3 of the plaquettes were pierced (a string network in an
 * otherwise smooth field, where most tiles skip the winding carries), else a
 * separate pass.  No effect in batches and the server. */

typedef struct ah_config {
    int32_t N;            /* lattice side, 4 <= N <= 2048                         */
    int32_t era;          /* AH_MINKOWSKI, AH_RADIATION, AH_MATTER                 */
    int32_t precision;    /* AH_FP32 or AH_FP64 field state and stencil arithmetic */
    int32_t kernel;       /* AH_KERNEL_*                                           */
    double dx;            /* lattice spacing, > 0                                   */
    double dt;            /* time step, 0 < dt <= dx / sqrt(3) (Courant)            */
    double s;             /* coupling exponent of Eq. 7                             */
    double lambda0;       /* scalar self-coupling, >= 0                             */
    double e0;            /* gauge coupling, > 0                                    */
    double sigma;         /* vacuum expectation value, > 0                         */
    double tau0;          /* conformal time at step 0, > 0 unless Minkowski         */
    double tau_end;       /* end of the run (default N dx / 2, half light-crossing) */
    double tau_ref;       /* normalisation a(tau_ref) = 1 (default tau_end)         */
    uint64_t seed;        /* Philox-4x32-10 key of the random-phase initial state   */
    int32_t diag_every;   /* diagnostic cadence used by batch and serve (0: end only) */
    int32_t flags;        /* AH_FLAG_* bits                                        */
} ah_config;

/* Network observables at one integer step (Sec. 2).  sums[] are the raw FP64
 * site sums, in the order:
 *   0 L, 1 rho, 2 p, 3 K=|Pi|^2, 4 G2=|D phi|^2, 5 V, 6 E_el, 7 B_mag,
 *   8 K V, 9 G2 V, 10 K L, 11 G2 L, 12 p L, 13 rho L, 14 G^2, 15 scale^2
 * with, per site at tau_n,
 *   G2 = dx^-2 sum_i |e^{i theta_i} phi^{x+i} - phi^x|^2,
 *   V = a^2 lambda/4 (|phi|^2 - sigma^2)^2, E_el = sum_i E_i^2 / (2 e^2 a^2 dx^2),
 *   B_mag = sum_{i<j} (1 - cos Xi_ij) / (e^2 a^2 dx^4),
 *   L = K - G2 - V + E_el - B_mag, rho = K + G2 + V + E_el + B_mag,
 *   p = K - G2/3 - V + (E_el + B_mag)/3,
 *   G = e_-^-2 sum_i (E_i^x - E_i^{x-i}) + 2 dx^2 a_-^2 Im(conj(phi) Pi)
 *       (Gauss residual, a_- and e_- at tau_n - dt/2; scale = |term 1| + |term 2|).
 * Derived: xi_L = sqrt(-2 pi sigma^2 / L_mean); xi_W = sqrt(n_sites dx^3 / l_W)
 * with l_W = (pi/6) dx sum_abs_W; <v^2>_X = 2R_X/(1+R_X), R_V = sums[8]/sums[9],
 * R_L = sums[10]/sums[11]; v2_omega = (1 + 3 p_over_rho_L)/2 with
 * p_over_rho_L = sums[12]/sums[13]; energy = dx^3 sums[1].  Zero denominators
 * follow IEEE rules (Inf/NaN are reported, not trapped). */
typedef struct ah_obs {
    double tau, a;
    int64_t step;
    int64_t n_sites;
    double L_mean, xi_L, xi_W;
    int64_t n_pierced;           /* plaquettes with W != 0                     */
    int64_t sum_abs_W;           /* sum of |W| over all plaquettes             */
    double R_V, R_L, v2_V, v2_L, p_over_rho_L, v2_omega;
    double gauss_rms, gauss_max, gauss_rel, energy, max_abs_theta;
    double sums[16];
    int64_t wind_abs_plane[3];   /* sum |W| by orientation 12, 13, 23          */
    int64_t wind_plane[3];       /* signed sums by orientation                 */
    int64_t nonfinite;           /* sites whose L, rho, p or G is not finite   */
} ah_obs;

typedef struct ah_sim ah_sim;

/* Version of this ABI (bumped on any change of a struct or signature). */
int ah_abi_version(void);

/* Fill *cfg with the defaults for an N^3 lattice: FP32, radiation era, s = 0,
 * lambda0 = 2, e0 = 1, sigma = 1, dx = 0.5, dt = 0.1, tau0 = 1,
 * tau_end = N dx / 2, tau_ref = tau_end, seed 1, kernel AUTO. */
void ah_config_default(ah_config *cfg, int32_t N);

/* Create a simulation with the defaults above, overriding N, dx, dt, era, s,
 * lambda0, e0 and seed; initial state: phi = sigma e^{i 2 pi u}, u from
 * Philox-4x32-10 (key = seed, counter = (0, 0, site index)), Pi = theta = E = 0
 * (Sec. 2).  Returns NULL on error (see ah_last_error). */
ah_sim *ah_create(int32_t N, double dx, double dt, int32_t era, double s,
                  double lambda0, double e0, uint64_t seed);

/* Create from a full configuration.  Validates the arguments (AH_ERR_ARG),
 * rejects with AH_ERR_UNSTABLE a configuration whose stiffest mode breaks
 * leapfrog stability, dt^2 (12/dx^2 + max(lambda0, 2 e0^2) sigma^2 a^(2s)) >= 3.6
 * for the largest a^(2s) over the run (over both stretches of a core-growth
 * schedule), allocates the state on the current CUDA device (AH_ERR_OOM) and
 * writes the initial state.  *out receives the handle. */
ah_status ah_create_ex(const ah_config *cfg, ah_sim **out);

/* Enqueue nsteps leapfrog steps (Eqs. up_pi, up_E, up_phi, up_A) on the
 * simulation's stream; returns without waiting.  nsteps >= 0. */
ah_status ah_step(ah_sim *sim, int64_t nsteps);

/* Compute the observables of the current state over the whole lattice and
 * write them to *out (waits for the simulation's stream).  Per-site energies
 * are evaluated in the state precision and summed with compensation per thread
 * and in FP64 across threads; the Gauss residual in FP64 (double-float
 * arithmetic for an FP32 state); windings equal the FP64 arctangent formula of
 * Eq. 9 on the same snapshot.  With AH_FLAG_EXACT_DIAG everything per site is
 * FP64.  Returns AH_ERR_NONFINITE (with *out filled) if any site is not
 * finite. */
ah_status ah_observables(ah_sim *sim, ah_obs *out);

/* Same over the sub-box [x0, x0+nx) x [y0, y0+ny) x [z0, z0+nz), taken mod N
 * (plaquettes and differences still reach the neighbours outside the box). */
ah_status ah_observables_box(ah_sim *sim, int32_t x0, int32_t y0, int32_t z0,
                             int32_t nx, int32_t ny, int32_t nz, ah_obs *out);

/* Asynchronous observables of the current state (the quantities of
 * ah_observables, Sec. 2).  ah_observables_start enqueues the whole-lattice
 * diagnostics pass on a second stream of the simulation and returns without
 * waiting; the pass reads the state as it is at the call (the snapshot), and a
 * list overflow of near-cut plaquettes is settled on the device (all windings
 * counted again in FP64).  Later ah_step calls go on: each launch that would
 * overwrite the snapshot first waits for the pass; in two-step mode the first
 * two-step launch after the start writes the other buffer set and runs
 * alongside the pass.  A two-step simulation may instead defer the pass (see
 * AH_FLAG_FUSED_DIAG): then the next ah_step of two or more steps runs its
 * first two steps with the diagnostics of the snapshot folded in (one kernel
 * pass over the state instead of two; the steps are those of the plain
 * two-step pass, bit for bit), and the pass runs on its own if
 * ah_observables_finish, ah_set_fields or a single step comes first.  The sums
 * then differ from those of ah_observables by the summation order only (a few
 * 1e-7 relative); windings, max |G| and max |theta| are the same.
 * ah_observables_finish waits for the pass and fills *out for the step of the
 * snapshot (status as ah_observables).  One pass at a time per simulation: a
 * second start, ah_observables, ah_observables_box and ah_autotune return
 * AH_ERR_BUSY while one is pending; ah_set_fields and ah_set_stream wait for
 * it. */
ah_status ah_observables_start(ah_sim *sim);
ah_status ah_observables_finish(ah_sim *sim, ah_obs *out);

/* Copy the state of the window [x0, x0+nx) x ... (mod N) to host memory `out`
 * as FP64: 10 components, each nz*ny*nx with x fastest (10*nx*ny*nz doubles).
 * Waits for the simulation's stream. */
ah_status ah_get_fields(ah_sim *sim, int32_t x0, int32_t y0, int32_t z0,
                        int32_t nx, int32_t ny, int32_t nz, double *out);

/* Replace the whole state by host FP64 data `in` (10*N^3 doubles, layout as
 * above; rounded to the state precision) and set the step counter. */
ah_status ah_set_fields(ah_sim *sim, const double *in, int64_t step);

/* Use the given cudaStream_t (as void*; NULL = the library's own stream) for
 * all later work of this simulation. */
ah_status ah_set_stream(ah_sim *sim, void *cuda_stream);

/* Wait for all work enqueued for this simulation. */
ah_status ah_sync(ah_sim *sim);

/* Current integer step n and conformal time tau_n. */
int64_t ah_get_step(const ah_sim *sim);
double ah_get_tau(const ah_sim *sim);

/* Information for measurement: bytes of device state, the algorithmic bytes
 * one leapfrog step must move (one read and one write of the 10-component
 * state: 80 B per site in FP32, 160 B in FP64; in two-step mode a launch
 * advances two steps with one read and one write, so the DRAM bytes per step
 * are half of step_bytes), and the kernel in use. */
typedef struct ah_info {
    int64_t N, n_sites;
    int32_t precision, kernel;
    int64_t state_bytes;
    int64_t step_bytes;
    int64_t step_launches;   /* kernel launches per leapfrog step (in
                                two-step mode: per pair of steps)         */
    int32_t variant;         /* shape of the fused step in use             */
    int32_t n_variants;      /* shapes available for this precision        */
    char variant_name[32];
    int64_t fused_diag_passes;   /* observables passes taken by two-step
                                    launches so far (AH_FLAG_FUSED_DIAG)   */
    int64_t weak_field_launches; /* two-step launches so far that used the
                                    kernel for weak gauge fields (taken
                                    while the last whole-lattice observables
                                    found max |theta| <= 2^-7)             */
} ah_info;
ah_status ah_get_info(const ah_sim *sim, ah_info *out);

/* Number of shapes of the fused step for the given precision (tile size,
 * resident CTAs per SM, z-chunk rule; for FP32 also the paired-FP32 and the
 * TMA-fed kernels).  The names are in ah_info.variant_name. */
int32_t ah_variant_count(int32_t precision);

/* Select the fused-step shape for later steps (0 <= variant < count).  Every
 * shape computes the same update; they differ only in speed. */
ah_status ah_set_variant(ah_sim *sim, int32_t variant);

/* Time every fused-step shape for `trial_steps` steps on the freshly created
 * state, keep the fastest (written to *chosen if not NULL) and restore the
 * initial state.  Only valid before the first ah_step / ah_set_fields
 * (AH_ERR_BUSY otherwise).  Waits for the simulation's stream. */
ah_status ah_autotune(ah_sim *sim, int32_t trial_steps, int32_t *chosen);

/* ---- batched ensembles (the ensembles of independent runs of Sec. 4, Table 3) ----
 *
 * Many independent FP32 lattices (any mix of N, era, s, seed) advance together:
 * one persistent kernel launch per leapfrog step covers every resident lattice
 * (work items = lattice tiles), each lattice with its own coefficient table and
 * step counter on the device; the steps between diagnostic points are replayed
 * from a CUDA graph.  Every lattice computes exactly what ah_step computes for
 * it alone. */
/* Steps in pairs.  A lattice whose configuration has AH_FLAG_TWO_STEP, and,
 * with the batch (or server) flag AH_BATCH_TWO_STEP, every lattice of side
 * N >= 512, is advanced two steps per launch by the batched two-step pass
 * (temporal blocking, as AH_FLAG_TWO_STEP does for one simulation: the state
 * is read and written once per two steps), and by a single step only when one
 * step is left before its next diagnostic point or its end, so the grouping of
 * its steps, and its results, do not depend on the other lattices of the
 * batch.  Such a lattice holds a second Pi/E set (20 instead of 15 arrays of
 * N^3 floats); from side 512 on it is launched with its own two-step grid
 * (the rounds of such a batch then run without a CUDA graph).  Its results
 * agree with one step per launch to FP32 rounding.
 * The other lattices take one step per launch.  (Small lattices gain nothing
 * from pairs: the two-step tile writes 30 x 6 of its 32 x 8 sites.) */
enum { AH_BATCH_AUTOTUNE = 1, AH_BATCH_NO_GRAPH = 2, AH_BATCH_TWO_STEP = 4 };

typedef struct ah_batch_stats {
    double seconds;          /* wall time of the evolution and diagnostics       */
    double setup_seconds;    /* allocation, initial states, shape tuning         */
    double site_updates;     /* sum over lattices of N^3 x steps                 */
    double sims_per_hour;    /* count x 3600 / seconds                           */
    int32_t shape;           /* batched-kernel shape used (the two-step pass's
                                shape with AH_BATCH_TWO_STEP)                    */
    int32_t rounds;          /* graph (or launch-sequence) replays               */
    int64_t launches;        /* kernel launches of the batched steps             */
    int64_t weak_field_launches; /* two-step launches of paired lattices of side
                                >= 512 in the form for weak gauge fields (taken
                                while the lattice's last observables found
                                max |theta| <= 2^-7, as for ah_step)             */
} ah_batch_stats;

/* Run `count` lattices (cfgs[i]: precision AH_FP32, N <= 1290; each runs
 * round((tau_end - tau0)/dt) steps) to their ends.  If series is not NULL it
 * holds count x series_cap ah_obs (lattice-major): for lattice i, observables at
 * step 0, every cfgs[i].diag_every steps (if > 0) and at the end;
 * series_len[i] receives the number produced (entries past series_cap are
 * dropped).  flags: AH_BATCH_AUTOTUNE (time each batched shape on the initial
 * states, then restore them), AH_BATCH_NO_GRAPH (plain launches),
 * AH_BATCH_TWO_STEP (lattices of side >= 512 in pairs, see above).  stats may
 * be NULL.  Synchronous; all device memory is released before return.  Of the
 * per-lattice cfgs[i].flags, AH_FLAG_WRAP_THETA, AH_FLAG_CORE_GROWTH and
 * AH_FLAG_TWO_STEP (steps in pairs) apply; AH_FLAG_AUTOTUNE and
 * AH_FLAG_EXACT_DIAG have no effect (the diagnostics are those of the
 * whole-lattice pass).  The same holds for requests to the server. */
ah_status ah_batch_run(const ah_config *cfgs, int32_t count, int32_t flags, ah_obs *series,
                       int64_t series_cap, int64_t *series_len, ah_batch_stats *stats);

/* A window of a lattice's final state to copy to host memory: the sites
 * [x0, x0+nx) x [y0, y0+ny) x [z0, z0+nz) taken mod N (1 <= nx, ny, nz <= N),
 * written to `out` as FP64 in the layout of ah_get_fields (10 components of
 * nz*ny*nx values, x fastest).  `out` is caller-owned host memory. */
typedef struct ah_window {
    int32_t lattice;              /* ah_batch_run_ex: index into cfgs; ignored by the server */
    int32_t x0, y0, z0, nx, ny, nz;
    double *out;
} ah_window;

/* ah_batch_run, plus field read-back: after every lattice has reached its end,
 * each of the `nwindows` windows (any number per lattice) receives its
 * lattice's final state (phi^n, theta^n, Pi^{n-1/2}, E^{n-1/2} at its last step
 * n, the state the last entry of its series describes).  AH_ERR_ARG for a
 * window whose lattice index or extent is out of range or whose buffer is
 * NULL (checked before any work). */
ah_status ah_batch_run_ex(const ah_config *cfgs, int32_t count, int32_t flags, ah_obs *series,
                          int64_t series_cap, int64_t *series_len, ah_batch_stats *stats,
                          const ah_window *windows, int32_t nwindows);

/* ---- continuous-batching server ----
 *
 * A scheduler thread admits submitted requests (FIFO) whenever a slot is free
 * and the request's device memory fits the HBM budget, keeps every admitted
 * lattice resident, advances all of them together with the batched step in
 * rounds of at most 20 steps (so newly admitted work joins within a round), and
 * retires each lattice at its tau_end with its final observables.  Times are in
 * seconds since the server was created. */
typedef struct ah_server ah_server;
typedef struct ah_server_stats {
    int64_t submitted, admitted, completed;
    int32_t running, queued;
    int64_t hbm_used;        /* bytes held by resident lattices                  */
    double site_updates;     /* total site-updates performed                     */
    int64_t launches;        /* kernel launches of the batched steps             */
} ah_server_stats;

/* Start a server on the current device.  flags: AH_BATCH_NO_GRAPH,
 * AH_BATCH_TWO_STEP (requests of side >= 512 in pairs; a request stepped in
 * pairs takes 20 instead of 15 arrays of N^3 floats of the budget). */
ah_status ah_server_create(size_t hbm_budget_bytes, int32_t max_slots, int32_t flags, ah_server **out);
/* Queue one run (precision AH_FP32, N <= 1290); AH_ERR_OOM if it can never fit
 * the budget. */
ah_status ah_server_submit(ah_server *srv, const ah_config *cfg, uint64_t *req_id);
/* The same, plus windows of the run's final state (ah_window; `lattice` is
 * ignored) written when the run completes, before ah_server_poll reports it
 * done.  The buffers must stay valid until ah_server_poll returns AH_OK,
 * AH_ERR_CANCELLED or AH_ERR_CUDA for this request (a cancelled or failed run
 * may leave them unwritten). */
ah_status ah_server_submit_ex(ah_server *srv, const ah_config *cfg, const ah_window *windows,
                              int32_t nwindows, uint64_t *req_id);
/* AH_OK with the final observables and times once done; AH_ERR_BUSY while queued
 * or running; AH_ERR_CANCELLED, AH_ERR_NOTFOUND, AH_ERR_CUDA (failed run). */
ah_status ah_server_poll(ah_server *srv, uint64_t req_id, ah_obs *final_out, double *t_submit,
                         double *t_done);
/* Drop a queued or running request (its memory is released by the scheduler). */
ah_status ah_server_cancel(ah_server *srv, uint64_t req_id);
ah_status ah_server_stats_get(ah_server *srv, ah_server_stats *out);
/* Stop the scheduler (running requests are abandoned) and free everything. */
void ah_server_destroy(ah_server *srv);

/* Raw diagnostic sums as written by ah_observables_noalloc (208 bytes):
 * sums[] in the order of ah_obs.sums, then max |G|, max |theta|, sum |W| by
 * plaquette orientation (12, 13, 23), signed sums by orientation, the number of
 * plaquettes with W != 0 and the number of non-finite sites. */
typedef struct ah_sums {
    double sums[16];
    double gauss_max, max_abs_theta;
    int64_t wind_abs_plane[3];
    int64_t wind_plane[3];
    int64_t n_pierced;
    int64_t nonfinite;
} ah_sums;

/* Diagnostics of an FP32 state held in caller-owned device memory, with no
 * device allocation of any kind.  The paper has no counterpart: this exists for
 * callers that cannot call cudaMalloc -- a host framework that owns the whole
 * device memory pool through its own allocator, loops that must not block on
 * the driver's allocator once running, or a sandbox that forbids new device
 * allocations after start-up.
 *
 *  fields   10 device pointers (component order above), each N^3 floats with x
 *           fastest, 8-byte aligned; read only.
 *  N, cfg   lattice side (must equal cfg->N; 4 <= N <= 2048) and the run's
 *           configuration (cfg->precision must be AH_FP32; the couplings and
 *           the scale factor at integer step `step` come from it).
 *  d_sums   caller-owned device memory for one ah_sums (8-byte aligned),
 *           written by the call.
 *  stream   cudaStream_t (as void*) the work is enqueued on; the call returns
 *           without waiting, so read d_sums after synchronising that stream.
 * The per-site values and the sums are the same as those of ah_observables
 * (fast path: FP32 energies, FP64 sums and Gauss residual, windings equal to the
 * FP64 arctangent formula).  Scratch memory -- per-block partial sums and a list
 * of at most 2^18 plaquettes near a branch cut -- lives in one static device
 * array of 2.31 MB that every GPU which loads the library holds until exit; if
 * a snapshot has more listed plaquettes than that, all windings of the call are
 * recounted in FP64 (slower, same result).  About 5e-5 of the 3 N^3 plaquettes
 * of a random-phase state (such as the initial one) are listed, so above
 * N ~ 1200 the recount is the expected path for such states.  The first call on a device looks up
 * that array's address (a one-time set-up): make the first call before any
 * stream capture.  All calls share the array, so calls whose work overlaps on
 * the GPU (concurrent streams or threads) race and give wrong sums: serialise
 * them.  Sizes out of range are rejected with AH_ERR_ARG. */
ah_status ah_observables_noalloc(const float *const fields[10], int32_t N, const ah_config *cfg,
                                 int64_t step, void *d_sums, void *cuda_stream);

/* Free all resources of the simulation (NULL-safe). */
void ah_destroy(ah_sim *sim);

/* Message for the last failed call on this thread ("" if none). */
const char *ah_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* AH_H */

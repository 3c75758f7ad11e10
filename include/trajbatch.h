/*
 * trajbatch.h -- C ABI of the B300 batched trajectory optimizer.
 *
 * The library solves, for a batch of trajectories, the alternating-
 * minimization (AM) problem of Rastgar's thesis, Paper II: each trajectory is
 * a set of degree-10 Bernstein coefficients per axis (eq. parameter), the
 * collision, velocity and acceleration constraints are written in
 * polar/spherical form with auxiliary angle and distance variables (eqs.
 * collision_1, fv, fa; 3D eqs. collision_priest, fv_priest, fa_priest), and
 * each iteration of Algorithm 2 performs
 *   Line 2  the batched QP step through a KKT inverse cached per problem
 *           (eqs. zeta_1_sepration_1, zeta_1_sepration_3, over_3),
 *   Lines 4-5 the closed-form alpha/beta/d projections over every
 *           trajectory x obstacle x timestep (eqs. zeta_2, alpha_v, alpha_a,
 *           compute_d_mij, compute_dv, compute_da, d_max),
 *   Line 6  the multiplier update lambda <- lambda - rho F^T (F xi - g)
 *           (eq. update_lambda2_1; PRIEST eq. lag).
 * The projection cost of Paper III (eqs. projection_cost, affine_trans,
 * matrix_vec) is the TRAJ_COST_PROJECT mode.
 *
 * Conventions shared by every entry point:
 *  - Return codes only: nothing aborts, exits or throws across the ABI. A NULL
 *    handle or pointer that is required gives TRAJ_EINVAL. The detail of the
 *    last failure on a handle is available from traj_last_error().
 *  - Arrays are dense, C order, FP32 unless stated. "Host or device" pointers
 *    are classified with cudaPointerGetAttributes; host data is staged through
 *    pinned memory and copied on the handle's stream.
 *  - One handle per CUDA stream; a handle is not thread-safe. All GPU work of a
 *    handle runs on the stream given at creation (cudaStream_t passed as
 *    void*; NULL is the legacy default stream).
 *  - The library owns its device workspace (allocated at creation from the
 *    max_* sizes and released by traj_batch_destroy); the caller owns every
 *    array it passes in or gets results into.
 *  - The library never falls back to a CPU implementation: without a CUDA
 *    device every call that needs one returns TRAJ_ECUDA.
 */
#ifndef TRAJBATCH_H
#define TRAJBATCH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TRAJ_OK = 0,
  TRAJ_NOT_CONVERGED = 1, /* solve finished; some trajectory hit the iteration cap */
  TRAJ_EINVAL = -1,       /* bad argument (NULL handle/pointer, size out of range) */
  TRAJ_ENOMEM = -2,       /* device or pinned allocation failed */
  TRAJ_ECUDA = -3,        /* a CUDA call failed; traj_last_error has its string */
  TRAJ_ESHAPE = -4,       /* inputs do not fit the capacities given at creation */
  TRAJ_ETIMEOUT = -5,     /* the solve's deadline passed; trajectories left are marked */
  TRAJ_ENAN = -6,         /* a non-finite input; the affected trajectories are marked */
  TRAJ_ESTATE = -7        /* call out of order (e.g. solve before set_initial) */
} traj_status;

/* Per-trajectory outcome written by traj_get_trajectories (int8). */
enum {
  TRAJ_TRAJ_CONVERGED = 0, /* all three residuals <= tol */
  TRAJ_TRAJ_CAP = 1,       /* iteration cap reached */
  TRAJ_TRAJ_NAN = 2,       /* non-finite input coefficients or obstacle data; skipped */
  TRAJ_TRAJ_TIMEOUT = 3    /* stopped by the deadline */
};

typedef enum {
  TRAJ_PREC_FP32 = 0, /* FP32 state and contractions; compensated FP32 QP step */
  TRAJ_PREC_MIXED = 1, /* residual contraction F^T r on tcgen05 tensor cores (BF16 operands,
                          FP32 accumulation in TMEM) plus one FP32 refinement pass when the
                          residuals first meet the tolerance (the refined iterate must meet it
                          too; it may add one iteration past the cap); residuals are always
                          FP32. Horizons up to 256 grid points, at most 16 distinct ones per
                          batch (uneven batches run in one launch). */
  TRAJ_PREC_MIXED_SPLIT = 2 /* as TRAJ_PREC_MIXED with both operands split into BF16 hi/lo
                               pairs (16 significant bits each): the basis's lo part doubles
                               the MMAs, the residual's rides in spare rows of the same MMA */
} traj_precision;

typedef enum {
  TRAJ_COST_SMOOTH_TRACK = 0, /* Q = w_s Pdd^T Pdd + w_t P^T P, q = -w_t P^T x_des
                                 (eq. Q_matrix); x_des the constant-velocity line */
  TRAJ_COST_PROJECT = 1       /* Q = I, q = -xi_sample (eq. matrix_vec): project each
                                 initial coefficient set onto the feasible set */
} traj_cost_mode;

typedef struct traj_config {
  int dim;           /* 2 or 3 */
  int degree;        /* Bernstein degree; must be 10 */
  int max_problems;  /* capacity: problems (scenes) */
  int max_traj;      /* capacity: trajectories */
  int max_obstacles; /* capacity: obstacles summed over problems */
  int max_steps;     /* capacity: timesteps n_p of any problem (<= 1024; above 256
                      * the FP32 form only) */
  double vmax, amax; /* velocity / acceleration bounds (eqs. fv, fa) */
  double rho;        /* penalty weight (one rho for every constraint group) */
  double w_smooth, w_track; /* cost weights of TRAJ_COST_SMOOTH_TRACK */
  int precision;     /* traj_precision */
  int cost_mode;     /* traj_cost_mode */
  void *cuda_stream; /* cudaStream_t on which every kernel and copy of the handle runs */
} traj_config;

typedef struct traj_batch traj_batch; /* opaque; owns the device workspace */

/* Create a handle. Validates the config (dim in {2,3}, degree 10, positive
 * capacities, max_steps <= 1024, vmax/amax/rho > 0) and allocates the
 * workspace on the stream. *out is set only on TRAJ_OK. */
traj_status traj_batch_create(const traj_config *cfg, traj_batch **out);

/* Synchronise the handle's stream and free everything it owns. NULL is a no-op. */
traj_status traj_batch_destroy(traj_batch *b);

/* Problem descriptions (host pointers, copied): n_steps[n_problems] timesteps
 * n_p >= 2 (grid tau_t = t/(n_p-1)), duration[n_problems] horizon T > 0 in
 * seconds, start[n_problems][dim] and goal[n_problems][dim] positions (FP64).
 * The boundary rows are start position, zero start velocity and acceleration,
 * and the goal position (PRIEST eq. eq1_multiagent_1_priest); traj_shift_horizon
 * later gives the start a velocity and an acceleration. */
traj_status traj_set_problems(traj_batch *b, int n_problems, const int *n_steps,
                              const double *duration, const double *start, const double *goal);

/* Obstacles of every problem as moving axis-aligned ellipses/ellipsoids with
 * constant velocity: obstacle j of problem p has index offsets[p] + j,
 * offsets[n_problems] = total (host int array, n_problems + 1 entries).
 * centers[N][dim] (at t = 0), semi_axes[N][dim] (> 0), velocities[N][dim];
 * FP32, host or device. Copied on the stream, then the FP64 set-up kernel
 * forms and inverts every problem's KKT matrix (eq. over_2) on the GPU. */
traj_status traj_set_obstacles(traj_batch *b, const int *offsets, const float *centers,
                               const float *semi_axes, const float *velocities);

/* Trajectories: traj_problem[n_traj] (host int) maps each trajectory to its
 * problem; coeffs0[n_traj][dim][11] FP32 initial coefficients (host or
 * device). In TRAJ_COST_PROJECT mode coeffs0 are also the samples that the
 * solve projects. Copied; the caller may reuse its buffers at once.
 * With traj_problem == NULL and the same n_traj as the previous call, only the
 * coefficients are replaced (asynchronously for a device source). */
traj_status traj_set_initial(traj_batch *b, int n_traj, const int *traj_problem,
                             const float *coeffs0);

typedef struct traj_solve_stats {
  int n_traj, n_solved;                /* solved = all three residuals <= tol */
  int iters_min, iters_median, iters_max;
  float max_res_obs, max_res_v, max_res_a; /* over the batch */
  float gpu_ms;                        /* device time of the solve (CUDA events) */
} traj_solve_stats;

/* Run Algorithm 2 on every trajectory in one persistent launch, captured once
 * as a CUDA graph (counter clears + kernel) and replayed while max_iters, tol,
 * timeout, the batch and the launch shape are unchanged: initialise by
 * projecting coeffs0 (lambda0 = 0), then iterate xi-step / projection /
 * multiplier update until the three L-infinity residuals (obstacle,
 * velocity, acceleration; metres, m/s, m/s^2) are all <= tol, checked after
 * every iteration k >= 1, or until max_iters. tol < 0 never stops early.
 * timeout_ms > 0 sets a device-side deadline (TRAJ_ETIMEOUT if hit).
 * Asynchronous on the stream when stats == NULL; with stats it synchronises
 * and fills them. Calling it again restarts from coeffs0.
 * Long horizons (Paper I plans over up to 1000 grid points): a batch whose
 * longest problem has more than 256 grid points runs one warp per trajectory
 * that streams its grid points in chunks (256 in 2D, 128 in 3D) every
 * iteration (FP32 form
 * only; TRAJ_ESHAPE in the tensor-core form or with warps_per_trajectory > 1).
 * The basis tables of the distinct horizons stay within 160 KB (n_p = 1000
 * alone takes 144 KB). */
traj_status traj_solve(traj_batch *b, int max_iters, float tol, double timeout_ms,
                       traj_solve_stats *stats);

/* Statistics of the last solve, as traj_solve fills them (synchronises the stream;
 * the same return codes as a traj_solve with stats): lets a caller launch
 * asynchronously (stats = NULL) and read the statistics later. No paper
 * counterpart. */
traj_status traj_get_solve_stats(traj_batch *b, traj_solve_stats *stats);

/* Results of the last solve into caller buffers (host or device, each
 * nullable): coeffs[n_traj][dim][11] FP32, residual[n_traj][3] FP32
 * (obstacle, velocity, acceleration), iters[n_traj] int32 (iterations run),
 * status[n_traj] int8 (TRAJ_TRAJ_*). Device destinations are written
 * asynchronously on the stream; host destinations synchronise. */
traj_status traj_get_trajectories(traj_batch *b, float *coeffs, float *residual, int *iters,
                                  signed char *status);

/* Smoothness cost of the last solve's trajectories, c_1 = sum_t ||p''(t)||^2
 * over the grid (PRIEST's acceleration cost), FP32 [n_traj], host or device. */
traj_status traj_get_accel_cost(traj_batch *b, float *cost);

/* Homotopy signature of each trajectory of the last solve (2D, n_p <= 256): bit j
 * (j < 64) is set when obstacle j of its problem is on the trajectory's left as they
 * pass, judged at the closest approach over the grid points (distances scaled by the
 * semi-axes): (p - o_j) x (p' - v_j) > 0 there.
 * Solutions of one problem with equal signatures pass every obstacle on the same
 * side. Used to choose training labels of the learned warm start that cover
 * different homotopy classes. sig: uint64 [n_traj], host or device. No paper
 * counterpart. */
traj_status traj_homotopy_signature(traj_batch *b, unsigned long long *sig);

/* Solver state for checkpoint/resume and warm starts (nullable outputs):
 * multipliers lambda[n_traj][dim][11] and the last residual contraction
 * u = F^T (F xi - g) [n_traj][dim][11], FP32, host or device. Together with the
 * coefficients of traj_get_trajectories this is the whole iteration state. */
traj_status traj_get_state(traj_batch *b, float *lambda, float *u);

/* Workspace bounds (Paper III, PRIEST: G xi <= tau with G = [-P; P] per axis and a
 * slack s = max(0, tau - G xi)): lower <= p(t) <= upper at every grid point, per
 * problem, host FP64 [n_problems][dim] each, finite with lower < upper; both NULL
 * removes them. The rows join the obstacle group: their residual
 * p - clamp(p, lower, upper) enters F^T r with the basis P and the obstacle
 * residual column takes the maximum of both. Recomputes the set-up if obstacles
 * are loaded; traj_set_problems clears the bounds. */
traj_status traj_set_workspace(traj_batch *b, const double *lower, const double *upper);

/* Penalty continuation (Paper I, Algorithm 1 line 9: the penalty grows while the
 * residuals stay above the threshold; Paper IV: the KKT inverse cached for ten
 * increasing penalties used in the later iterations): a ladder of `levels`
 * penalties rho * growth^l (l = 0 .. levels-1, levels <= 10), each with its own
 * KKT inverse formed once in FP64. A trajectory starts at level 0 and moves up one
 * level after every `every`-th iteration at which it has not converged (the
 * threshold is the solve's tol; with tol < 0, at every `every`-th iteration) until
 * the last level. levels = 1 (the default) is the fixed penalty of the config.
 * Recomputes the set-up if obstacles are loaded; TRAJ_EINVAL on bad arguments. */
traj_status traj_set_rho_schedule(traj_batch *b, int levels, double growth, int every);

/* Resume from an exported state (checkpoint/resume; the multipliers carried from
 * one receding-horizon call to the next, Paper II's MPC use): coefficients,
 * lambda and u as traj_get_trajectories / traj_get_state return them, FP32
 * [n_traj][dim][11] each, host or device, for the current trajectories. The
 * following traj_solve calls start with a QP step from this state instead of the
 * initial projection, and run up to max_iters more iterations (iters counts these);
 * solving N iterations, exporting, and resuming for M gives the iterate of N + M
 * iterations (bitwise, same launch shape). traj_set_initial returns to fresh
 * starts. Smoothness/tracking cost only (TRAJ_EINVAL in projection mode). No
 * paper counterpart as an interface. */
traj_status traj_set_state(traj_batch *b, const float *coeffs, const float *lambda, const float *u);

/* Receding-horizon step (Paper II's MPC: the batch optimizer runs once per control
 * loop, and each loop's solve starts from the Lagrange multipliers of the previous
 * one). After a solve, the robot has followed one planned trajectory per problem for
 * `delta` seconds (0 < delta < T of every problem). This call prepares the next
 * control loop's solve, on the device (FP64 where it forms new values):
 *  - executed[n_problems] (host int, or NULL): the trajectory of each problem that
 *    the robot followed; NULL picks, per problem, the trajectory with the smallest
 *    worst-of-three residual of the last solve (ties to the lower index). Each
 *    entry must be a trajectory of its problem (TRAJ_EINVAL otherwise).
 *  - the executed plan's position, velocity and acceleration at delta become the
 *    problem's start boundary rows (goal, horizon T and grid unchanged; the tracking
 *    line x_des now runs from the new start);
 *  - every obstacle moves on to c + v delta (its constant-velocity prediction);
 *    traj_set_obstacles afterwards replaces them with fresh data if the caller has any;
 *  - every trajectory's coefficients are re-expressed on the shifted window
 *    [delta, delta + T] (the same polynomial, extrapolated past its old end) and
 *    become the next initial iterate; the multipliers lambda are kept as they are;
 *  - the constants that depend on the boundary values (K12 b and the tracking term
 *    K11 q, eq. Q_matrix) are formed again in FP64; the KKT inverse itself (which the
 *    shift leaves as it was: same n_p, T, obstacle count, rho and bounds) is not.
 *    The FP64 set-up of traj_set_obstacles, traj_set_rho_schedule and
 *    traj_set_workspace keeps its FP64 blocks (1.5 KB per problem and penalty level,
 *    allocated then; TRAJ_ENOMEM if that fails), so every shift only launches the
 *    obstacle packing and the boundary update, asynchronously.
 * The next traj_solve projects the shifted iterate, so u is formed for the moved
 * problem, with lambda0 = the carried multipliers instead of 0, then iterates as
 * usual (iters counts from 0). traj_set_initial returns to fresh starts and
 * traj_set_state to a resume. TRAJ_ESTATE before a solve has run; TRAJ_EINVAL in
 * projection mode or for a delta outside (0, T). */
traj_status traj_shift_horizon(traj_batch *b, double delta, const int *executed);

/* One receding-horizon control step: traj_shift_horizon(delta, executed) followed by
 * traj_solve(max_iters, tol, timeout_ms, NULL), with the same results bit for bit,
 * replayed as one CUDA graph on the handle's stream (the shift's kernels, the
 * obstacle packing, the boundary update, the counters' reset and the persistent
 * solve). The graph is captured at the first call and again when delta, whether
 * executed is given, the solve's arguments or the launch shape change, or after any
 * traj_set_* call; executed (host int[n_problems], or NULL for each problem's
 * smallest worst residual) is checked on the host and copied before the replay.
 * Asynchronous; traj_get_solve_stats afterwards reports the step's GPU time (shift and
 * solve). Errors as the two calls it stands for, and TRAJ_ECUDA if the capture fails
 * (then nothing of the step has run and the handle is as before the call).
 * Without kept FP64 blocks (a handle whose set-up has not run with its obstacles) it
 * makes the two calls instead. Passage: Paper II, the MPC use of Algorithm 2
 * (warm-started iterations per control loop). */
traj_status traj_mpc_step(traj_batch *b, double delta, const int *executed, int max_iters,
                          float tol, double timeout_ms);

/* Solve without allocating any memory, for callers that cannot allocate
 * device memory: code running under an allocator or memory pool owned by
 * another framework, plugins that may only use the buffers they are handed,
 * or real-time paths where an allocation could stall. Such callers cannot
 * create a traj_batch (its workspace is allocated), so this entry point runs
 * the same set-up and solve kernels with every intermediate kept in one
 * fixed-size device array (about 1.4 MB) that the library reserves at load
 * time in every GPU that loads it, until the process exits. The paper has no
 * counterpart; this is an interface for constrained callers.
 *  - cfg: as for traj_batch_create (capacity fields ignored; precision must
 *    be TRAJ_PREC_FP32); its stream carries all the work.
 *  - Host arrays: n_steps, duration, start, goal (as traj_set_problems) and
 *    obs_offsets[n_problems + 1] (as traj_set_obstacles).
 *  - Device arrays (FP32 unless stated): centers, semi_axes, velocities
 *    [N][dim]; traj_problem[n_traj] (int32); coeffs0[n_traj][dim][11]; and
 *    the outputs coeffs[n_traj][dim][11], residual[n_traj][3],
 *    iters[n_traj] (int32), status[n_traj] (int8), as traj_get_trajectories.
 *  - Limits: n_problems <= 256, N <= 8192 obstacles, n_traj <= 8192, n_p <=
 *    256, basis tables of the distinct horizons <= 160 KB; beyond them the
 *    call returns TRAJ_ESHAPE with the limit named in traj_last_error(NULL).
 *  - Every traj_problem entry must lie in [0, n_problems): the entries are
 *    range-checked on the device before any kernel indexes a problem with
 *    them, and a bad one makes the call return TRAJ_EINVAL with no output
 *    written. The device arrays must hold the sizes above; the library cannot
 *    check the size of a device allocation.
 *  - Synchronous: returns after the solve has finished on the stream. The
 *    first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress), so make that first call before any stream capture.
 *  - Every call shares the one array: calls that overlap on the GPU (other
 *    threads, other streams) race and corrupt each other. Each call rewrites
 *    the parts it uses and clears its counters, so nothing leaks between calls
 *    that run one after another.
 *  - Calls no cudaMalloc, cudaFree or other allocating routine. */
traj_status traj_solve_noalloc(const traj_config *cfg, int n_problems, const int *n_steps,
                               const double *duration, const double *start, const double *goal,
                               const int *obs_offsets, const float *centers,
                               const float *semi_axes, const float *velocities, int n_traj,
                               const int *traj_problem, const float *coeffs0, int max_iters,
                               float tol, float *coeffs, float *residual, int *iters,
                               signed char *status);

/* CTA shape of the persistent solve launch: warps per block (1..8; 0 = the
 * default of the form), resident blocks per SM (0 = as many as the occupancy
 * query allows; a positive count caps it, and in the tensor-core forms it is also
 * honoured above the query's answer, which is conservative for these kernels, as
 * far as registers, shared memory, tensor memory and warp slots hold) and the warps
 * that share one trajectory (1, 2 or 4,
 * dividing warps_per_block: the grid's 32-point blocks dealt round-robin to the
 * warps, partial contractions exchanged through shared memory; FP32 form only). occupancy = 1
 * selects the build whose registers are capped so that more warps stay resident
 * (FP32 form: 128 registers, at most 4 warps per block; tensor-core forms: 170
 * registers, at most 6), for one warp per trajectory and horizons up to 160 grid
 * points; 0 leaves the registers unrestricted (the lowest latency per warp). The grid
 * never exceeds what the batch needs. Results are bitwise identical across shapes and
 * builds with the same warps per trajectory; across those they differ only in the
 * summation order of the contraction. */
typedef struct traj_launch_shape {
  int warps_per_block;
  int blocks_per_sm;
  int warps_per_trajectory;
  int occupancy;
} traj_launch_shape;

/* Use this launch shape for later solves (default: FP32 form 4 warps per block,
 * tensor-core form and horizons above 256 grid points the batch spread over all
 * SMs; occupancy-bound blocks per SM). */
traj_status traj_set_launch_shape(traj_batch *b, const traj_launch_shape *shape);

/* The shape the last captured solve launch resolved to: warps per block, resident
 * blocks per SM the launch counted on (after occupancy, shared memory and, in the
 * tensor-core form, tensor-memory limits), warps per trajectory and build, the grid
 * size, the kernel's registers per thread and its dynamic shared memory per block
 * in bytes (nullable outputs; 0 registers for a long-horizon launch). TRAJ_ESTATE
 * before the first solve. No paper counterpart. */
traj_status traj_get_launch_info(traj_batch *b, traj_launch_shape *resolved, int *grid,
                                 int *registers, int *shared_bytes);

/* Autotuner: times every candidate shape (warps per block in {0,1,2,4,8} x
 * blocks per SM in {occupancy,1,2,4} x warps per trajectory in {1,2,4}, the
 * latter in the FP32 form only, plus the register-capped build with one warp per
 * trajectory, warps per block in {0,2,4} (tensor-core forms also 6) and blocks per
 * SM in {occupancy,2,3} where the horizons allow it) on this handle's own batch with `iters`
 * fixed iterations, keeps the fastest for later solves and reports it in
 * *chosen and its time per solve in *best_ms (both nullable). Synchronises;
 * the previous solve's results are discarded. No paper counterpart. */
traj_status traj_autotune(traj_batch *b, int iters, traj_launch_shape *chosen, float *best_ms);

/* ---- Projection-guided sampler (Paper III, Algorithm 3) ---------------------
 * Settings of one outer iteration. Samples are drawn from N(mu, Sigma + eps I);
 * n_inner projection iterations (Algorithm 2 order with Q = I, q = -sample,
 * eq. matrix_vec); r = the worst of the three L-infinity residuals; the
 * n_proj lowest r form the ConstraintEliteSet, the n_elite lowest
 * c_aug = c_1 + w_res * r among them the EliteSet, where
 * c_1 = sum_t (||p''(t)||^2 + w_curv c_kappa(t) + w_path c_p(t)) on the grid:
 * c_kappa = ||p' x p''||^2 / ||p'||^6 is the squared curvature (the planar
 * form of the BARN cost, Section 5; taken as 0 where ||p'|| < 1e-3, which covers the rest start) and c_p the
 * distance of p(t) from the segment between problem 0's start and goal (a cost
 * with no closed form: it needs the projection onto the path); weights
 * exp(-(c_aug - min c_aug) / gamma); mean and covariance move by sigma_lr
 * toward the weighted elite mean/covariance (eqs. update_mean,
 * update_covariance; the covariance about the new mean). */
typedef struct traj_sampler_config {
  int n_inner, n_proj, n_elite;
  float gamma, sigma_lr, eps, w_res;
  unsigned long long seed; /* Philox4x32-10 key (counter = sample, iteration, pair, 0) */
  float w_curv, w_path;    /* >= 0; 0 and 0 give the acceleration-only cost */
} traj_sampler_config;

/* Largest number of sampling distributions of traj_sampler_step_multi. */
#define TRAJ_SAMPLER_MAX_DIST 64

/* Optional device copies of one step's intermediates (each nullable):
 * samples and projected [n_traj][dim*11], residual and cost_aug [n_traj],
 * proj_idx [n_proj] and elite_idx [n_elite] (ascending by key, ties by index). */
typedef struct traj_sampler_trace {
  float *samples, *projected, *residual, *cost_aug;
  int *proj_idx, *elite_idx;
} traj_sampler_trace;

/* One outer iteration of Algorithm 3 on problem 0 of a TRAJ_COST_PROJECT
 * handle whose n_traj trajectories (<= 8192) all belong to problem 0.
 * mu [dim*11] and sigma [(dim*11)^2] are device arrays updated in place
 * (coefficient order [axis][11]); z is a device array [n_traj][dim*11] of
 * standard normal draws, or NULL to draw them on the device with Philox and
 * Box-Muller; best [dim*11 + 1] receives the lowest-c_aug elite and its c_aug.
 * Asynchronous on the handle's stream. */
traj_status traj_sampler_step(traj_batch *b, const traj_sampler_config *cfg, int iteration,
                              float *mu, float *sigma, const float *z, float *best,
                              const traj_sampler_trace *trace);

/* Decentralised sampler (D-PRIEST, Section 5): n_dist distributions refined in
 * parallel. The n_traj samples split into n_dist contiguous groups of
 * Bg = n_traj / n_dist (n_dist must divide n_traj, 1 <= n_dist <=
 * TRAJ_SAMPLER_MAX_DIST, Bg <= 8192); group g draws from N(mu_g, Sigma_g), and
 * its ConstraintEliteSet, EliteSet and refit use its own samples only, with
 * cfg->n_proj and cfg->n_elite counted per group (<= Bg). One projection solve
 * covers all groups. mu [n_dist][dim*11], sigma [n_dist][dim*11][dim*11] and
 * best [n_dist][dim*11 + 1] are device arrays; Philox draws use the sample's
 * index in the whole batch, so n_dist = 1 is traj_sampler_step. Trace arrays:
 * samples ... cost_aug as above over all n_traj; proj_idx [n_dist][n_proj] and
 * elite_idx [n_dist][n_elite] hold indices local to the group. */
traj_status traj_sampler_step_multi(traj_batch *b, const traj_sampler_config *cfg, int iteration,
                                    int n_dist, float *mu, float *sigma, const float *z,
                                    float *best, const traj_sampler_trace *trace);

/* BF16 tensor-core GEMM, the building block of the warm-start network:
 * C[M][N] = A[M][K] * B[N][K]^T with FP32 accumulation (tcgen05, TMA-staged
 * operands). A, B: device BF16, row-major, K % 8 == 0, 16-byte aligned; C:
 * device FP32 [M][N]; err: device int whose bit 0 is set if a pipeline wait
 * expired (the result is then incomplete). Asynchronous on the stream. No
 * paper counterpart. */
traj_status traj_gemm_bf16(int M, int N, int K, const void *A, const void *B, float *C, int *err,
                           void *cuda_stream);

/* ---- Learned warm start (no paper counterpart: the thesis lists learning-
 * based methods as future work) ------------------------------------------------
 * An MLP 388 -> 256 -> 256 -> 256 -> 176 (GELU, tanh form) maps a scene's
 * features to K = 8 proposal coefficient sets, read as offsets from the
 * straight-line coefficients. BF16 weights and activations on the tcgen05
 * tensor cores with FP32 accumulation; FP32 master weights and AdamW
 * (beta 0.9/0.999, eps 1e-8, decoupled decay on the weight matrices).
 * Features (388 per scene, stored BF16 in rows of 400): start and goal
 * relative to the start, x0.1; then the 64 obstacles whose t = 0 centre is
 * nearest to the start->goal segment (ascending distance, ties by index),
 * each (cx, cy) relative to the start x0.1, semi-axes (a, b), velocity
 * (vx, vy); absent slots are zero. 2D only.
 * Parameters (public flat FP32 order): W1[256][388], b1[256], W2[256][256],
 * b2, W3[256][256], b3, W4[176][256], b4[176].
 * Loss: for each solved label t_m of a scene (offsets from the line, up to 8),
 * min_k ||y_k - t_m||^2 + 0.05 * mean_k ||y_k - t_m||^2, averaged over all
 * labels of the batch. Rows of a batch: a multiple of 8, <= max_rows. */
typedef struct traj_warmstart traj_warmstart;
int traj_warmstart_num_params(void);
traj_status traj_warmstart_create(int max_rows, void *cuda_stream, traj_warmstart **out);
traj_status traj_warmstart_destroy(traj_warmstart *w);
/* params: host or device FP32 [num_params]; resets the optimizer state */
traj_status traj_warmstart_set_params(traj_warmstart *w, const float *params);
traj_status traj_warmstart_get_params(traj_warmstart *w, float *params);
/* Training checkpoint and resume (no paper counterpart: the thesis leaves the
 * learned warm start to future work). params, m, v: FP32 [num_params] each, in
 * the public flat order, host or device: the FP32 master parameters and AdamW's
 * first and second moment estimates; step: AdamW's step count (its bias
 * corrections). get copies them out (synchronises); set restores all four and
 * the BF16 copies of the weights, so that the next train_step continues as the
 * uninterrupted run would, bit for bit. TRAJ_EINVAL for NULL buffers or
 * step < 0; the caller owns every buffer. */
traj_status traj_warmstart_get_state(traj_warmstart *w, float *params, float *m, float *v,
                                     int *step);
traj_status traj_warmstart_set_state(traj_warmstart *w, const float *params, const float *m,
                                     const float *v, int step);
/* start, goal [n][2] FP64 and offsets [n + 1] host; obstacles device FP32 [N][2];
 * features: device BF16 [n][400]; line: device FP32 [n][22] straight-line coefficients */
traj_status traj_warmstart_features(traj_warmstart *w, int n_scenes, const double *start,
                                    const double *goal, const int *offsets, const float *centers,
                                    const float *semi_axes, const float *velocities,
                                    void *features, float *line);
/* proposals: device FP32 [rows][8][2][11] = line + network output */
traj_status traj_warmstart_forward(traj_warmstart *w, int rows, const void *features,
                                   const float *line, float *proposals);
/* Features, forward and proposals in one asynchronous pass on device inputs only
 * (no host copy, no synchronisation): start, goal device FP64 [n][2]; offsets
 * device int [n + 1] into n_obs obstacles (device FP32 [n_obs][2] each); features
 * (device BF16 [n][400]) and line (device FP32 [n][22]) are caller scratch that
 * receive the same values as traj_warmstart_features; proposals device FP32
 * [n][8][2][11]. n_scenes is a multiple of 8 in [8, max_rows]. Offsets are
 * checked on the device: a scene whose range leaves [0, n_obs] gets no obstacle
 * features and makes the next traj_warmstart_sync return TRAJ_EINVAL. */
traj_status traj_warmstart_propose(traj_warmstart *w, int n_scenes, int n_obs, const double *start,
                                   const double *goal, const int *offsets, const float *centers,
                                   const float *semi_axes, const float *velocities, void *features,
                                   float *line, float *proposals);
/* targets: device FP32 [rows][8][22] label offsets; n_labels: device int [rows];
 * loss: device FP32 scalar; grads (nullable): FP32 [num_params], host or device */
traj_status traj_warmstart_gradients(traj_warmstart *w, int rows, const void *features,
                                     const float *targets, const int *n_labels, float *grads,
                                     float *loss);
/* The same loss and gradients with every GEMM operand, activation and gradient in
 * FP32 on the CUDA cores (no tensor cores, no BF16 rounding): the debug
 * instantiation that checks the network's backward pass against an FP64
 * reference to FP32 accuracy. Arguments as traj_warmstart_gradients (the BF16
 * features are read as FP32 values); allocates its FP32 buffers on the first call. */
traj_status traj_warmstart_gradients_fp32(traj_warmstart *w, int rows, const void *features,
                                          const float *targets, const int *n_labels, float *grads,
                                          float *loss);
traj_status traj_warmstart_train_step(traj_warmstart *w, int rows, const void *features,
                                      const float *targets, const int *n_labels, float lr,
                                      float weight_decay, float *loss);
/* synchronise; TRAJ_EINVAL if traj_warmstart_propose met bad offsets, TRAJ_ECUDA if
 * a GEMM pipeline wait expired, since the previous sync (the flags are then cleared) */
traj_status traj_warmstart_sync(traj_warmstart *w);

/* Human-readable name of a status code (static string). */
const char *traj_status_string(traj_status s);

/* Detail of the last failure on this handle (static per handle; "" if none). */
const char *traj_last_error(traj_batch *b);

/* FP32 FMA throughput microbenchmark, the denominator of the ALU roofline:
 * runs independent-chain kernels of scalar FMA and of packed two-lane FMA
 * (f32x2) on the stream and returns the better achieved FP32 FLOP/s (2 per
 * FMA), best of `reps` timed launches each. No paper counterpart (measurement). */
traj_status traj_measure_fp32_peak(void *cuda_stream, int reps, double *flops_per_s);

/* MUFU throughput microbenchmark, the denominator of the MUFU roofline: runs a
 * kernel of independent rsqrtf chains (the special-function instruction the
 * projections issue, once per point inside an obstacle and per velocity /
 * acceleration bound test) and returns the achieved rsqrtf/s, best of `reps`
 * timed launches. No paper counterpart (measurement). */
traj_status traj_measure_mufu_peak(void *cuda_stream, int reps, double *rsqrt_per_s);

/* ---- Joint multi-agent optimizer (Paper IV, Algorithm 5) ---------------------
 * A batch of independent scenes, each with n_agents agents solved jointly: every
 * agent is a degree-10 Bernstein polynomial per axis on an n_steps-point grid
 * over [0, T_s]; cost 1/2 sum_i sum_t ||p_i''(t)||^2 (the QP form of eq.
 * eq_step_x); position fixed at both ends with zero velocity and acceleration
 * (eqs. eq_multiagent_start, eq_multiagent_final); agents are spheroids of
 * horizontal radius r_s and half-height h_s (circles of radius r_s in 2D), kept
 * apart pairwise through x_i - x_j = d_ij e(alpha_ij, beta_ij), d_ij >= 1, on the
 * spheroid (2r, 2r, 2h) (eq. sphere_proposed); static obstacles are spheres of
 * radius r_o kept out through the spheroid (r + r_o, r + r_o, h + r_o).
 * Each iteration: the x-step through KKT inverses cached once per scene and
 * penalty (eq. kkt_step_x), alpha/beta in closed form (eqs. com_alpha_i,
 * com_beta_i), d (eq. com_d_i, then d >= 1) and the multiplier updates (eqs.
 * update_lamda_xi .. update_lamda_zi). The initial iterate is each agent's
 * obstacle-free optimum; the residual is the largest ||x_i - x_j - d e|| over
 * pairs, obstacles and grid points, and a scene stops at the first iteration
 * whose residual is <= tol. Penalty ladder: rho growth^l, l < rho_levels, one
 * level up after every rho_every-th unconverged iteration (the paper caches ten
 * increasing penalties for the later iterations). One CTA solves one scene. */
typedef struct traj_ma_batch traj_ma_batch;

typedef struct traj_ma_config {
  int dim;           /* 2 or 3 */
  int max_scenes;    /* >= 1 */
  int max_agents;    /* 1 .. 64 */
  int max_obstacles; /* static spheres over all scenes, >= 0 */
  int n_steps;       /* grid points per agent trajectory, 2 .. 256 */
  float rho;         /* rho_o of level 0, > 0 */
  int rho_levels;    /* 0 or 1: a fixed rho; up to 10 */
  float rho_growth;  /* > 0 when rho_levels > 1 */
  int rho_every;     /* >= 0; 0 keeps level 0 */
} traj_ma_config;

typedef struct traj_ma_stats {
  float gpu_ms;         /* CUDA-event time of the solve launch */
  int n_converged;      /* scenes with residual <= tol */
  int max_iters_run;    /* largest iteration count over the scenes */
  int lambda_in_shared; /* 1 if the pair multipliers stayed in shared memory */
} traj_ma_stats;

/* Allocates the device workspace for the capacities (multipliers for every agent
 * pair and obstacle-agent pair of every grid point) on the given stream. */
traj_status traj_ma_create(const traj_ma_config *cfg, void *cuda_stream, traj_ma_batch **out);
traj_status traj_ma_destroy(traj_ma_batch *b);

/* Host arrays: duration [n_scenes] (s, FP64), start and goal [n_scenes][n_agents][dim]
 * (FP64), radius [n_scenes] and height [n_scenes] (FP32; height may be NULL in 2D),
 * obs_offsets [n_scenes + 1] (CSR over the obstacles, obs_offsets[0] = 0),
 * obs_centers [n_obs][dim] and obs_radii [n_obs] (FP32; NULL when there are none).
 * Forms and inverts the scenes' KKT matrices in FP64 on the GPU and synchronises.
 * TRAJ_ESHAPE if the sizes exceed the capacities or n_agents x n_steps does not fit
 * one CTA's shared memory; TRAJ_EINVAL for a singular KKT matrix or bad values. */
traj_status traj_ma_set_problems(traj_ma_batch *b, int n_scenes, int n_agents,
                                 const double *duration, const double *start, const double *goal,
                                 const float *radius, const float *height, const int *obs_offsets,
                                 const float *obs_centers, const float *obs_radii);

/* Runs up to max_iters iterations (0: the initial iterate only) from the initial
 * iterate; tol < 0 runs all of them. Asynchronous unless stats is non-NULL, which
 * synchronises and fills it. */
traj_status traj_ma_solve(traj_ma_batch *b, int max_iters, float tol, traj_ma_stats *stats);

/* coeffs [n_scenes][n_agents][dim][11], residual [n_scenes], iters [n_scenes]
 * (each nullable; host or device); synchronises. */
traj_status traj_ma_get_trajectories(traj_ma_batch *b, float *coeffs, float *residual, int *iters);

/* Detail of the last failure on this multi-agent handle, or of the last failed
 * traj_ma_create on this thread when b is NULL. */
const char *traj_ma_last_error(traj_ma_batch *b);

/* ---- Multi-circle footprint with heading (Paper II, Algorithm 2) -------------
 * A batch of 2D trajectories of a robot whose footprint is n_circles circles of
 * radius r_circle at offsets r_m along its heading psi(t) (a rectangle as
 * overlapping circles, eq. coll_multiagent). Per trajectory x, y and psi are
 * degree-10 Bernstein polynomials, with slack copies c, s of cos psi, sin psi
 * (eqs. cos_ref, sin_ref); cost sum_t (x''^2 + y''^2 + psi''^2 + (x - x_des)^2 +
 * (y - y_des)^2), x_des the constant-velocity line (eq. acc_cost); start
 * position with zero velocity and acceleration and goal position fixed, the
 * heading fixed at both ends (eqs. eq_multiagent_1, eq1_multiagent_1); speed <=
 * vmax, acceleration <= amax; every circle kept outside every moving ellipse
 * inflated by r_circle. One iteration: the xi-step per half (x, c) and (y, s)
 * through a KKT inverse cached per problem (eq. zeta_1_sepration_1), the heading
 * step through the convex surrogate on the unwrapped atan2(s, c) (eq.
 * compute_convex_surrogate), the alpha/d steps in closed form (eqs. zeta_2,
 * alpha_v, alpha_a, compute_d_mij, compute_dv, compute_da) and the multiplier
 * updates (eqs. update_lambda2_1, update_lambda2_2). One warp per trajectory. */
typedef struct traj_fp_batch traj_fp_batch;

typedef struct traj_fp_config {
  int max_problems, max_traj, max_obstacles; /* capacities, >= 1 (obstacles >= 0) */
  int max_steps;                             /* grid points per problem, 2 .. 256 */
  int n_circles;                             /* 1 .. 8 */
  float circle_offsets[8];                   /* r_m along the heading (m), first n_circles used */
  float r_circle;                            /* circle radius (m), >= 0 */
  float vmax, amax;                          /* > 0 */
  float rho, rho_psi;                        /* penalties of the xi- and heading steps, > 0 */
} traj_fp_config;

typedef struct traj_fp_stats {
  float gpu_ms;      /* CUDA-event time of the solve launch */
  int n_solved;      /* trajectories with all four residuals <= tol */
  int max_iters_run; /* largest iteration count */
} traj_fp_stats;

traj_status traj_fp_create(const traj_fp_config *cfg, void *cuda_stream, traj_fp_batch **out);
traj_status traj_fp_destroy(traj_fp_batch *b);

/* Host arrays: n_steps [P], duration [P] (s), start and goal [P][2] (FP64),
 * heading_start and heading_goal [P] (rad, FP64), obs_offsets [P + 1] (CSR,
 * obs_offsets[0] = 0), centers, semi_axes, velocities [n_obs][2] (FP32; an
 * obstacle sits at centre + velocity t). Forms the per-problem tables and the
 * FP64 KKT inverses on the GPU and synchronises. */
traj_status traj_fp_set_problems(traj_fp_batch *b, int n_problems, const int *n_steps,
                                 const double *duration, const double *start, const double *goal,
                                 const double *heading_start, const double *heading_goal,
                                 const int *obs_offsets, const float *centers,
                                 const float *semi_axes, const float *velocities);

/* Host arrays: traj_problem [n_traj], xi0 [n_traj][3][11] (x, y, psi). The copies
 * c, s start as cos psi, sin psi of xi0 on the grid; multipliers start at 0. */
traj_status traj_fp_set_initial(traj_fp_batch *b, int n_traj, const int *traj_problem,
                                const float *xi0);

/* Up to max_iters iterations per trajectory; a trajectory stops at the first
 * iteration whose four residuals (obstacle, speed, acceleration: L-infinity
 * distance to the feasible target over the grid; heading copy: max_t
 * ||(c, s) - (cos psi, sin psi)||) are <= tol (tol < 0: never). Asynchronous
 * unless stats is non-NULL (then synchronises). TRAJ_ESHAPE if a problem has
 * more than 456 704 obstacles (the solve keeps one bit per obstacle of a
 * problem in shared memory for its exact cull of the circle tests). */
traj_status traj_fp_solve(traj_fp_batch *b, int max_iters, float tol, traj_fp_stats *stats);

/* coeffs [n_traj][5][11] in the order x, c, y, s, psi; residual [n_traj][4];
 * iters [n_traj] (each nullable; host or device); synchronises. */
traj_status traj_fp_get_trajectories(traj_fp_batch *b, float *coeffs, float *residual, int *iters);

const char *traj_fp_last_error(traj_fp_batch *b);

#ifdef __cplusplus
}
#endif
#endif /* TRAJBATCH_H */

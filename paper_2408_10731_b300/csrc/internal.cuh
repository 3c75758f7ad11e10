// internal.cuh -- device data layouts and helpers shared by the library's
// translation units. Not part of the public ABI (include/trajbatch.h).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace tb {

constexpr int NC = 11;      // Bernstein degree 10 -> 11 coefficients per axis
constexpr int NE = 4;       // boundary rows per axis
constexpr int NK = NC + NE; // KKT size
constexpr int ROW = 12;     // padded row length (floats) of every 11-wide table row
constexpr int MAX_STEPS = 256;       // grid points per problem held in registers by a warp
constexpr int MAX_STEPS_LONG = 1024; // batch handle, FP32 form: longer horizons run chunked
constexpr int RHO_MAX_LEVELS = 10; // penalty levels of the continuation ladder
constexpr int MAX_HZ = 16;         // distinct horizons of one batch in the tensor-core form

// Per-problem record on the device (64 bytes).
struct ProblemDev {
  int n_p;        // timesteps
  int n_o;        // obstacles
  int pair_off;   // first obstacle-pair record (index into the packed pair array)
  int tbl_off;    // float offset of this horizon's P/dB/ddB tables in the table buffer
  float dt;       // T / (n_p - 1), seconds between grid points
  float invT;     // 1 / T   (Pdot = dB/dtau * invT)
  float invT2;    // 1 / T^2 (Pddot = d2B/dtau2 * invT2)
  int const_off;  // float offset of the problem's constants block
  int nan_flag;   // nonzero if the problem's obstacle data is not finite / not positive
  int box;        // 1: workspace bounds lo <= p(t) <= hi (PRIEST's G xi <= tau with slack)
  float lo[3], hi[3];
};

// Constants block per problem (floats), every row padded to ROW:
//   K11 hi/lo  [11][12] x 2     (top-left 11x11 block of the KKT inverse)
//   G   hi/lo  [11][12] x 2     (rho * K11 * F^T F)
//   hq  hi/lo  [3][12]  x 2     (K11 (-q_axis) + K12 b_axis; smoothness/tracking mode)
//   c   hi/lo  [3][12]  x 2     (K12 b_axis; projection mode adds K11 xi_sample)
// "hi/lo" is the FP64 value split into two FP32 numbers (hi = fl(x), lo = fl(x - hi)).
constexpr int C_K11_HI = 0;
constexpr int C_K11_LO = C_K11_HI + NC * ROW;
constexpr int C_G_HI = C_K11_LO + NC * ROW;
constexpr int C_G_LO = C_G_HI + NC * ROW;
constexpr int C_HQ_HI = C_G_LO + NC * ROW;
constexpr int C_HQ_LO = C_HQ_HI + 3 * ROW;
constexpr int C_C_HI = C_HQ_LO + 3 * ROW;
constexpr int C_C_LO = C_C_HI + 3 * ROW;
constexpr int CONST_FLOATS = C_C_LO + 3 * ROW; // 672

// Tables per horizon (floats): P [n_p][12], dB/dtau [n_p][12], d2B/dtau2 [n_p][12],
// FP32 copies of FP64 values, column 11 zero. TABLE_FLOATS(n_p) = 36 n_p.
__host__ __device__ inline int table_floats(int n_p) { return 3 * ROW * n_p; }

// Packed obstacle-pair records: a problem's obstacles j = 2q, 2q + 1 share record q
// (an odd count is padded with a sentinel that is never inside), each record
// PAIR_VEC(dim) float4, every float4 holding the same quantity of both obstacles so
// that the containment test runs on packed two-lane arithmetic. The values are
// normalised by the semi-axes a, u = (p - c - v t) / a = p * ia + (nc + nv t), with
// nc = -c / a, nv = -v / a, ia = 1 / a (formed in FP64, rounded once):
//  2D: {ncx0, ncx1, nvx0, nvx1}, {ncy0, ncy1, nvy0, nvy1}, {iax0, iax1, iay0, iay1},
//      {ax0, ax1, ay0, ay1}
//  3D: {ncx0, ncx1, nvx0, nvx1}, {ncy0, ncy1, nvy0, nvy1}, {ncz0, ncz1, nvz0, nvz1},
//      {iax0, iax1, iay0, iay1}, {iaz0, iaz1, ax0, ax1}, {ay0, ay1, az0, az1}
// Sentinel half: nc = 1e18, nv = 0, ia = a = 1.
__host__ __device__ constexpr int pair_vec(int dim) { return dim == 2 ? 4 : 6; }
// The containment test reads only the first pair_test_vec float4 of a record.
__host__ __device__ constexpr int pair_test_vec(int dim) { return dim == 2 ? 3 : 5; }
__host__ __device__ constexpr int pair_count(int n_o) { return (n_o + 1) / 2; }
constexpr float PAIR_SENTINEL = 1.0e18f;

// Arguments of one solve launch.
struct SolveArgs {
  const ProblemDev *problems;
  const float4 *obstacles;
  const float *constants;
  const float *tables;
  int table_floats_total;
  const int *traj_problem;
  const int *order;
  const float *xi0;
  const float *lam0;          // resume: multipliers and last contraction of the iterate in
  const float *u0;            //   xi0 ([n_traj][dim][11]); both NULL for a fresh start;
                              //   carry (receding horizon): lam0 only, u0 NULL
  float *xi;
  float *lam;
  float *u;
  float *res;
  int *iters;
  signed char *status;
  int n_traj;
  int max_iters;
  float tol;
  float rho;
  float vmax, amax;
  int cost_mode;
  unsigned long long timeout_ns;
  int *queue;                 // work-queue counter, zeroed before the launch
  unsigned long long *t0;     // launch start time (globaltimer), zeroed before the launch
  int *flags;                 // bit 0: timeout hit, bit 1: NaN input seen, bit 3: MMA wait expired
  // penalty continuation: rho_levels constants blocks per problem (level l at const_off +
  // l CONST_FLOATS) for the penalties rho_ladder[l]; the level rises by one after every
  // rho_every-th iteration that has not converged (rho_every = 0: a single rho)
  const float *rho_ladder;
  int rho_levels;
  int rho_every;
  // distinct horizons of the batch (the tensor-core form builds one basis operand per
  // horizon): n_p and basis-table offset of each, in table order
  int hz_n;
  int hz_np[MAX_HZ];
  int hz_tbl[MAX_HZ];
};

// ---- compensated (double-float) helpers -----------------------------------
// acc(hi, lo) += (a_hi + a_lo) * x with the exact product error of a_hi * x and a
// TwoSum accumulation (Knuth); the _rn intrinsics keep the compiler from fusing
// or reassociating the error-free transformations.
__device__ __forceinline__ void df_fma(float &hi, float &lo, float a_hi, float a_lo, float x) {
  float p = __fmul_rn(a_hi, x);
  float e = __fmaf_rn(a_hi, x, -p);
  e = __fmaf_rn(a_lo, x, e);
  float s = __fadd_rn(hi, p);
  float bb = __fsub_rn(s, hi);
  float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(err, e));
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

} // namespace tb

// Launch wrappers implemented in the .cu files (host side, C++ linkage).
namespace tb {
cudaError_t launch_setup_tables(const int *d_horizons, const int *d_offsets, int n_horizons,
                                float *d_tables, cudaStream_t s);
// d_start_va [n_problems][2][dim]: start velocity and acceleration of the boundary rows
// (NULL: at rest)
// kkt_out (nullable): per problem p, FP64 K11 [11][11], K12 [11][4] and the basis
// moments m0 = sum_t P_t (1 - tau_t), m1 = sum_t P_t tau_t [11] each, at
// kkt_out + p * kkt_stride (KKT64_DOUBLES doubles), so that a change of the boundary
// values alone (launch_setup_boundary) need not form and invert K again.
constexpr int KKT64_DOUBLES = NC * NC + NC * NE + 2 * NC; // 187
cudaError_t launch_setup_problems(ProblemDev *d_problems, int n_problems, const double *d_T,
                                  const double *d_start, const double *d_goal,
                                  const double *d_start_va, int dim, double rho, double w_smooth,
                                  double w_track, int cost_mode, int max_np, float *d_constants,
                                  cudaStream_t s, double *kkt_out = nullptr, size_t kkt_stride = 0);
// The boundary-dependent constants alone (hq and c of the smoothness/tracking cost, eq.
// Q_matrix's q = -w_t P^T x_des with x_des the start -> goal line, and K12 b with b =
// (start, v0, a0, goal)) of every problem and penalty level, from the FP64 blocks that
// launch_setup_problems stored: after a receding-horizon shift, which moves the start
// state but leaves the KKT matrix (n_p, T, n_o, rho) unchanged. Level l of problem p:
// kkt64 + (p * levels + l) * KKT64_DOUBLES, constants + p * CONST_FLOATS * levels +
// l * CONST_FLOATS.
cudaError_t launch_setup_boundary(int n_problems, int levels, const double *d_start,
                                  const double *d_goal, const double *d_start_va, int dim,
                                  double w_track, const double *kkt64, float *d_constants,
                                  cudaStream_t s);
// Receding-horizon step (mpc.cu): executed [n_problems] device indices (or NULL: per
// problem the trajectory with the smallest worst residual, chosen into exec_scratch);
// every trajectory's xi re-expressed on the window shifted by delta seconds into xi0,
// lam copied to lam0; the executed plans' state at delta into start / start_va; every
// obstacle centre moved by v delta in the staged centres.
struct ShiftArgs {
  int dim, n_problems, n_traj, n_obs;
  double delta;
  const double *T;                 // [n_problems]
  const int *traj_problem;         // [n_traj]
  const float *xi, *lam, *res;     // last solve: [n_traj][dim][11] x2, [n_traj][3]
  float *xi0, *lam0;               // next solve's start
  const int *executed;             // [n_problems] or NULL
  int *exec_scratch;               // [n_problems]
  unsigned long long *key_scratch; // [n_problems]
  double *start, *start_va;        // [n_problems][dim], [n_problems][2][dim]
  float *centers;                  // staged obstacle centres [n_obs][dim]
  const float *velocities;         // [n_obs][dim]
};
cudaError_t launch_mpc_shift(const ShiftArgs &a, cudaStream_t s);
// Obstacle-pair records of all problems: n_slots = 2 x (total pair records); offsets
// (CSR obstacle offsets, n_problems + 1) and pair_off (first record of each problem,
// n_problems + 1) are device arrays.
cudaError_t launch_pack_obstacles(int dim, int n_problems, int n_slots, const int *offsets,
                                  const int *pair_off, const float *centers, const float *axes,
                                  const float *vel, float4 *out, ProblemDev *problems,
                                  cudaStream_t s);
// CTA shape of the persistent solve launch (the autotuner's search space);
// zero fields take the defaults (FP32 form: 4 warps; tensor-core form: the batch
// spread over all SMs; occupancy-limited blocks per SM; one warp per trajectory).
struct LaunchShape {
  int warps_per_block;
  int blocks_per_sm;
  int grid; // filled in by the launcher
  int team; // warps per trajectory: 1 or 2
  int occupancy; // 1: the build whose registers are capped for more resident warps
                 // (FP32 form: 128 per thread, at most 4 warps per block; tensor-core
                 // form: 170, at most 6 warps), one warp per trajectory, horizons up
                 // to 160 grid points; 0: registers unrestricted
  int regs;      // filled in by the launcher: registers per thread of the kernel,
  int smem;      //   dynamic shared memory per block (bytes)
};
// tensor-core form (am_mixed.cu); horizons up to max_np <= 256, the distinct ones in
// a.hz_*; split: hi/lo BF16 operand pairs; the shape's warps per block (0: the batch
// spread over all SMs) and blocks per SM apply
cudaError_t launch_am_mixed(int dim, int max_np, bool split, const SolveArgs &a,
                            const LaunchShape &shape, int n_sm, cudaStream_t s, LaunchShape *used);
// shared memory of one CTA of the tensor-core form with `warps` warps
size_t mixed_smem_bytes(const SolveArgs &a, int dim, bool split, int warps);
cudaError_t launch_am_solve(int dim, int max_np, int precision, const SolveArgs &a,
                            const LaunchShape &shape, int n_sm, cudaStream_t s,
                            LaunchShape *used);
// The sampler's stages for n_dist distributions of B / n_dist samples each
// (mu [n_dist][D], sigma and L_scratch [n_dist][D][D]).
cudaError_t launch_sampler_front(const float *mu, const float *sigma, int D, int B, int n_dist,
                                 float eps, const float *z, unsigned long long seed, int iteration,
                                 float *L_scratch, int *flag, float *xi0, float *samples_out,
                                 cudaStream_t s);
// cost terms: c_aug = sum_t (||p''||^2 + w_curv c_kappa + w_path c_p) + w_res r, with the
// path from start to goal (device FP64 [dim])
// refit_scratch: 2 * n_dist * ((n_elite * D + 3) & ~3) + n_dist * (D + 1) floats, 16-byte
// aligned (the elites' weighted and centred coefficients, and the refit's new means and
// weight sums).
struct SamplerCost {
  float w_res, w_curv, w_path;
  const double *start, *goal;
};
cudaError_t launch_sampler_back(const float *xi, const float *res, const float *tables,
                                int tbl_off, int n_p, float invT, float invT2, int dim, int B,
                                int n_dist, const SamplerCost &cost, int n_proj, int n_elite,
                                float gamma, float sig, float *r_out, float *caug_out,
                                int *proj_idx, int *elite_idx, float *refit_scratch, float *mu,
                                float *sigma, float *best, cudaStream_t s);
// tcgen05 BF16 GEMM C = A B^T (gemm_tc.cu); epi: 0 FP32 store, 1 bias+GELU (Z f32 and
// GELU(Z) bf16), 2 bias FP32, 3 C * GELU'(aux) -> bf16.
cudaError_t launch_gemm_bf16(int epi, const void *A, const void *B, int M, int N, int K,
                             float *out_f32, void *out_bf16, int ldo, const float *bias,
                             const float *aux, int *err, cudaStream_t s);
cudaError_t launch_accel_cost(const float *xi, const int *traj_problem, const ProblemDev *problems,
                              const float *tables, int dim, int B, float *out, cudaStream_t s);
// 2D homotopy signatures of the trajectories xi (homotopy.cu): bit j = obstacle j passed
// on the left of the relative motion at the closest approach (j < 64)
cudaError_t launch_homotopy(const float *xi, const int *traj_problem, const ProblemDev *problems,
                            const float *tables, const float *centers, const float *axes,
                            const float *vel, const int *obs_offsets, int n_traj,
                            unsigned long long *sig, cudaStream_t s);
cudaError_t launch_ffma_peak(float *out, int blocks, int iters, cudaStream_t s);
cudaError_t launch_ffma2_peak(float *out, int blocks, int iters, cudaStream_t s);
cudaError_t launch_rsqrt_peak(float *out, int blocks, int iters, cudaStream_t s);
} // namespace tb

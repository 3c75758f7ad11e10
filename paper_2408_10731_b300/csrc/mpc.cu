// mpc.cu -- the receding-horizon step of Paper II's MPC use of Algorithm 2:
// the robot has followed one planned trajectory per problem for delta seconds,
// and the next control loop's solve starts from the previous one's multipliers
// (the paper initialises the Lagrange multipliers with the preceding loop's
// solution). On the device, in FP64:
//
//  * the executed plan of each problem: the caller's choice, or the trajectory
//    with the smallest worst-of-three residual (ties to the lower index), found
//    with a 64-bit atomic minimum of (residual bits, index): non-negative floats
//    order as their bit patterns, and a NaN residual sorts after every number;
//  * every trajectory's polynomial re-expressed on the shifted window: the
//    coefficients of q(tau') = p(f + tau'), f = delta / T, are the blossom
//    (polar form) of p at (f, ..., f, 1 + f, ..., 1 + f) with i arguments 1 + f
//    for coefficient i, each evaluated by de Casteljau's scheme with one
//    parameter per level; past the old end the polynomial is extrapolated;
//  * the executed plan's position, velocity and acceleration at delta: the first
//    three shifted coefficients give q(0), q'(0) = 10 (c1 - c0) and
//    q''(0) = 90 (c2 - 2 c1 + c0), scaled by 1/T and 1/T^2;
//  * every obstacle centre moved on to c + v delta (its constant-velocity
//    prediction; multiply and add rounded separately, then rounded to FP32);
//  * the multipliers copied unchanged.
#include "internal.cuh"

namespace tb {

// Coefficient i of the polynomial with coefficients c re-expressed on [f, 1 + f].
__device__ __forceinline__ double blossom_shift(const double (&c)[NC], int i, double f) {
  double w[NC];
#pragma unroll
  for (int j = 0; j < NC; ++j) w[j] = c[j];
#pragma unroll
  for (int r = 1; r < NC; ++r) {
    const double u = r <= NC - 1 - i ? f : 1.0 + f;
#pragma unroll
    for (int j = 0; j < NC - r; ++j) w[j] = fma(u, w[j + 1] - w[j], w[j]);
  }
  return w[0];
}

__global__ void k_exec_pick(int n_traj, const int *traj_problem, const float *res,
                            unsigned long long *key) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n_traj) return;
  const float r0 = res[b * 3 + 0], r1 = res[b * 3 + 1], r2 = res[b * 3 + 2];
  const float r = fmaxf(fmaxf(r0, r1), r2);
  const bool nan = isnan(r0) || isnan(r1) || isnan(r2); // fmaxf would drop a NaN operand
  const unsigned bits = nan ? 0x7fc00000u : __float_as_uint(r);
  atomicMin(&key[traj_problem[b]], ((unsigned long long)bits << 32) | (unsigned)b);
}

// The executed plan of every problem from its key, which is then cleared for the next
// step (the keys start cleared when the handle is created).
__global__ void k_exec_index(int n_problems, unsigned long long *key, int *exec) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_problems) return;
  const unsigned long long k = key[p];
  exec[p] = k == ~0ull ? -1 : (int)(unsigned)(k & 0xffffffffull);
  key[p] = ~0ull;
}

// One thread per (trajectory, axis, coefficient): xi0 = shifted xi, lam0 = lam.
__device__ __forceinline__ void shift_traj(const ShiftArgs &a, long long e) {
  const long long row = e / NC;
  const int i = (int)(e - row * NC), b = (int)(row / a.dim);
  const double f = a.delta / a.T[a.traj_problem[b]];
  const float *x = a.xi + (size_t)row * NC;
  double c[NC];
#pragma unroll
  for (int j = 0; j < NC; ++j) c[j] = (double)x[j];
  a.xi0[e] = (float)blossom_shift(c, i, f);
  a.lam0[e] = a.lam[e];
}

// One thread per (problem, axis): the executed plan's state at delta becomes the start.
__device__ __forceinline__ void shift_start(const ShiftArgs &a, const int *exec, int e) {
  const int p = e / a.dim, ax = e % a.dim;
  const int b = exec[p];
  if (b < 0) return; // no trajectory of this problem: its start stays
  const double T = a.T[p], f = a.delta / T;
  const float *x = a.xi + ((size_t)b * a.dim + ax) * NC;
  double c[NC];
#pragma unroll
  for (int j = 0; j < NC; ++j) c[j] = (double)x[j];
  const double q0 = blossom_shift(c, 0, f), q1 = blossom_shift(c, 1, f), q2 = blossom_shift(c, 2, f);
  const double v0 = 10.0 * (q1 - q0) / T, a0 = 90.0 * ((q2 - q1) - (q1 - q0)) / (T * T);
  if (!isfinite(q0) || !isfinite(v0) || !isfinite(a0)) return; // a failed plan: keep the start
  a.start[p * a.dim + ax] = q0;
  a.start_va[(p * 2 + 0) * a.dim + ax] = v0;
  a.start_va[(p * 2 + 1) * a.dim + ax] = a0;
}

// The three independent parts of the shift in one launch of small blocks, so that the
// FP64 work spreads over every SM: blocks [0, nb_start) the start states (three blossoms
// each), then the iterates, then the obstacle centres.
constexpr int SHIFT_THREADS = 32;

__global__ void __launch_bounds__(SHIFT_THREADS) k_shift(ShiftArgs a, const int *exec,
                                                         int nb_start, int nb_traj) {
  const int blk = blockIdx.x;
  if (blk < nb_start) {
    const int e = blk * SHIFT_THREADS + threadIdx.x;
    if (e < a.n_problems * a.dim) shift_start(a, exec, e);
  } else if (blk < nb_start + nb_traj) {
    const long long e = (long long)(blk - nb_start) * SHIFT_THREADS + threadIdx.x;
    if (e < (long long)a.n_traj * a.dim * NC) shift_traj(a, e);
  } else {
    const int e = (blk - nb_start - nb_traj) * SHIFT_THREADS + threadIdx.x;
    if (e < a.n_obs * a.dim)
      a.centers[e] = (float)__dadd_rn((double)a.centers[e], __dmul_rn((double)a.velocities[e], a.delta));
  }
}

cudaError_t launch_mpc_shift(const ShiftArgs &a, cudaStream_t s) {
  const int *exec = a.executed;
  if (!exec) {
    k_exec_pick<<<(a.n_traj + 255) / 256, 256, 0, s>>>(a.n_traj, a.traj_problem, a.res,
                                                        a.key_scratch);
    k_exec_index<<<(a.n_problems + 255) / 256, 256, 0, s>>>(a.n_problems, a.key_scratch,
                                                             a.exec_scratch);
    exec = a.exec_scratch;
  }
  const int nb_start = (a.n_problems * a.dim + SHIFT_THREADS - 1) / SHIFT_THREADS;
  const long long n_coef = (long long)a.n_traj * a.dim * NC;
  const int nb_traj = (int)((n_coef + SHIFT_THREADS - 1) / SHIFT_THREADS);
  const int nb_obs = (a.n_obs * a.dim + SHIFT_THREADS - 1) / SHIFT_THREADS;
  k_shift<<<nb_start + nb_traj + nb_obs, SHIFT_THREADS, 0, s>>>(a, exec, nb_start, nb_traj);
  return cudaGetLastError();
}

} // namespace tb

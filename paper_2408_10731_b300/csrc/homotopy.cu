// homotopy.cu -- which side of every obstacle a 2D trajectory passes: the signature
// that tells solutions of one scene apart by homotopy class, so that the labels
// the learned warm start is trained on can cover different classes.
//
// For obstacle j moving as o_j(t) = c_j + v_j t, the trajectory's closest approach
// (in coordinates scaled by the semi-axes, over the grid points) is at t*, and the
// obstacle is on the trajectory's left as they pass when the cross product
// (p - o_j)(t*) x (p' - v_j)(t*) is positive: bit j of the signature is then set.
// Two trajectories of a problem that pass every obstacle on the same sides share
// the signature. Obstacles past the 64th of a problem are not encoded.
#include "trajbatch.h"
#include "internal.cuh"

namespace tb {

// One warp per trajectory: the lanes evaluate p and p' on the grid into shared
// memory, then lane l scans obstacles l and l + 32 over every grid point.
__global__ void k_homotopy(const float *xi, const int *traj_problem, const ProblemDev *problems,
                           const float *tables, const float *centers, const float *axes,
                           const float *vel, const int *obs_offsets, int n_traj,
                           unsigned long long *sig) {
  extern __shared__ float hs[];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int b = blockIdx.x * (blockDim.x >> 5) + wib;
  if (b >= n_traj) return;
  const ProblemDev pr = problems[traj_problem[b]];
  const int n_p = pr.n_p;
  float *pv = hs + (size_t)wib * 4 * MAX_STEPS; // x, y, x', y' per grid point
  const float *tP = tables + pr.tbl_off, *tD = tP + n_p * ROW;
  const float *x = xi + (size_t)b * 2 * NC;
  for (int t = lane; t < n_p; t += 32) {
    float px = 0.f, py = 0.f, vx = 0.f, vy = 0.f;
    for (int i = 0; i < NC; ++i) {
      px = fmaf(tP[t * ROW + i], x[i], px);
      py = fmaf(tP[t * ROW + i], x[NC + i], py);
      vx = fmaf(tD[t * ROW + i], x[i], vx);
      vy = fmaf(tD[t * ROW + i], x[NC + i], vy);
    }
    pv[4 * t + 0] = px; pv[4 * t + 1] = py;
    pv[4 * t + 2] = vx * pr.invT; pv[4 * t + 3] = vy * pr.invT;
  }
  __syncwarp();
  const int o0 = obs_offsets[traj_problem[b]];
  unsigned long long bits = 0ull;
  for (int j = lane; j < pr.n_o && j < 64; j += 32) {
    const int o = o0 + j;
    const float cx = centers[2 * o], cy = centers[2 * o + 1];
    const float ax = axes[2 * o], ay = axes[2 * o + 1];
    const float ux = vel[2 * o], uy = vel[2 * o + 1];
    float best = 3.0e38f;
    int tb_ = 0;
    for (int t = 0; t < n_p; ++t) {
      const float tm = pr.dt * (float)t;
      const float dx = (pv[4 * t] - fmaf(ux, tm, cx)) / ax, dy = (pv[4 * t + 1] - fmaf(uy, tm, cy)) / ay;
      const float d2 = dx * dx + dy * dy;
      if (d2 < best) { best = d2; tb_ = t; }
    }
    const float tm = pr.dt * (float)tb_;
    const float dx = pv[4 * tb_] - fmaf(ux, tm, cx), dy = pv[4 * tb_ + 1] - fmaf(uy, tm, cy);
    const float rx = pv[4 * tb_ + 2] - ux, ry = pv[4 * tb_ + 3] - uy;
    if (dx * ry - dy * rx > 0.f) bits |= 1ull << j;
  }
  // OR the lanes' bits
  for (int s = 16; s >= 1; s >>= 1) bits |= __shfl_xor_sync(0xffffffffu, bits, s);
  if (lane == 0) sig[b] = bits;
}

cudaError_t launch_homotopy(const float *xi, const int *traj_problem, const ProblemDev *problems,
                            const float *tables, const float *centers, const float *axes,
                            const float *vel, const int *obs_offsets, int n_traj,
                            unsigned long long *sig, cudaStream_t s) {
  if (n_traj <= 0) return cudaSuccess;
  const int warps = 4;
  const size_t smem = sizeof(float) * 4 * MAX_STEPS * warps;
  k_homotopy<<<(n_traj + warps - 1) / warps, 32 * warps, smem, s>>>(
      xi, traj_problem, problems, tables, centers, axes, vel, obs_offsets, n_traj, sig);
  return cudaGetLastError();
}

} // namespace tb

// noalloc.cu -- traj_solve_noalloc: the whole solve (set-up and iteration)
// without any device allocation, for callers that cannot allocate memory.
//
// Who needs it: code that runs where cudaMalloc is unavailable or forbidden --
// inside a memory pool that must not grow, under an allocator that another
// framework owns, in a plugin that may only use the buffers its host hands
// it, or on a real-time path where an allocation could stall. Such callers
// cannot create a traj_batch handle (it allocates its workspace), so this
// entry point keeps every intermediate in one file-scope device array of fixed
// size instead.
//
// The scratch array below is reserved in every GPU that loads the library and
// stays reserved until the process exits. In host code its name is only a
// host-side stand-in, never a device address: the device address is fetched
// once per device with cudaGetSymbolAddress (with that device current) and
// passed to the kernels.
#include "trajbatch.h"
#include "internal.cuh"

#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>

namespace tb {
void set_thread_error(const std::string &msg); // trajbatch.cu: read by traj_last_error(NULL)
}

using namespace tb;

namespace {

// Limits of one call (the scratch layout is sized for exactly these).
constexpr int NA_MAX_PROBLEMS = 256;
constexpr int NA_MAX_OBSTACLES = 8192;
constexpr int NA_MAX_TRAJ = 8192;
constexpr int NA_MAX_TABLE_FLOATS = 160 * 1024 / 4; // basis tables of all distinct horizons

// Scratch layout (byte offsets, each 256-aligned).
constexpr size_t al(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t OFF_PROBLEMS = 0;
constexpr size_t OFF_T = al(OFF_PROBLEMS + sizeof(ProblemDev) * NA_MAX_PROBLEMS);
constexpr size_t OFF_START = al(OFF_T + sizeof(double) * NA_MAX_PROBLEMS);
constexpr size_t OFF_GOAL = al(OFF_START + sizeof(double) * 3 * NA_MAX_PROBLEMS);
constexpr size_t OFF_CONST = al(OFF_GOAL + sizeof(double) * 3 * NA_MAX_PROBLEMS);
constexpr size_t OFF_TABLES = al(OFF_CONST + sizeof(float) * CONST_FLOATS * NA_MAX_PROBLEMS);
constexpr size_t OFF_HZ = al(OFF_TABLES + sizeof(float) * NA_MAX_TABLE_FLOATS);
constexpr size_t OFF_HOFF = al(OFF_HZ + sizeof(int) * (MAX_STEPS + 1));
constexpr size_t OFF_OFFSETS = al(OFF_HOFF + sizeof(int) * (MAX_STEPS + 1));
constexpr size_t OFF_OBS = al(OFF_OFFSETS + sizeof(int) * (NA_MAX_PROBLEMS + 1));
constexpr size_t OFF_PAIR_OFF = al(OFF_OBS + sizeof(float4) * pair_vec(3) *
                                             ((NA_MAX_OBSTACLES + NA_MAX_PROBLEMS) / 2 + 1));
constexpr size_t OFF_ORDER = al(OFF_PAIR_OFF + sizeof(int) * (NA_MAX_PROBLEMS + 1));
constexpr size_t OFF_WORDS = al(OFF_ORDER + sizeof(int) * NA_MAX_TRAJ); // queue, flags, t0
constexpr size_t SCRATCH_BYTES = al(OFF_WORDS + 64);                    // about 1.4 MB

} // namespace

// The scratch itself: every call on a device shares it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

namespace {

std::mutex g_mu;
void *g_scratch_dev[64] = {}; // device address of g_noalloc_scratch, per device ordinal

// First call on a device: look up the array's device address with the device current.
cudaError_t scratch_address(int dev, unsigned char **out) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!g_scratch_dev[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_dev[dev] = p;
  }
  *out = static_cast<unsigned char *>(g_scratch_dev[dev]);
  return cudaSuccess;
}

// order[k] = k (the queue runs the trajectories in index order), and the range
// check of the caller's trajectory -> problem map, which lives in device memory:
// an entry outside [0, n_problems) sets bit 4 of *flags and nothing reads through it
// (the host looks at the flag before it launches anything that would).
__global__ void k_noalloc_order(int n_traj, const int *traj_problem, int n_problems, int *order,
                                int *flags) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_traj) return;
  order[i] = i;
  const int p = traj_problem[i];
  if (p < 0 || p >= n_problems) atomicOr(flags, 16);
}

traj_status err(traj_status s, const std::string &msg) {
  set_thread_error(msg);
  return s;
}

} // namespace

#define NA_CK(expr)                                                                  \
  do {                                                                               \
    cudaError_t _e = (expr);                                                         \
    if (_e != cudaSuccess) return err(TRAJ_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
  } while (0)

extern "C" traj_status traj_solve_noalloc(
    const traj_config *cfg, int n_problems, const int *n_steps, const double *duration,
    const double *start, const double *goal, const int *obs_offsets, const float *centers,
    const float *semi_axes, const float *velocities, int n_traj, const int *traj_problem,
    const float *coeffs0, int max_iters, float tol, float *coeffs, float *residual, int *iters,
    signed char *status) {
  set_thread_error("");
  if (!cfg || !n_steps || !duration || !start || !goal || !obs_offsets || !traj_problem ||
      !coeffs0 || !coeffs || !residual || !iters || !status)
    return err(TRAJ_EINVAL, "NULL argument");
  const traj_config &c = *cfg;
  const int D = c.dim;
  if ((D != 2 && D != 3) || c.degree != 10) return err(TRAJ_EINVAL, "dim must be 2 or 3, degree 10");
  if (!(c.vmax > 0) || !(c.amax > 0) || !(c.rho > 0) || !(c.w_smooth >= 0) || !(c.w_track >= 0))
    return err(TRAJ_EINVAL, "vmax, amax, rho must be positive; weights non-negative");
  if (c.cost_mode != TRAJ_COST_SMOOTH_TRACK && c.cost_mode != TRAJ_COST_PROJECT)
    return err(TRAJ_EINVAL, "unknown cost mode");
  if (c.precision != TRAJ_PREC_FP32) return err(TRAJ_EINVAL, "traj_solve_noalloc runs the FP32 form only");
  if (max_iters < 0 || std::isnan(tol)) return err(TRAJ_EINVAL, "bad max_iters or tol");
  if (n_problems < 1 || n_problems > NA_MAX_PROBLEMS)
    return err(TRAJ_ESHAPE, "traj_solve_noalloc: n_problems must be in [1, 256]");
  if (n_traj < 1 || n_traj > NA_MAX_TRAJ)
    return err(TRAJ_ESHAPE, "traj_solve_noalloc: n_traj must be in [1, 8192]");
  if (obs_offsets[0] != 0) return err(TRAJ_EINVAL, "offsets[0] must be 0");
  for (int p = 0; p < n_problems; ++p)
    if (obs_offsets[p + 1] < obs_offsets[p]) return err(TRAJ_EINVAL, "offsets must be non-decreasing");
  const int N = obs_offsets[n_problems];
  if (N > NA_MAX_OBSTACLES) return err(TRAJ_ESHAPE, "traj_solve_noalloc: at most 8192 obstacles in total");
  if (N > 0 && (!centers || !semi_axes || !velocities)) return err(TRAJ_EINVAL, "NULL obstacle array");

  // problem records and distinct horizons, on the stack (no host allocation either)
  int hz[MAX_STEPS + 1], hoff[MAX_STEPS + 1], n_hz = 0, max_np = 0;
  bool seen[MAX_STEPS + 1] = {};
  for (int p = 0; p < n_problems; ++p) {
    if (n_steps[p] < 2 || n_steps[p] > MAX_STEPS) return err(TRAJ_ESHAPE, "n_steps out of [2, 256]");
    if (!(duration[p] > 0) || !std::isfinite(duration[p])) return err(TRAJ_EINVAL, "duration must be positive");
    for (int d = 0; d < D; ++d)
      if (!std::isfinite(start[p * D + d]) || !std::isfinite(goal[p * D + d]))
        return err(TRAJ_ENAN, "non-finite start/goal");
    seen[n_steps[p]] = true;
    max_np = std::max(max_np, n_steps[p]);
  }
  int tot = 0;
  for (int n = 2; n <= MAX_STEPS; ++n)
    if (seen[n]) { hz[n_hz] = n; hoff[n_hz] = tot; tot += table_floats(n); ++n_hz; }
  if (tot > NA_MAX_TABLE_FLOATS) return err(TRAJ_ESHAPE, "too many distinct horizons (tables > 160 KB)");
  ProblemDev recs[NA_MAX_PROBLEMS];
  int pair_off[NA_MAX_PROBLEMS + 1];
  pair_off[0] = 0;
  for (int p = 0; p < n_problems; ++p)
    pair_off[p + 1] = pair_off[p] + pair_count(obs_offsets[p + 1] - obs_offsets[p]);
  for (int p = 0; p < n_problems; ++p) {
    ProblemDev r{};
    r.n_p = n_steps[p];
    r.n_o = obs_offsets[p + 1] - obs_offsets[p];
    r.pair_off = pair_off[p];
    for (int h = 0; h < n_hz; ++h)
      if (hz[h] == r.n_p) r.tbl_off = hoff[h];
    const double T = duration[p];
    r.dt = (float)(T / (double)(r.n_p - 1));
    r.invT = (float)(1.0 / T);
    r.invT2 = (float)(1.0 / (T * T));
    r.const_off = p * CONST_FLOATS;
    recs[p] = r;
  }

  int dev = 0, n_sm = 0;
  NA_CK(cudaGetDevice(&dev));
  NA_CK(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
  unsigned char *S = nullptr;
  NA_CK(scratch_address(dev, &S));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(c.cuda_stream);
  ProblemDev *d_problems = reinterpret_cast<ProblemDev *>(S + OFF_PROBLEMS);
  double *d_T = reinterpret_cast<double *>(S + OFF_T);
  double *d_start = reinterpret_cast<double *>(S + OFF_START);
  double *d_goal = reinterpret_cast<double *>(S + OFF_GOAL);
  float *d_const = reinterpret_cast<float *>(S + OFF_CONST);
  float *d_tables = reinterpret_cast<float *>(S + OFF_TABLES);
  int *d_hz = reinterpret_cast<int *>(S + OFF_HZ);
  int *d_hoff = reinterpret_cast<int *>(S + OFF_HOFF);
  int *d_offsets = reinterpret_cast<int *>(S + OFF_OFFSETS);
  float4 *d_obs = reinterpret_cast<float4 *>(S + OFF_OBS);
  int *d_pair_off = reinterpret_cast<int *>(S + OFF_PAIR_OFF);
  int *d_order = reinterpret_cast<int *>(S + OFF_ORDER);
  int *d_words = reinterpret_cast<int *>(S + OFF_WORDS);

  // the array keeps the previous call's contents: everything below is rewritten,
  // and the counters that must start at zero are cleared
  NA_CK(cudaMemcpyAsync(d_problems, recs, sizeof(ProblemDev) * n_problems, cudaMemcpyHostToDevice, s));
  NA_CK(cudaMemcpyAsync(d_T, duration, sizeof(double) * n_problems, cudaMemcpyHostToDevice, s));
  NA_CK(cudaMemcpyAsync(d_start, start, sizeof(double) * n_problems * D, cudaMemcpyHostToDevice, s));
  NA_CK(cudaMemcpyAsync(d_goal, goal, sizeof(double) * n_problems * D, cudaMemcpyHostToDevice, s));
  NA_CK(cudaMemcpyAsync(d_hz, hz, sizeof(int) * n_hz, cudaMemcpyHostToDevice, s));
  NA_CK(cudaMemcpyAsync(d_hoff, hoff, sizeof(int) * n_hz, cudaMemcpyHostToDevice, s));
  NA_CK(cudaMemcpyAsync(d_offsets, obs_offsets, sizeof(int) * (n_problems + 1), cudaMemcpyHostToDevice, s));
  NA_CK(cudaMemcpyAsync(d_pair_off, pair_off, sizeof(int) * (n_problems + 1), cudaMemcpyHostToDevice, s));
  NA_CK(cudaMemsetAsync(d_words, 0, 64, s));
  k_noalloc_order<<<(n_traj + 255) / 256, 256, 0, s>>>(n_traj, traj_problem, n_problems, d_order,
                                                         d_words + 1);
  NA_CK(cudaGetLastError());
  int flags = 0;
  NA_CK(cudaMemcpyAsync(&flags, d_words + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
  NA_CK(cudaStreamSynchronize(s));
  if (flags & 16) return err(TRAJ_EINVAL, "traj_solve_noalloc: a traj_problem entry is outside [0, n_problems)");
  NA_CK(launch_setup_tables(d_hz, d_hoff, n_hz, d_tables, s));
  NA_CK(launch_pack_obstacles(D, n_problems, 2 * pair_off[n_problems], d_offsets, d_pair_off,
                              centers, semi_axes, velocities, d_obs, d_problems, s));
  NA_CK(launch_setup_problems(d_problems, n_problems, d_T, d_start, d_goal, nullptr, D, c.rho,
                              c.w_smooth, c.w_track, c.cost_mode, max_np, d_const, s));
  SolveArgs a{};
  a.problems = d_problems;
  a.obstacles = d_obs;
  a.constants = d_const;
  a.tables = d_tables;
  a.table_floats_total = tot;
  a.traj_problem = traj_problem;
  a.order = d_order;
  a.xi0 = coeffs0;
  a.xi = coeffs;
  a.lam = nullptr;
  a.u = nullptr;
  a.res = residual;
  a.iters = iters;
  a.status = status;
  a.n_traj = n_traj;
  a.max_iters = max_iters;
  a.tol = tol;
  a.rho = (float)c.rho;
  a.vmax = (float)c.vmax;
  a.amax = (float)c.amax;
  a.cost_mode = c.cost_mode;
  a.timeout_ns = 0;
  a.queue = d_words;
  a.flags = d_words + 1;
  a.t0 = reinterpret_cast<unsigned long long *>(d_words + 2);
  // four warps per block, one warp per trajectory
  LaunchShape shape{};
  shape.warps_per_block = 4;
  shape.team = 1;
  NA_CK(launch_am_solve(D, max_np, TRAJ_PREC_FP32, a, shape, n_sm, s, nullptr));
  // the host-side sources above live on this stack frame: finish before returning
  NA_CK(cudaMemcpyAsync(&flags, d_words + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
  NA_CK(cudaStreamSynchronize(s));
  if (flags & 2) return err(TRAJ_ENAN, "non-finite input in some trajectories");
  return TRAJ_OK;
}

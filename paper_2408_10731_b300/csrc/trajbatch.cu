// trajbatch.cu -- host side of the C ABI declared in include/trajbatch.h.
//
// Validation, workspace ownership, copies on the caller's stream and kernel
// launches. Every step of the method itself runs in the kernels of setup.cu
// (FP64 set-up) and am_solve.cu (the iteration); this file only marshals.
#include "trajbatch.h"
#include "internal.cuh"
#include "nvtx_range.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

using namespace tb;

// What a captured solve graph was built for; the graph is replayed while it matches.
struct GraphKey {
  int max_iters = -1, n_traj = -1, warps = -1, bps = -1, team = -1, occ = -1, resume = -1;
  float tol = 0.f;
  unsigned long long timeout = 0;
  bool operator==(const GraphKey &o) const {
    return max_iters == o.max_iters && n_traj == o.n_traj && warps == o.warps && bps == o.bps &&
           team == o.team && occ == o.occ && resume == o.resume && tol == o.tol &&
           timeout == o.timeout;
  }
};

struct traj_batch {
  traj_config cfg{};
  cudaStream_t stream = nullptr;
  std::string err;
  int n_sm = 0;
  int n_problems = 0, n_traj = 0, n_obs = 0, max_np_used = 0;
  bool have_problems = false, have_obstacles = false, have_initial = false, have_result = false;
  std::vector<int> n_steps;
  std::vector<double> duration;
  std::vector<int> obs_offsets;
  std::vector<int> traj_problem;
  // device workspace
  ProblemDev *d_problems = nullptr;
  double *d_T = nullptr, *d_start = nullptr, *d_goal = nullptr;
  double *d_start_va = nullptr;               // [P][2][dim] start velocity, acceleration
  int *d_exec = nullptr;                      // receding-horizon step: executed plan per problem
  unsigned long long *d_exec_key = nullptr;
  unsigned long long *d_sig = nullptr;        // homotopy signatures [B]
  float *d_constants = nullptr;
  int const_levels = 1;                       // constants blocks allocated per problem
  // FP64 K11, K12 and basis moments per problem and level (receding-horizon shifts:
  // allocated at the first one; valid while the problems, obstacles, penalties and
  // workspace bounds stay as they were set up)
  double *d_kkt64 = nullptr;
  size_t kkt64_cap = 0;
  bool kkt_valid = false;
  // penalty continuation (traj_set_rho_schedule): levels, growth per level, switch period
  int rho_levels = 1, rho_every = 0;
  double rho_growth = 1.0;
  float *d_rho_ladder = nullptr;
  std::vector<ProblemDev> recs;               // problem records as uploaded (nan flags cleared)
  std::vector<double> box_lo, box_hi;         // workspace bounds [P][dim] (empty: none)
  std::vector<int> pair_index;                // CSR offsets and first pair record per problem
  float *d_tables = nullptr;
  int table_floats = 0, table_cap = 0;
  int *d_horizons = nullptr, *d_hoffsets = nullptr;
  float4 *d_obs = nullptr;
  float *d_obs_stage = nullptr;
  int *d_obs_index = nullptr; // CSR obstacle offsets [P + 1], then first pair record [P + 1]
  int *d_traj_problem = nullptr, *d_order = nullptr;
  float *d_xi0 = nullptr, *d_xi = nullptr, *d_lam = nullptr, *d_u = nullptr, *d_res = nullptr;
  float *d_lam0 = nullptr, *d_u0 = nullptr; // imported state (traj_set_state)
  bool resume = false;                       // the next solves continue the imported state
  bool carry = false;                        // the next solves start from the shifted iterate
                                             // and the carried multipliers
  int *d_iters = nullptr;
  signed char *d_status = nullptr;
  int *d_queue = nullptr, *d_flags = nullptr;
  unsigned long long *d_t0 = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // launch shape of the solve (set by traj_autotune / traj_set_launch_shape)
  LaunchShape shape{0, 0, 0, 1};
  LaunchShape used{0, 0, 0, 0}; // what the last captured solve launch resolved the shape to
  // the solve captured as a CUDA graph, replayed while its key is unchanged
  cudaStream_t capture_stream = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  bool graph_valid = false;
  GraphKey g_key;
  // one receding-horizon control step (shift, boundary update, solve) as a CUDA graph
  cudaGraphExec_t mpc_exec = nullptr;
  bool mpc_valid = false;
  GraphKey mpc_key;
  double mpc_delta = 0.0;
  bool mpc_given = false;
  std::vector<int> tbl_off; // per problem, float offset of its basis tables
  // sampler scratch (allocated at creation from max_traj)
  float *d_L = nullptr, *d_r = nullptr, *d_caug = nullptr, *d_refit = nullptr;
  int *d_proj = nullptr, *d_elite = nullptr, *d_sflag = nullptr;
};

static thread_local std::string g_create_error;

namespace tb {
// Error detail of calls that have no handle (creation, traj_solve_noalloc).
void set_thread_error(const std::string &msg) { g_create_error = msg; }
} // namespace tb

#define CK(b, expr)                                                                     \
  do {                                                                                  \
    cudaError_t _e = (expr);                                                            \
    if (_e != cudaSuccess) {                                                            \
      (b)->err = std::string(#expr) + ": " + cudaGetErrorString(_e);                    \
      return TRAJ_ECUDA;                                                                \
    }                                                                                   \
  } while (0)

static traj_status fail(traj_batch *b, traj_status s, const std::string &msg) {
  if (b) b->err = msg;
  return s;
}

static bool is_host_ptr(const void *p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeUnregistered;
}

template <class T> static cudaError_t dalloc(T **p, size_t n) {
  return cudaMalloc(reinterpret_cast<void **>(p), sizeof(T) * (n > 0 ? n : 1));
}

static void free_all(traj_batch *b) {
  void *ptrs[] = {b->d_problems, b->d_T, b->d_start, b->d_goal, b->d_start_va, b->d_exec,
                  b->d_exec_key, b->d_sig, b->d_constants, b->d_rho_ladder, b->d_tables,
                  b->d_horizons, b->d_hoffsets, b->d_obs, b->d_obs_stage, b->d_obs_index,
                  b->d_traj_problem, b->d_order, b->d_xi0, b->d_xi, b->d_lam, b->d_u, b->d_res, b->d_lam0, b->d_u0,
                  b->d_iters, b->d_status, b->d_queue, b->d_flags, b->d_t0, b->d_L, b->d_r,
                  b->d_caug, b->d_proj, b->d_elite, b->d_sflag, b->d_kkt64, b->d_refit};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  if (b->ev0) cudaEventDestroy(b->ev0);
  if (b->ev1) cudaEventDestroy(b->ev1);
  if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
  if (b->mpc_exec) cudaGraphExecDestroy(b->mpc_exec);
  if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
}

static void drop_solve_graph(traj_batch *b) {
  if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
  b->graph_exec = nullptr;
  b->graph_valid = false;
}

// Drop the captured graphs (the solve's and the control step's): their nodes hold the
// buffers and arguments of the handle's state at capture.
static void invalidate_graph(traj_batch *b) {
  drop_solve_graph(b);
  if (b->mpc_exec) cudaGraphExecDestroy(b->mpc_exec);
  b->mpc_exec = nullptr;
  b->mpc_valid = false;
}

extern "C" {

const char *traj_status_string(traj_status s) {
  switch (s) {
  case TRAJ_OK: return "TRAJ_OK";
  case TRAJ_NOT_CONVERGED: return "TRAJ_NOT_CONVERGED";
  case TRAJ_EINVAL: return "TRAJ_EINVAL";
  case TRAJ_ENOMEM: return "TRAJ_ENOMEM";
  case TRAJ_ECUDA: return "TRAJ_ECUDA";
  case TRAJ_ESHAPE: return "TRAJ_ESHAPE";
  case TRAJ_ETIMEOUT: return "TRAJ_ETIMEOUT";
  case TRAJ_ENAN: return "TRAJ_ENAN";
  case TRAJ_ESTATE: return "TRAJ_ESTATE";
  }
  return "TRAJ_UNKNOWN";
}

const char *traj_last_error(traj_batch *b) {
  return b ? b->err.c_str() : g_create_error.c_str();
}

traj_status traj_batch_create(const traj_config *cfg, traj_batch **out) {
  g_create_error.clear();
  if (!cfg || !out) { g_create_error = "NULL config or output pointer"; return TRAJ_EINVAL; }
  const traj_config &c = *cfg;
  if (c.dim != 2 && c.dim != 3) { g_create_error = "dim must be 2 or 3"; return TRAJ_EINVAL; }
  if (c.degree != 10) { g_create_error = "degree must be 10"; return TRAJ_EINVAL; }
  if (c.max_problems < 1 || c.max_traj < 1 || c.max_obstacles < 0 || c.max_steps < 2 ||
      c.max_steps > MAX_STEPS_LONG) {
    g_create_error = "capacities out of range (max_steps must be in [2, 1024])";
    return TRAJ_EINVAL;
  }
  if (!(c.vmax > 0) || !(c.amax > 0) || !(c.rho > 0) || !(c.w_smooth >= 0) || !(c.w_track >= 0) ||
      !std::isfinite(c.vmax) || !std::isfinite(c.amax) || !std::isfinite(c.rho)) {
    g_create_error = "vmax, amax, rho must be positive and finite; weights non-negative";
    return TRAJ_EINVAL;
  }
  if (c.precision != TRAJ_PREC_FP32 && c.precision != TRAJ_PREC_MIXED &&
      c.precision != TRAJ_PREC_MIXED_SPLIT) {
    g_create_error = "unknown precision";
    return TRAJ_EINVAL;
  }
  if (c.cost_mode != TRAJ_COST_SMOOTH_TRACK && c.cost_mode != TRAJ_COST_PROJECT) {
    g_create_error = "unknown cost mode";
    return TRAJ_EINVAL;
  }
  int dev = 0, n_dev = 0;
  cudaError_t e = cudaGetDeviceCount(&n_dev);
  if (e != cudaSuccess || n_dev < 1) {
    cudaGetLastError();
    g_create_error = std::string("no CUDA device: ") + cudaGetErrorString(e);
    return TRAJ_ECUDA;
  }
  traj_batch *b = new (std::nothrow) traj_batch();
  if (!b) { g_create_error = "host allocation failed"; return TRAJ_ENOMEM; }
  b->cfg = c;
  b->stream = reinterpret_cast<cudaStream_t>(c.cuda_stream);
  auto bail = [&](const char *what, cudaError_t err) {
    g_create_error = std::string(what) + ": " + cudaGetErrorString(err);
    free_all(b);
    delete b;
    return err == cudaErrorMemoryAllocation ? TRAJ_ENOMEM : TRAJ_ECUDA;
  };
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return bail("cudaGetDevice", e);
  if ((e = cudaDeviceGetAttribute(&b->n_sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return bail("cudaDeviceGetAttribute", e);
  const size_t P = c.max_problems, B = c.max_traj, N = c.max_obstacles, D = c.dim;
  if ((e = dalloc(&b->d_problems, P)) || (e = dalloc(&b->d_T, P)) || (e = dalloc(&b->d_start, P * D)) ||
      (e = dalloc(&b->d_goal, P * D)) || (e = dalloc(&b->d_start_va, P * 2 * D)) ||
      (e = dalloc(&b->d_exec, P)) || (e = dalloc(&b->d_exec_key, P)) || (e = dalloc(&b->d_sig, B)) ||
      (e = dalloc(&b->d_constants, P * CONST_FLOATS)) ||
      (e = dalloc(&b->d_rho_ladder, RHO_MAX_LEVELS)) ||
      (e = dalloc(&b->d_horizons, MAX_STEPS_LONG + 1)) || (e = dalloc(&b->d_hoffsets, MAX_STEPS_LONG + 1)) ||
      (e = dalloc(&b->d_obs, ((N + P) / 2 + 1) * pair_vec(c.dim))) ||
      (e = dalloc(&b->d_obs_stage, 3 * N * D)) || (e = dalloc(&b->d_obs_index, 2 * (P + 1))) || (e = dalloc(&b->d_traj_problem, B)) ||
      (e = dalloc(&b->d_order, B)) || (e = dalloc(&b->d_xi0, B * D * NC)) ||
      (e = dalloc(&b->d_xi, B * D * NC)) || (e = dalloc(&b->d_lam, B * D * NC)) ||
      (e = dalloc(&b->d_u, B * D * NC)) || (e = dalloc(&b->d_res, B * 3)) ||
      (e = dalloc(&b->d_lam0, B * D * NC)) || (e = dalloc(&b->d_u0, B * D * NC)) ||
      (e = dalloc(&b->d_iters, B)) || (e = dalloc(&b->d_status, B)) || (e = dalloc(&b->d_queue, 1)) ||
      (e = dalloc(&b->d_flags, 1)) || (e = dalloc(&b->d_t0, 1)) || (e = dalloc(&b->d_L, TRAJ_SAMPLER_MAX_DIST * (D * NC) * (D * NC))) ||
      (e = dalloc(&b->d_r, B)) || (e = dalloc(&b->d_caug, B)) || (e = dalloc(&b->d_proj, B)) ||
      (e = dalloc(&b->d_elite, B)) || (e = dalloc(&b->d_sflag, 1)) ||
      (e = dalloc(&b->d_refit, TRAJ_SAMPLER_MAX_DIST * (D * NC + 7) + 2 * B * D * NC)))
    return bail("cudaMalloc", e);
  // the executed-plan keys start cleared; each receding-horizon step clears them again
  // after reading them
  if ((e = cudaMemset(b->d_exec_key, 0xff, sizeof(unsigned long long) * P)) != cudaSuccess)
    return bail("cudaMemset", e);
  if ((e = cudaEventCreate(&b->ev0)) || (e = cudaEventCreate(&b->ev1))) return bail("cudaEventCreate", e);
  if ((e = cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking)))
    return bail("cudaStreamCreateWithFlags", e);
  *out = b;
  return TRAJ_OK;
}

traj_status traj_batch_destroy(traj_batch *b) {
  if (!b) return TRAJ_OK;
  cudaStreamSynchronize(b->stream);
  free_all(b);
  delete b;
  return TRAJ_OK;
}

traj_status traj_set_problems(traj_batch *b, int n_problems, const int *n_steps,
                              const double *duration, const double *start, const double *goal) {
  tb::NvtxRange nvtx_range("traj_set_problems");
  if (!b) return TRAJ_EINVAL;
  if (!n_steps || !duration || !start || !goal) return fail(b, TRAJ_EINVAL, "NULL problem array");
  if (n_problems < 1 || n_problems > b->cfg.max_problems)
    return fail(b, TRAJ_ESHAPE, "n_problems exceeds max_problems (or < 1)");
  const int D = b->cfg.dim;
  int max_np = 0;
  for (int p = 0; p < n_problems; ++p) {
    if (n_steps[p] < 2 || n_steps[p] > b->cfg.max_steps)
      return fail(b, TRAJ_ESHAPE, "n_steps out of [2, max_steps] for problem " + std::to_string(p));
    if (!(duration[p] > 0) || !std::isfinite(duration[p]))
      return fail(b, TRAJ_EINVAL, "duration must be positive and finite");
    for (int d = 0; d < D; ++d)
      if (!std::isfinite(start[p * D + d]) || !std::isfinite(goal[p * D + d]))
        return fail(b, TRAJ_ENAN, "non-finite start/goal for problem " + std::to_string(p));
    max_np = std::max(max_np, n_steps[p]);
  }
  // distinct horizons -> table offsets (tables staged to shared memory by the solve)
  std::vector<int> hz(n_steps, n_steps + n_problems);
  std::sort(hz.begin(), hz.end());
  hz.erase(std::unique(hz.begin(), hz.end()), hz.end());
  std::vector<int> hoff(hz.size());
  int tot = 0;
  for (size_t h = 0; h < hz.size(); ++h) { hoff[h] = tot; tot += table_floats(hz[h]); }
  if ((size_t)tot * sizeof(float) > 160 * 1024)
    return fail(b, TRAJ_ESHAPE, "too many distinct horizons: basis tables exceed 160 KB");
  if (tot > b->table_cap) {
    if (b->d_tables) cudaFree(b->d_tables);
    b->d_tables = nullptr;
    CK(b, dalloc(&b->d_tables, tot));
    b->table_cap = tot;
  }
  b->table_floats = tot;
  CK(b, cudaMemcpyAsync(b->d_horizons, hz.data(), sizeof(int) * hz.size(), cudaMemcpyHostToDevice, b->stream));
  CK(b, cudaMemcpyAsync(b->d_hoffsets, hoff.data(), sizeof(int) * hz.size(), cudaMemcpyHostToDevice, b->stream));
  CK(b, cudaMemcpyAsync(b->d_T, duration, sizeof(double) * n_problems, cudaMemcpyHostToDevice, b->stream));
  CK(b, cudaMemcpyAsync(b->d_start, start, sizeof(double) * n_problems * D, cudaMemcpyHostToDevice, b->stream));
  CK(b, cudaMemcpyAsync(b->d_goal, goal, sizeof(double) * n_problems * D, cudaMemcpyHostToDevice, b->stream));
  CK(b, cudaMemsetAsync(b->d_start_va, 0, sizeof(double) * n_problems * 2 * D, b->stream)); // at rest
  CK(b, launch_setup_tables(b->d_horizons, b->d_hoffsets, (int)hz.size(), b->d_tables, b->stream));
  CK(b, cudaStreamSynchronize(b->stream)); // host arrays may be reused by the caller
  b->n_steps.assign(n_steps, n_steps + n_problems);
  b->duration.assign(duration, duration + n_problems);
  b->n_problems = n_problems;
  b->kkt_valid = false; // new problems: the set-up with their obstacles keeps new blocks
  b->max_np_used = max_np;
  b->have_problems = true;
  invalidate_graph(b);
  b->have_obstacles = false;
  b->box_lo.clear();
  b->box_hi.clear();
  b->have_result = false;
  b->err.clear();
  return TRAJ_OK;
}

// Upload the problem records (constants offsets for the current number of penalty
// levels), pack the staged obstacles into pair records (which also flags bad
// obstacle data) and form the FP64 set-up of every penalty level; synchronises.
// The FP64 blocks (K11, K12 and the basis moments of every problem and level) are
// kept, so that receding-horizon shifts update only the boundary-dependent constants.
static traj_status upload_problems(traj_batch *b) {
  const int P = b->n_problems, D = b->cfg.dim, N = b->n_obs, L = b->rho_levels;
  b->kkt_valid = false;
  if (b->kkt64_cap < (size_t)P * L * KKT64_DOUBLES) {
    CK(b, cudaStreamSynchronize(b->stream));
    if (b->d_kkt64) cudaFree(b->d_kkt64);
    b->d_kkt64 = nullptr;
    b->kkt64_cap = 0;
    cudaError_t e = dalloc(&b->d_kkt64, (size_t)P * L * KKT64_DOUBLES);
    if (e != cudaSuccess) return fail(b, e == cudaErrorMemoryAllocation ? TRAJ_ENOMEM : TRAJ_ECUDA,
                                      std::string("cudaMalloc: ") + cudaGetErrorString(e));
    b->kkt64_cap = (size_t)P * L * KKT64_DOUBLES;
  }
  const bool box = !b->box_lo.empty();
  for (int p = 0; p < P; ++p) {
    b->recs[p].const_off = p * CONST_FLOATS * L;
    b->recs[p].nan_flag = 0;
    b->recs[p].box = box ? 1 : 0;
    for (int a = 0; a < 3; ++a) {
      b->recs[p].lo[a] = box && a < D ? (float)b->box_lo[(size_t)p * D + a] : 0.f;
      b->recs[p].hi[a] = box && a < D ? (float)b->box_hi[(size_t)p * D + a] : 0.f;
    }
  }
  std::vector<float> ladder(RHO_MAX_LEVELS, 0.f);
  for (int l = 0; l < L; ++l) ladder[l] = (float)(b->cfg.rho * std::pow(b->rho_growth, (double)l));
  const float *st_c = b->d_obs_stage, *st_a = st_c + (size_t)N * D, *st_v = st_a + (size_t)N * D;
  const int *index = b->pair_index.data();
  CK(b, cudaMemcpyAsync(b->d_problems, b->recs.data(), sizeof(ProblemDev) * P, cudaMemcpyHostToDevice, b->stream));
  CK(b, cudaMemcpyAsync(b->d_obs_index, index, sizeof(int) * 2 * (P + 1), cudaMemcpyHostToDevice, b->stream));
  CK(b, cudaMemcpyAsync(b->d_rho_ladder, ladder.data(), sizeof(float) * RHO_MAX_LEVELS, cudaMemcpyHostToDevice, b->stream));
  CK(b, launch_pack_obstacles(D, P, 2 * index[2 * P + 1], b->d_obs_index, b->d_obs_index + P + 1,
                              st_c, st_a, st_v, b->d_obs, b->d_problems, b->stream));
  for (int l = 0; l < L; ++l)
    CK(b, launch_setup_problems(b->d_problems, P, b->d_T, b->d_start, b->d_goal, b->d_start_va, D,
                                b->cfg.rho * std::pow(b->rho_growth, (double)l), b->cfg.w_smooth,
                                b->cfg.w_track, b->cfg.cost_mode, b->max_np_used,
                                b->d_constants + (size_t)l * CONST_FLOATS, b->stream,
                                b->d_kkt64 + (size_t)l * KKT64_DOUBLES,
                                (size_t)L * KKT64_DOUBLES));
  CK(b, cudaStreamSynchronize(b->stream));
  b->kkt_valid = true;
  return TRAJ_OK;
}

// After a receding-horizon shift with the FP64 blocks at hand: the moved obstacles
// re-packed, and only the boundary-dependent constants (hq, c) of every level
// recomputed; the KKT matrix (n_p, T, n_o, rho, bounds) is the one set up before.
static traj_status shift_boundary(traj_batch *b, cudaStream_t s) {
  const int P = b->n_problems, D = b->cfg.dim, N = b->n_obs, L = b->rho_levels;
  const float *st_c = b->d_obs_stage, *st_a = st_c + (size_t)N * D, *st_v = st_a + (size_t)N * D;
  const int *index = b->pair_index.data();
  CK(b, launch_pack_obstacles(D, P, 2 * index[2 * P + 1], b->d_obs_index, b->d_obs_index + P + 1,
                              st_c, st_a, st_v, b->d_obs, b->d_problems, s));
  CK(b, launch_setup_boundary(P, L, b->d_start, b->d_goal, b->d_start_va, D, b->cfg.w_track,
                              b->d_kkt64, b->d_constants, s));
  return TRAJ_OK;
}

traj_status traj_set_obstacles(traj_batch *b, const int *offsets, const float *centers,
                               const float *semi_axes, const float *velocities) {
  tb::NvtxRange nvtx_range("traj_set_obstacles");
  if (!b) return TRAJ_EINVAL;
  if (!b->have_problems) return fail(b, TRAJ_ESTATE, "traj_set_problems must come first");
  if (!offsets) return fail(b, TRAJ_EINVAL, "NULL offsets");
  const int P = b->n_problems, D = b->cfg.dim;
  if (offsets[0] != 0) return fail(b, TRAJ_EINVAL, "offsets[0] must be 0");
  for (int p = 0; p < P; ++p)
    if (offsets[p + 1] < offsets[p]) return fail(b, TRAJ_EINVAL, "offsets must be non-decreasing");
  const int N = offsets[P];
  if (N > b->cfg.max_obstacles) return fail(b, TRAJ_ESHAPE, "obstacle count exceeds max_obstacles");
  if (N > 0 && (!centers || !semi_axes || !velocities))
    return fail(b, TRAJ_EINVAL, "NULL obstacle array");
  // pair records: problem p owns pair_count(n_o) of them from index[P + 1 + p]
  std::vector<int> index(2 * (P + 1));
  for (int p = 0; p <= P; ++p) index[p] = offsets[p];
  for (int p = 0; p < P; ++p) index[P + 2 + p] = index[P + 1 + p] + pair_count(offsets[p + 1] - offsets[p]);
  // tables offsets per horizon (same order as in set_problems)
  std::vector<int> hz(b->n_steps);
  std::sort(hz.begin(), hz.end());
  hz.erase(std::unique(hz.begin(), hz.end()), hz.end());
  std::vector<ProblemDev> recs(P);
  std::vector<int> tbl_host(P);
  for (int p = 0; p < P; ++p) {
    ProblemDev r{};
    r.n_p = b->n_steps[p];
    r.n_o = offsets[p + 1] - offsets[p];
    r.pair_off = index[P + 1 + p];
    int off = 0;
    for (int h : hz) { if (h == r.n_p) break; off += table_floats(h); }
    r.tbl_off = off;
    tbl_host[p] = off;
    const double T = b->duration[p];
    r.dt = (float)(T / (double)(r.n_p - 1));
    r.invT = (float)(1.0 / T);
    r.invT2 = (float)(1.0 / (T * T));
    r.nan_flag = 0;
    recs[p] = r;
  }
  float *st_c = b->d_obs_stage, *st_a = st_c + (size_t)N * D, *st_v = st_a + (size_t)N * D;
  if (N > 0) {
    CK(b, cudaMemcpyAsync(st_c, centers, sizeof(float) * N * D, cudaMemcpyDefault, b->stream));
    CK(b, cudaMemcpyAsync(st_a, semi_axes, sizeof(float) * N * D, cudaMemcpyDefault, b->stream));
    CK(b, cudaMemcpyAsync(st_v, velocities, sizeof(float) * N * D, cudaMemcpyDefault, b->stream));
  }
  b->recs = recs;
  b->pair_index = index;
  b->n_obs = N;
  traj_status rs = upload_problems(b);
  if (rs != TRAJ_OK) return rs;
  b->obs_offsets.assign(offsets, offsets + P + 1);
  b->tbl_off = tbl_host;
  b->have_obstacles = true;
  invalidate_graph(b);
  b->have_result = false;
  b->err.clear();
  return TRAJ_OK;
}

traj_status traj_set_initial(traj_batch *b, int n_traj, const int *traj_problem,
                             const float *coeffs0) {
  if (!b) return TRAJ_EINVAL;
  if (!b->have_obstacles) return fail(b, TRAJ_ESTATE, "traj_set_obstacles must come first");
  if (b->resume || b->carry) { // a fresh start from here on
    b->resume = false;
    b->carry = false;
    invalidate_graph(b);
  }
  if (!traj_problem && coeffs0 && b->have_initial && n_traj == b->n_traj) {
    // coefficients only: keep the trajectory -> problem map and the work order
    CK(b, cudaMemcpyAsync(b->d_xi0, coeffs0, sizeof(float) * n_traj * b->cfg.dim * NC,
                          cudaMemcpyDefault, b->stream));
    if (is_host_ptr(coeffs0)) CK(b, cudaStreamSynchronize(b->stream));
    b->have_result = false;
    return TRAJ_OK;
  }
  if (!traj_problem || !coeffs0) return fail(b, TRAJ_EINVAL, "NULL trajectory array");
  if (n_traj < 1 || n_traj > b->cfg.max_traj) return fail(b, TRAJ_ESHAPE, "n_traj exceeds max_traj (or < 1)");
  for (int k = 0; k < n_traj; ++k)
    if (traj_problem[k] < 0 || traj_problem[k] >= b->n_problems)
      return fail(b, TRAJ_EINVAL, "traj_problem entry out of range");
  // work-queue order: by the number of 32-point slots (the kernels specialise their
  // code on it), most first, so that the warps of an SM run one specialisation at a
  // time instead of fetching several in turn; within it, most expensive (n_o * n_p)
  // first; stable
  std::vector<int> order(n_traj);
  for (int k = 0; k < n_traj; ++k) order[k] = k;
  std::vector<long long> cost(b->n_problems);
  std::vector<int> slots(b->n_problems);
  for (int p = 0; p < b->n_problems; ++p) {
    cost[p] = (long long)(b->obs_offsets[p + 1] - b->obs_offsets[p] + 2) * b->n_steps[p];
    slots[p] = (b->n_steps[p] + 31) / 32;
  }
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    const int px = traj_problem[x], py = traj_problem[y];
    if (slots[px] != slots[py]) return slots[px] > slots[py];
    return cost[px] > cost[py];
  });
  CK(b, cudaMemcpyAsync(b->d_xi0, coeffs0, sizeof(float) * n_traj * b->cfg.dim * NC, cudaMemcpyDefault, b->stream));
  CK(b, cudaMemcpyAsync(b->d_traj_problem, traj_problem, sizeof(int) * n_traj, cudaMemcpyHostToDevice, b->stream));
  CK(b, cudaMemcpyAsync(b->d_order, order.data(), sizeof(int) * n_traj, cudaMemcpyHostToDevice, b->stream));
  CK(b, cudaStreamSynchronize(b->stream));
  b->traj_problem.assign(traj_problem, traj_problem + n_traj);
  b->n_traj = n_traj;
  b->have_initial = true;
  invalidate_graph(b);
  b->have_result = false;
  b->err.clear();
  return TRAJ_OK;
}

// Statistics of the last solve (synchronises the stream) and its status: the
// error flags first, then TRAJ_NOT_CONVERGED unless every trajectory converged.
static traj_status solve_stats(traj_batch *b, traj_solve_stats *stats) {
  CK(b, cudaStreamSynchronize(b->stream));
  const int B = b->n_traj;
  std::vector<int> it(B);
  std::vector<float> res((size_t)B * 3);
  std::vector<signed char> st(B);
  int flags = 0;
  CK(b, cudaMemcpy(it.data(), b->d_iters, sizeof(int) * B, cudaMemcpyDeviceToHost));
  CK(b, cudaMemcpy(res.data(), b->d_res, sizeof(float) * B * 3, cudaMemcpyDeviceToHost));
  CK(b, cudaMemcpy(st.data(), b->d_status, B, cudaMemcpyDeviceToHost));
  CK(b, cudaMemcpy(&flags, b->d_flags, sizeof(int), cudaMemcpyDeviceToHost));
  float ms = 0.f;
  CK(b, cudaEventElapsedTime(&ms, b->ev0, b->ev1));
  traj_solve_stats s{};
  s.n_traj = B;
  std::vector<int> sorted = it;
  std::sort(sorted.begin(), sorted.end());
  s.iters_min = sorted.front();
  s.iters_max = sorted.back();
  s.iters_median = sorted[B / 2];
  for (int k = 0; k < B; ++k) {
    if (st[k] == TRAJ_TRAJ_CONVERGED) ++s.n_solved;
    if (st[k] == TRAJ_TRAJ_NAN) continue;
    s.max_res_obs = std::max(s.max_res_obs, res[k * 3 + 0]);
    s.max_res_v = std::max(s.max_res_v, res[k * 3 + 1]);
    s.max_res_a = std::max(s.max_res_a, res[k * 3 + 2]);
  }
  s.gpu_ms = ms;
  *stats = s;
  if (flags & 8) return fail(b, TRAJ_ECUDA, "a tensor-core pipeline wait expired");
  if (flags & 1) return fail(b, TRAJ_ETIMEOUT, "deadline reached");
  if (flags & 2) return fail(b, TRAJ_ENAN, "non-finite input in some trajectories");
  return s.n_solved == B ? TRAJ_OK : TRAJ_NOT_CONVERGED;
}

// How the solve starts: 0 fresh (project xi0, lambda0 = 0), 1 resume (QP step from
// the imported xi, lambda, u), 2 carry (project the shifted xi0, lambda0 = carried).
static int start_mode(const traj_batch *b) { return b->resume ? 1 : (b->carry ? 2 : 0); }

// The solve's arguments from the handle's state, after checking the call.
static traj_status solve_args(traj_batch *b, int max_iters, float tol, double timeout_ms,
                              SolveArgs &a) {
  if (!b->have_initial) return fail(b, TRAJ_ESTATE, "traj_set_initial must come first");
  if (max_iters < 0) return fail(b, TRAJ_EINVAL, "max_iters must be >= 0");
  if (std::isnan(tol) || !(timeout_ms >= 0)) return fail(b, TRAJ_EINVAL, "bad tol or timeout");
  const bool mixed = b->cfg.precision != TRAJ_PREC_FP32;
  if (mixed && b->max_np_used > MAX_STEPS)
    return fail(b, TRAJ_ESHAPE, "the tensor-core form takes at most 256 grid points per problem");
  if (b->max_np_used > MAX_STEPS && b->shape.team != 1)
    return fail(b, TRAJ_ESHAPE, "horizons above 256 grid points run one warp per trajectory "
                                "(warps_per_trajectory 1)");
  a = SolveArgs{};
  a.problems = b->d_problems;
  a.obstacles = b->d_obs;
  a.constants = b->d_constants;
  a.rho_ladder = b->d_rho_ladder;
  a.rho_levels = b->rho_levels;
  a.rho_every = b->rho_levels > 1 ? b->rho_every : 0;
  a.tables = b->d_tables;
  a.table_floats_total = b->table_floats;
  a.traj_problem = b->d_traj_problem;
  a.order = b->d_order;
  a.xi0 = b->d_xi0;
  a.lam0 = (b->resume || b->carry) ? b->d_lam0 : nullptr;
  a.u0 = b->resume ? b->d_u0 : nullptr; // carry: u is formed by the initial projection
  a.xi = b->d_xi;
  a.lam = b->d_lam;
  a.u = b->d_u;
  a.res = b->d_res;
  a.iters = b->d_iters;
  a.status = b->d_status;
  a.n_traj = b->n_traj;
  a.max_iters = max_iters;
  a.tol = tol;
  a.rho = (float)b->cfg.rho;
  a.vmax = (float)b->cfg.vmax;
  a.amax = (float)b->cfg.amax;
  a.cost_mode = b->cfg.cost_mode;
  a.timeout_ns = timeout_ms > 0 ? (unsigned long long)(timeout_ms * 1e6) : 0ull;
  {
    // distinct horizons in table order (ascending n_p, as traj_set_problems laid them out)
    std::vector<int> hz(b->n_steps);
    std::sort(hz.begin(), hz.end());
    hz.erase(std::unique(hz.begin(), hz.end()), hz.end());
    if (mixed && (int)hz.size() > MAX_HZ)
      return fail(b, TRAJ_ESHAPE, "the tensor-core form takes at most 16 distinct horizons per batch");
    int off = 0;
    a.hz_n = std::min((int)hz.size(), MAX_HZ);
    for (int h = 0; h < a.hz_n; ++h) {
      a.hz_np[h] = hz[h];
      a.hz_tbl[h] = off;
      off += table_floats(hz[h]);
    }
    a.table_floats_total = b->table_floats;
    if (mixed && mixed_smem_bytes(a, b->cfg.dim, b->cfg.precision == TRAJ_PREC_MIXED_SPLIT, 1) >
                     227 * 1024)
      return fail(b, TRAJ_ESHAPE, "the tensor-core form's basis operands of these horizons exceed "
                                  "the shared memory of one CTA");
  }
  a.queue = b->d_queue;
  a.t0 = b->d_t0;
  a.flags = b->d_flags;
  return TRAJ_OK;
}

// One solve on stream cs (also while it is capturing): clear the counters, then the
// persistent solve launch.
static cudaError_t record_solve(traj_batch *b, const SolveArgs &a, cudaStream_t cs) {
  cudaError_t ce = cudaMemsetAsync(b->d_queue, 0, sizeof(int), cs);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(b->d_flags, 0, sizeof(int), cs);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(b->d_t0, 0, sizeof(unsigned long long), cs);
  if (ce == cudaSuccess)
    ce = launch_am_solve(b->cfg.dim, b->max_np_used, b->cfg.precision, a, b->shape, b->n_sm, cs,
                         &b->used);
  return ce;
}

// The key of a captured solve: the arguments that reach the graph's nodes by value.
static GraphKey graph_key(const traj_batch *b, int max_iters, float tol, const SolveArgs &a) {
  GraphKey k;
  k.max_iters = max_iters; k.tol = tol; k.timeout = a.timeout_ns; k.n_traj = b->n_traj;
  k.warps = b->shape.warps_per_block; k.bps = b->shape.blocks_per_sm; k.team = b->shape.team;
  k.occ = b->shape.occupancy; k.resume = start_mode(b);
  return k;
}

traj_status traj_solve(traj_batch *b, int max_iters, float tol, double timeout_ms,
                       traj_solve_stats *stats) {
  tb::NvtxRange nvtx_range("traj_solve");
  if (!b) return TRAJ_EINVAL;
  SolveArgs a;
  traj_status rs = solve_args(b, max_iters, tol, timeout_ms, a);
  if (rs != TRAJ_OK) return rs;
  const GraphKey key = graph_key(b, max_iters, tol, a);
  if (!(b->graph_valid && b->g_key == key)) {
    // capture {clear counters; persistent solve} on the handle's capture stream
    drop_solve_graph(b);
    cudaStream_t cs = b->capture_stream;
    CK(b, cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    cudaError_t ce = record_solve(b, a, cs);
    cudaGraph_t g = nullptr;
    cudaError_t ee = cudaStreamEndCapture(cs, &g);
    if (ce == cudaSuccess) ce = ee;
    if (ce == cudaSuccess) ce = cudaGraphInstantiate(&b->graph_exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (ce != cudaSuccess) {
      drop_solve_graph(b);
      return fail(b, TRAJ_ECUDA, std::string("solve graph capture: ") + cudaGetErrorString(ce));
    }
    b->graph_valid = true;
    b->g_key = key;
  }
  CK(b, cudaEventRecord(b->ev0, b->stream));
  CK(b, cudaGraphLaunch(b->graph_exec, b->stream));
  CK(b, cudaEventRecord(b->ev1, b->stream));
  b->have_result = true;
  if (!stats) return TRAJ_OK;
  return solve_stats(b, stats);
}

traj_status traj_get_solve_stats(traj_batch *b, traj_solve_stats *stats) {
  if (!b || !stats) return TRAJ_EINVAL;
  if (!b->have_result) return fail(b, TRAJ_ESTATE, "no solve has run");
  return solve_stats(b, stats);
}

traj_status traj_get_trajectories(traj_batch *b, float *coeffs, float *residual, int *iters,
                                  signed char *status) {
  tb::NvtxRange nvtx_range("traj_get_trajectories");
  if (!b) return TRAJ_EINVAL;
  if (!b->have_result) return fail(b, TRAJ_ESTATE, "no solve has run");
  const size_t B = b->n_traj, D = b->cfg.dim;
  bool host = false;
  if (coeffs) { CK(b, cudaMemcpyAsync(coeffs, b->d_xi, sizeof(float) * B * D * NC, cudaMemcpyDefault, b->stream)); host |= is_host_ptr(coeffs); }
  if (residual) { CK(b, cudaMemcpyAsync(residual, b->d_res, sizeof(float) * B * 3, cudaMemcpyDefault, b->stream)); host |= is_host_ptr(residual); }
  if (iters) { CK(b, cudaMemcpyAsync(iters, b->d_iters, sizeof(int) * B, cudaMemcpyDefault, b->stream)); host |= is_host_ptr(iters); }
  if (status) { CK(b, cudaMemcpyAsync(status, b->d_status, B, cudaMemcpyDefault, b->stream)); host |= is_host_ptr(status); }
  if (host) CK(b, cudaStreamSynchronize(b->stream));
  return TRAJ_OK;
}

traj_status traj_get_accel_cost(traj_batch *b, float *cost) {
  if (!b || !cost) return TRAJ_EINVAL;
  if (!b->have_result) return fail(b, TRAJ_ESTATE, "no solve has run");
  CK(b, launch_accel_cost(b->d_xi, b->d_traj_problem, b->d_problems, b->d_tables, b->cfg.dim,
                          b->n_traj, b->d_r, b->stream));
  CK(b, cudaMemcpyAsync(cost, b->d_r, sizeof(float) * b->n_traj, cudaMemcpyDefault, b->stream));
  if (is_host_ptr(cost)) CK(b, cudaStreamSynchronize(b->stream));
  return TRAJ_OK;
}

traj_status traj_homotopy_signature(traj_batch *b, unsigned long long *sig) {
  if (!b || !sig) return TRAJ_EINVAL;
  if (!b->have_result) return fail(b, TRAJ_ESTATE, "no solve has run");
  if (b->cfg.dim != 2) return fail(b, TRAJ_EINVAL, "homotopy signatures are defined for 2D problems");
  if (b->max_np_used > MAX_STEPS) return fail(b, TRAJ_ESHAPE, "homotopy signatures take n_p <= 256");
  const int N = b->n_obs, D = b->cfg.dim;
  const float *st_c = b->d_obs_stage, *st_a = st_c + (size_t)N * D, *st_v = st_a + (size_t)N * D;
  CK(b, launch_homotopy(b->d_xi, b->d_traj_problem, b->d_problems, b->d_tables, st_c, st_a, st_v,
                        b->d_obs_index, b->n_traj, b->d_sig, b->stream));
  CK(b, cudaMemcpyAsync(sig, b->d_sig, sizeof(unsigned long long) * b->n_traj, cudaMemcpyDefault,
                        b->stream));
  if (is_host_ptr(sig)) CK(b, cudaStreamSynchronize(b->stream));
  return TRAJ_OK;
}

traj_status traj_get_state(traj_batch *b, float *lambda, float *u) {
  if (!b) return TRAJ_EINVAL;
  if (!b->have_result) return fail(b, TRAJ_ESTATE, "no solve has run");
  const size_t n = (size_t)b->n_traj * b->cfg.dim * NC;
  bool host = false;
  if (lambda) { CK(b, cudaMemcpyAsync(lambda, b->d_lam, sizeof(float) * n, cudaMemcpyDefault, b->stream)); host |= is_host_ptr(lambda); }
  if (u) { CK(b, cudaMemcpyAsync(u, b->d_u, sizeof(float) * n, cudaMemcpyDefault, b->stream)); host |= is_host_ptr(u); }
  if (host) CK(b, cudaStreamSynchronize(b->stream));
  return TRAJ_OK;
}

traj_status traj_set_workspace(traj_batch *b, const double *lower, const double *upper) {
  if (!b) return TRAJ_EINVAL;
  if (!b->have_problems) return fail(b, TRAJ_ESTATE, "traj_set_problems must come first");
  if ((lower == nullptr) != (upper == nullptr)) return fail(b, TRAJ_EINVAL, "give both bounds or neither");
  const int P = b->n_problems, D = b->cfg.dim;
  if (lower) {
    for (int k = 0; k < P * D; ++k)
      if (!std::isfinite(lower[k]) || !std::isfinite(upper[k]) || !(lower[k] < upper[k]))
        return fail(b, TRAJ_EINVAL, "workspace bounds must be finite with lower < upper");
    b->box_lo.assign(lower, lower + (size_t)P * D);
    b->box_hi.assign(upper, upper + (size_t)P * D);
  } else {
    b->box_lo.clear();
    b->box_hi.clear();
  }
  invalidate_graph(b);
  b->have_result = false;
  if (b->have_obstacles) return upload_problems(b);
  return TRAJ_OK;
}

traj_status traj_set_rho_schedule(traj_batch *b, int levels, double growth, int every) {
  if (!b) return TRAJ_EINVAL;
  if (levels < 1 || levels > RHO_MAX_LEVELS || !(growth > 0) || !std::isfinite(growth) ||
      (levels > 1 && every < 1))
    return fail(b, TRAJ_EINVAL, "levels in [1, 10], growth > 0, every >= 1 (when levels > 1)");
  if (levels > b->const_levels) { // room for the constants of every level
    float *c = nullptr;
    const size_t n = (size_t)b->cfg.max_problems * CONST_FLOATS * levels;
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&c), sizeof(float) * n);
    if (e != cudaSuccess) return fail(b, e == cudaErrorMemoryAllocation ? TRAJ_ENOMEM : TRAJ_ECUDA,
                                      std::string("cudaMalloc: ") + cudaGetErrorString(e));
    CK(b, cudaStreamSynchronize(b->stream));
    cudaFree(b->d_constants);
    b->d_constants = c;
    b->const_levels = levels;
  }
  b->rho_levels = levels;
  b->rho_growth = growth;
  b->rho_every = levels > 1 ? every : 0;
  invalidate_graph(b);
  b->have_result = false;
  if (b->have_obstacles) return upload_problems(b);
  return TRAJ_OK;
}

traj_status traj_set_state(traj_batch *b, const float *coeffs, const float *lambda, const float *u) {
  if (!b) return TRAJ_EINVAL;
  if (!coeffs || !lambda || !u) return fail(b, TRAJ_EINVAL, "NULL state array");
  if (!b->have_initial) return fail(b, TRAJ_ESTATE, "traj_set_initial must come first");
  if (b->cfg.cost_mode != TRAJ_COST_SMOOTH_TRACK)
    return fail(b, TRAJ_EINVAL, "resume needs the smoothness/tracking cost (projection mode reads "
                                "its sample from the initial coefficients)");
  const size_t n = (size_t)b->n_traj * b->cfg.dim * NC;
  CK(b, cudaMemcpyAsync(b->d_xi0, coeffs, sizeof(float) * n, cudaMemcpyDefault, b->stream));
  CK(b, cudaMemcpyAsync(b->d_lam0, lambda, sizeof(float) * n, cudaMemcpyDefault, b->stream));
  CK(b, cudaMemcpyAsync(b->d_u0, u, sizeof(float) * n, cudaMemcpyDefault, b->stream));
  if (is_host_ptr(coeffs) || is_host_ptr(lambda) || is_host_ptr(u)) CK(b, cudaStreamSynchronize(b->stream));
  if (!b->resume || b->carry) {
    b->resume = true;
    b->carry = false;
    invalidate_graph(b);
  }
  b->have_result = false;
  return TRAJ_OK;
}

// Check a receding-horizon step and fill its arguments; a given executed array is
// copied to the device on the handle's stream.
static traj_status shift_args(traj_batch *b, double delta, const int *executed, ShiftArgs &a) {
  if (!b->have_result) return fail(b, TRAJ_ESTATE, "traj_shift_horizon needs a finished solve");
  if (b->cfg.cost_mode != TRAJ_COST_SMOOTH_TRACK)
    return fail(b, TRAJ_EINVAL, "the receding-horizon step needs the smoothness/tracking cost");
  const int P = b->n_problems, B = b->n_traj;
  double tmin = b->duration[0];
  for (int p = 1; p < P; ++p) tmin = std::min(tmin, b->duration[p]);
  if (!(delta > 0) || !(delta < tmin) || !std::isfinite(delta))
    return fail(b, TRAJ_EINVAL, "delta must lie in (0, T) for every problem");
  if (executed) {
    for (int p = 0; p < P; ++p)
      if (executed[p] < 0 || executed[p] >= B || b->traj_problem[executed[p]] != p)
        return fail(b, TRAJ_EINVAL, "executed[" + std::to_string(p) + "] is not a trajectory of problem " +
                                        std::to_string(p));
    CK(b, cudaMemcpyAsync(b->d_exec, executed, sizeof(int) * P, cudaMemcpyHostToDevice, b->stream));
  }
  a = ShiftArgs{};
  a.dim = b->cfg.dim;
  a.n_problems = P;
  a.n_traj = B;
  a.n_obs = b->n_obs;
  a.delta = delta;
  a.T = b->d_T;
  a.traj_problem = b->d_traj_problem;
  a.xi = b->d_xi;
  a.lam = b->d_lam;
  a.res = b->d_res;
  a.xi0 = b->d_xi0;
  a.lam0 = b->d_lam0;
  a.executed = executed ? b->d_exec : nullptr;
  a.exec_scratch = b->d_exec;
  a.key_scratch = b->d_exec_key;
  a.start = b->d_start;
  a.start_va = b->d_start_va;
  a.centers = b->d_obs_stage;
  a.velocities = b->d_obs_stage + (size_t)2 * b->n_obs * b->cfg.dim;
  return TRAJ_OK;
}

// After a shift the next solves start from the shifted iterate and the carried
// multipliers.
static void shift_state(traj_batch *b) {
  if (!b->carry || b->resume) {
    b->carry = true;
    b->resume = false;
    invalidate_graph(b);
  }
  b->have_result = false;
}

traj_status traj_shift_horizon(traj_batch *b, double delta, const int *executed) {
  tb::NvtxRange nvtx_range("traj_shift_horizon");
  if (!b) return TRAJ_EINVAL;
  ShiftArgs a;
  traj_status rs = shift_args(b, delta, executed, a);
  if (rs != TRAJ_OK) return rs;
  CK(b, launch_mpc_shift(a, b->stream));
  // re-pack the moved obstacles and recompute the boundary-dependent constants of every
  // level from the FP64 blocks that the last set-up kept (a full set-up only if none
  // has been kept)
  rs = b->kkt_valid ? shift_boundary(b, b->stream) : upload_problems(b);
  if (rs != TRAJ_OK) return rs;
  shift_state(b);
  b->err.clear();
  return TRAJ_OK;
}

traj_status traj_mpc_step(traj_batch *b, double delta, const int *executed, int max_iters,
                          float tol, double timeout_ms) {
  tb::NvtxRange nvtx_range("traj_mpc_step");
  if (!b) return TRAJ_EINVAL;
  if (!b->kkt_valid) { // no FP64 blocks kept: the shift sets up in full and synchronises
    traj_status rs = traj_shift_horizon(b, delta, executed);
    return rs != TRAJ_OK ? rs : traj_solve(b, max_iters, tol, timeout_ms, nullptr);
  }
  // check the solve first, as it will run from the shifted state
  const bool carry0 = b->carry, resume0 = b->resume;
  b->carry = true;
  b->resume = false;
  SolveArgs a;
  traj_status rs = solve_args(b, max_iters, tol, timeout_ms, a);
  b->carry = carry0;
  b->resume = resume0;
  if (rs != TRAJ_OK) return rs;
  ShiftArgs sa;
  if ((rs = shift_args(b, delta, executed, sa)) != TRAJ_OK) return rs;
  shift_state(b);
  const GraphKey key = graph_key(b, max_iters, tol, a);
  const bool given = executed != nullptr;
  if (!(b->mpc_valid && b->mpc_key == key && b->mpc_delta == delta && b->mpc_given == given)) {
    // capture {shift; obstacle packing; boundary update; clear counters; solve}
    if (b->mpc_exec) cudaGraphExecDestroy(b->mpc_exec);
    b->mpc_exec = nullptr;
    b->mpc_valid = false;
    cudaStream_t cs = b->capture_stream;
    cudaError_t ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (ce == cudaSuccess) {
      ce = launch_mpc_shift(sa, cs);
      if (ce == cudaSuccess && shift_boundary(b, cs) != TRAJ_OK) ce = cudaErrorUnknown;
      if (ce == cudaSuccess) ce = record_solve(b, a, cs);
      cudaGraph_t g = nullptr;
      cudaError_t ee = cudaStreamEndCapture(cs, &g);
      if (ce == cudaSuccess) ce = ee;
      if (ce == cudaSuccess) ce = cudaGraphInstantiate(&b->mpc_exec, g, 0);
      if (g) cudaGraphDestroy(g);
    }
    if (ce != cudaSuccess) { // nothing of the step ran: the handle stays as it was
      if (b->mpc_exec) cudaGraphExecDestroy(b->mpc_exec);
      b->mpc_exec = nullptr;
      b->carry = carry0;
      b->resume = resume0;
      b->have_result = true;
      return fail(b, TRAJ_ECUDA, std::string("control step graph capture: ") + cudaGetErrorString(ce));
    }
    b->mpc_valid = true;
    b->mpc_key = key;
    b->mpc_delta = delta;
    b->mpc_given = given;
  }
  CK(b, cudaEventRecord(b->ev0, b->stream));
  CK(b, cudaGraphLaunch(b->mpc_exec, b->stream));
  CK(b, cudaEventRecord(b->ev1, b->stream));
  b->have_result = true;
  b->err.clear();
  return TRAJ_OK;
}

traj_status traj_set_launch_shape(traj_batch *b, const traj_launch_shape *shape) {
  if (!b || !shape) return TRAJ_EINVAL;
  const bool tc = b->cfg.precision != TRAJ_PREC_FP32;
  if (shape->warps_per_block < 0 || shape->warps_per_block > 8 || shape->blocks_per_sm < 0 ||
      (shape->warps_per_trajectory != 1 && shape->warps_per_trajectory != 2 &&
       shape->warps_per_trajectory != 4) ||
      (shape->warps_per_block % shape->warps_per_trajectory) != 0 ||
      (tc && shape->warps_per_trajectory != 1))
    return fail(b, TRAJ_EINVAL, "warps_per_block in [0, 8] (0: default; a multiple of "
                                "warps_per_trajectory), blocks_per_sm >= 0, warps_per_trajectory "
                                "1, 2 or 4 (1 in the tensor-core form)");
  if (shape->occupancy != 0 && shape->occupancy != 1)
    return fail(b, TRAJ_EINVAL, "occupancy must be 0 or 1");
  if (shape->occupancy && (shape->warps_per_trajectory != 1 || shape->warps_per_block > (tc ? 6 : 4)))
    return fail(b, TRAJ_EINVAL, "the register-capped build runs one warp per trajectory and at "
                                "most 4 warps per block (6 in the tensor-core form)");
  if (shape->occupancy && b->have_problems && b->max_np_used > 160)
    return fail(b, TRAJ_ESHAPE, "the register-capped build takes horizons up to 160 grid points");
  b->shape = LaunchShape{shape->warps_per_block, shape->blocks_per_sm, 0, shape->warps_per_trajectory,
                         shape->occupancy};
  invalidate_graph(b);
  return TRAJ_OK;
}

traj_status traj_get_launch_info(traj_batch *b, traj_launch_shape *resolved, int *grid,
                                 int *registers, int *shared_bytes) {
  if (!b) return TRAJ_EINVAL;
  if (!b->graph_valid) return fail(b, TRAJ_ESTATE, "no solve launch has been captured");
  if (resolved) {
    resolved->warps_per_block = b->used.warps_per_block;
    resolved->blocks_per_sm = b->used.blocks_per_sm;
    resolved->warps_per_trajectory = b->used.team;
    resolved->occupancy = b->used.occupancy;
  }
  if (grid) *grid = b->used.grid;
  if (registers) *registers = b->used.regs;
  if (shared_bytes) *shared_bytes = b->used.smem;
  return TRAJ_OK;
}

traj_status traj_autotune(traj_batch *b, int iters, traj_launch_shape *chosen, float *best_ms) {
  tb::NvtxRange nvtx_range("traj_autotune");
  if (!b) return TRAJ_EINVAL;
  if (!b->have_initial) return fail(b, TRAJ_ESTATE, "traj_set_initial must come first");
  if (iters < 1) return fail(b, TRAJ_EINVAL, "iters must be >= 1");
  static const int cand_w[] = {0, 1, 2, 4, 8}; // 0: the form's default shape
  static const int cand_b[] = {0, 1, 2, 4};
  const bool tc = b->cfg.precision != TRAJ_PREC_FP32;
  std::vector<LaunchShape> cands;
  for (int team = 1; team <= (tc ? 1 : 4); team *= 2)
    for (int w : cand_w)
      for (int bps : cand_b)
        if (w % team == 0) cands.push_back(LaunchShape{w, bps, 0, team, 0});
  if (b->max_np_used <= 160) // the register-capped build, one warp per trajectory
    for (int w : {0, 2, 4, 6})
      for (int bps : {0, 2, 3})
        if (w <= (tc ? 6 : 4)) cands.push_back(LaunchShape{w, bps, 0, 1, 1});
  LaunchShape best{4, 0, 0, 1, 0};
  float best_t = 1e30f;
  for (const LaunchShape &c : cands) {
    b->shape = c;
    invalidate_graph(b);
    float tot = 0.f;
    bool ok = true;
    for (int r = 0; r < 3 && ok; ++r) { // first run captures the graph, then two timed replays
      traj_solve_stats st{};
      traj_status rc = traj_solve(b, iters, -1.0f, 0.0, &st);
      if (rc != TRAJ_OK && rc != TRAJ_NOT_CONVERGED) ok = false;
      else if (r > 0) tot += st.gpu_ms;
    }
    if (ok && tot < best_t) { best_t = tot; best = b->shape; }
  }
  b->shape = best;
  invalidate_graph(b);
  b->have_result = false;
  if (chosen) {
    chosen->warps_per_block = best.warps_per_block;
    chosen->blocks_per_sm = best.blocks_per_sm;
    chosen->warps_per_trajectory = best.team;
    chosen->occupancy = best.occupancy;
  }
  if (best_ms) *best_ms = best_t / 2.f;
  if (best_t >= 1e30f) return fail(b, TRAJ_ECUDA, "no launch shape ran");
  b->err.clear(); // candidates the batch refuses (teams on long horizons) are not errors
  return TRAJ_OK;
}

traj_status traj_sampler_step_multi(traj_batch *b, const traj_sampler_config *sc, int iteration,
                                    int n_dist, float *mu, float *sigma, const float *z,
                                    float *best, const traj_sampler_trace *trace) {
  tb::NvtxRange nvtx_range("traj_sampler_step_multi");
  if (!b) return TRAJ_EINVAL;
  if (!sc || !mu || !sigma || !best) return fail(b, TRAJ_EINVAL, "NULL sampler argument");
  if (!b->have_initial) return fail(b, TRAJ_ESTATE, "traj_set_initial must come first");
  if (b->cfg.cost_mode != TRAJ_COST_PROJECT)
    return fail(b, TRAJ_ESTATE, "the sampler needs a handle in TRAJ_COST_PROJECT mode");
  const int B = b->n_traj, D = b->cfg.dim * NC;
  for (int k = 0; k < B; ++k)
    if (b->traj_problem[k] != 0) return fail(b, TRAJ_EINVAL, "sampler trajectories must all belong to problem 0");
  if (n_dist < 1 || n_dist > TRAJ_SAMPLER_MAX_DIST || B % n_dist != 0)
    return fail(b, TRAJ_EINVAL, "n_dist must be in [1, TRAJ_SAMPLER_MAX_DIST] and divide n_traj");
  const int Bg = B / n_dist;
  if (Bg > 8192) return fail(b, TRAJ_ESHAPE, "samples per distribution must be <= 8192");
  if (sc->n_inner < 0 || sc->n_proj < 1 || sc->n_proj > Bg || sc->n_elite < 1 ||
      sc->n_elite > sc->n_proj || !(sc->gamma > 0) || !(sc->sigma_lr > 0) || sc->sigma_lr > 1 ||
      !(sc->eps >= 0) || !(sc->w_res >= 0) || !(sc->w_curv >= 0) || !(sc->w_path >= 0))
    return fail(b, TRAJ_EINVAL, "sampler config out of range");
  CK(b, launch_sampler_front(mu, sigma, D, B, n_dist, sc->eps, z, sc->seed, iteration, b->d_L,
                             b->d_sflag, b->d_xi0, trace ? trace->samples : nullptr, b->stream));
  traj_status rc = traj_solve(b, sc->n_inner, -1.0f, 0.0, nullptr);
  if (rc != TRAJ_OK) return rc;
  const int n_p = b->n_steps[0];
  const double T = b->duration[0];
  const SamplerCost cost{sc->w_res, sc->w_curv, sc->w_path, b->d_start, b->d_goal};
  CK(b, launch_sampler_back(b->d_xi, b->d_res, b->d_tables, b->tbl_off[0], n_p, (float)(1.0 / T),
                            (float)(1.0 / (T * T)), b->cfg.dim, B, n_dist, cost, sc->n_proj,
                            sc->n_elite, sc->gamma, sc->sigma_lr, b->d_r, b->d_caug, b->d_proj,
                            b->d_elite, b->d_refit, mu, sigma, best, b->stream));
  if (trace) {
    const size_t np = (size_t)n_dist * sc->n_proj, ne = (size_t)n_dist * sc->n_elite;
    if (trace->projected) CK(b, cudaMemcpyAsync(trace->projected, b->d_xi, sizeof(float) * B * D, cudaMemcpyDeviceToDevice, b->stream));
    if (trace->residual) CK(b, cudaMemcpyAsync(trace->residual, b->d_r, sizeof(float) * B, cudaMemcpyDeviceToDevice, b->stream));
    if (trace->cost_aug) CK(b, cudaMemcpyAsync(trace->cost_aug, b->d_caug, sizeof(float) * B, cudaMemcpyDeviceToDevice, b->stream));
    if (trace->proj_idx) CK(b, cudaMemcpyAsync(trace->proj_idx, b->d_proj, sizeof(int) * np, cudaMemcpyDeviceToDevice, b->stream));
    if (trace->elite_idx) CK(b, cudaMemcpyAsync(trace->elite_idx, b->d_elite, sizeof(int) * ne, cudaMemcpyDeviceToDevice, b->stream));
  }
  return TRAJ_OK;
}

traj_status traj_sampler_step(traj_batch *b, const traj_sampler_config *sc, int iteration,
                              float *mu, float *sigma, const float *z, float *best,
                              const traj_sampler_trace *trace) {
  return traj_sampler_step_multi(b, sc, iteration, 1, mu, sigma, z, best, trace);
}

traj_status traj_gemm_bf16(int M, int N, int K, const void *A, const void *B, float *C, int *err,
                           void *cuda_stream) {
  if (!A || !B || !C || !err || M < 1 || N < 1 || K < 1 || (K % 8) != 0) return TRAJ_EINVAL;
  cudaError_t e = launch_gemm_bf16(0, A, B, M, N, K, C, nullptr, N, nullptr, nullptr, err,
                                   reinterpret_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess) { g_create_error = cudaGetErrorString(e); return TRAJ_ECUDA; }
  return TRAJ_OK;
}

traj_status traj_measure_fp32_peak(void *cuda_stream, int reps, double *flops_per_s) {
  if (!flops_per_s || reps < 1) return TRAJ_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  int dev = 0, n_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return TRAJ_ECUDA;
  }
  float *out = nullptr;
  cudaEvent_t e0, e1;
  if (cudaMalloc(&out, sizeof(float) * n_sm * 8) != cudaSuccess) return TRAJ_ENOMEM;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int blocks = n_sm * 8, iters = 4096;
  // both kernels run 8 x 16 x iters FMA instructions per thread; the packed one
  // does two FP32 FMAs per instruction
  const double flops1 = 2.0 * 8 * 16 * (double)iters * 256.0 * blocks;
  double best = 0.0;
  traj_status rc = TRAJ_OK;
  for (int kind = 0; kind < 2; ++kind) {
    const double flops = kind == 0 ? flops1 : 2.0 * flops1;
    for (int r = 0; r <= reps && rc == TRAJ_OK; ++r) {
      cudaEventRecord(e0, s);
      cudaError_t le = kind == 0 ? tb::launch_ffma_peak(out, blocks, iters, s)
                                 : tb::launch_ffma2_peak(out, blocks, iters, s);
      if (le != cudaSuccess) rc = TRAJ_ECUDA;
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) rc = TRAJ_ECUDA;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (r > 0 && ms > 0) best = std::max(best, flops / (ms * 1e-3));
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  *flops_per_s = best;
  return rc;
}

traj_status traj_measure_mufu_peak(void *cuda_stream, int reps, double *rsqrt_per_s) {
  if (!rsqrt_per_s || reps < 1) return TRAJ_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  int dev = 0, n_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return TRAJ_ECUDA;
  }
  float *out = nullptr;
  cudaEvent_t e0, e1;
  if (cudaMalloc(&out, sizeof(float) * n_sm * 8) != cudaSuccess) return TRAJ_ENOMEM;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int blocks = n_sm * 8, iters = 1024;
  const double ops = 8.0 * 16 * (double)iters * 256.0 * blocks; // rsqrtf per launch
  double best = 0.0;
  traj_status rc = TRAJ_OK;
  for (int r = 0; r <= reps && rc == TRAJ_OK; ++r) {
    cudaEventRecord(e0, s);
    if (tb::launch_rsqrt_peak(out, blocks, iters, s) != cudaSuccess) rc = TRAJ_ECUDA;
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) rc = TRAJ_ECUDA;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (r > 0 && ms > 0) best = std::max(best, ops / (ms * 1e-3));
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  *rsqrt_per_s = best;
  return rc;
}

} // extern "C"

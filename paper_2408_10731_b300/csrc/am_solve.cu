// am_solve.cu -- the fused persistent kernel of the batched AM optimizer.
//
// One warp owns one trajectory for its whole solve; warps pull trajectories
// from an atomic work queue (ordered by estimated cost), so a batch with
// uneven obstacle counts and horizons runs in a single launch. Per iteration
// of Algorithm 2 (Paper II):
//
//  Line 2 (xi-step, eqs. zeta_1_sepration_1/3 solved as in eq. over_3):
//     xi^k = hq + G xi^{k-1} + K11 (lambda^{k-1} - rho u^{k-1}),
//     the algebraic rewrite of K11 (-q + lambda + rho F^T g) + K12 b with
//     F^T g = F^T F xi - u, u = F^T (F xi - g), G = rho K11 F^T F and
//     hq = K11 (-q) + K12 b precomputed in FP64. It runs in compensated FP32
//     (K11, G, hq stored as FP32 hi/lo pairs, exact products, TwoSum
//     accumulation): plain FP32 loses ~5 bits to the KKT inverse's
//     conditioning.
//  Lines 4-5 (eqs. zeta_2, compute_d_mij, d_max, alpha_v/a, compute_dv/a):
//     for every obstacle j and timestep t, Delta = p(t) - o_j(t) with
//     o_j(t) = c_j + v_j t, u = Delta / axes, and the alternating alpha-then-d
//     steps give g_j - o_j = Delta * max(1, 1/||u||), so the residual
//     r_j = p - g_j = -Delta * max(0, 1/||u||-1) is zero outside the ellipse
//     and needs one rsqrt inside it (no atan2/cos/sin: identical values).
//     Velocity / acceleration: r = w * max(0, 1 - bound/||w||).
//  Line 6 (eq. update_lambda2_1): u^k = F^T r^k = P^T sum_j r_j + Pd^T r_v +
//     Pdd^T r_a (the stacked F is never formed), lambda^k = lambda^{k-1} - rho u^k.
//  Stop: L-infinity residuals (obstacle, velocity, acceleration) all <= tol.
//
// Lanes own timesteps t = lane + 32 m for evaluation, projection and the
// contraction; the contraction's 11 x dim partial sums are reduce-scattered
// over the warp so that lane 16 a + i owns coefficient i of axis a (axis 2 in
// 3D: lanes i and 16 + i).
#include "internal.cuh"
#include "am_device.cuh"

namespace tb {

constexpr int MAX_WARPS_PER_BLOCK = 8;

template <int DIM, int MAXNT, bool CHUNKED = false>
__device__ __noinline__ void solve_one(const SolveArgs &A, int b, const float *stab, int lane,
                                       unsigned long long deadline) {
  const int p = A.traj_problem[b];
  const ProblemDev pr = A.problems[p];
  const int n_p = pr.n_p;
  const int nt = (n_p + 31) >> 5;
  const float *Cb = A.constants + pr.const_off, *C = Cb; // constants of the penalty level
  const float *tP = stab + pr.tbl_off;
  const float *tD = tP + n_p * ROW;
  const float *tA = tD + n_p * ROW;
  const float4 *obs = A.obstacles + (size_t)pr.pair_off * pair_vec(DIM);
  float rho = A.rho;

  // ownership: lane 16 a + i holds coefficient i of axis a (a < 2); axis 2 of a 3D
  // trajectory is held (twice) by lanes i and 16 + i.
  const int oi = lane & 15, oa = lane >> 4;
  const int ri = oi < NC ? oi : NC - 1; // clamped row for the non-owner lanes
  const float *x0 = A.xi0 + (size_t)b * DIM * NC;
  float xo = x0[oa * NC + ri];
  float xo2 = DIM == 3 ? x0[2 * NC + ri] : 0.f;
  bool finite = isfinite(xo) && isfinite(xo2);
  finite = __all_sync(FULL, finite) && pr.nan_flag == 0;

  float *xout = A.xi + (size_t)b * DIM * NC;
  if (!finite) {
    if (oi < NC) {
      xout[oa * NC + oi] = xo;
      if (DIM == 3 && oa == 0) xout[2 * NC + oi] = xo2;
    }
    if (lane < 3) A.res[b * 3 + lane] = __int_as_float(0x7fc00000);
    if (lane == 0) { A.iters[b] = 0; A.status[b] = 2; atomicOr(A.flags, 2); }
    return;
  }

  // hq of the first penalty level (projection mode: from the sample xs)
  const float xs = xo, xs2 = xo2;
  float hq_hi, hq_lo, hq2_hi, hq2_lo;
  load_hq<DIM>(C, A.cost_mode, lane, xs, xs2, hq_hi, hq_lo, hq2_hi, hq2_lo);
  int level = 0;

  float lam = 0.f, lam2 = 0.f, uo = 0.f, uo2 = 0.f;
  float mo, mv, ma;
  int k = 0;
  if (A.lam0) { // resume from (xi, lambda, u) of an earlier solve, or carry lambda over a shift
    resume_state<DIM>(A, b, oa, ri, lam, lam2, uo, uo2);
    k = A.u0 ? 1 : 0; // resume: the next step is a QP step; carry: project first
  }
  signed char st = 1;
  for (;; ++k) {
    if (k > 0) qp_step<DIM>(C, lane, rho, hq_hi, hq_lo, hq2_hi, hq2_lo, lam, lam2, uo, uo2, xo, xo2);
    float2 xp[DIM][6];
    broadcast_pairs<DIM>(xo, xo2, xp);
    float2 up[DIM][6];
    if constexpr (CHUNKED)
      project_contract_chunked<DIM, MAXNT>(xp, tP, tD, tA, obs, A.problems + p, n_p, pr.dt,
                                           pr.invT, pr.invT2, A.vmax, A.amax, lane, up, mo, mv, ma);
    else
      project_contract<DIM, MAXNT, true>(xp, tP, tD, tA, obs, A.problems + p, n_p, nt, pr.dt, pr.invT,
                                   pr.invT2, A.vmax, A.amax, lane, up, mo, mv, ma);
    scatter_pairs<DIM>(up, lane, uo, uo2);
    mo = warp_max(mo); mv = warp_max(mv); ma = warp_max(ma);
    if (k > 0) { // Line 6: multiplier update (lambda0 = 0 at the initial projection)
      lam -= rho * uo;
      if (DIM == 3) lam2 -= rho * uo2;
      if (A.tol >= 0.f && sqrtf(mo) <= A.tol && sqrtf(mv) <= A.tol && sqrtf(ma) <= A.tol) {
        st = 0;
        break;
      }
    }
    if (k >= A.max_iters) { st = 1; break; }
    if (deadline) {
      unsigned long long now = 0;
      if (lane == 0) now = globaltimer_ns();
      now = __shfl_sync(FULL, now, 0);
      if (now > deadline) { st = 3; break; }
    }
    rho_step<DIM>(A, k, level, Cb, C, rho, lane, xs, xs2, hq_hi, hq_lo, hq2_hi, hq2_lo);
  }
  if (oi < NC) {
    xout[oa * NC + oi] = xo;
    if (A.lam) A.lam[(size_t)b * DIM * NC + oa * NC + oi] = lam;
    if (A.u) A.u[(size_t)b * DIM * NC + oa * NC + oi] = uo;
    if (DIM == 3 && oa == 0) {
      xout[2 * NC + oi] = xo2;
      if (A.lam) A.lam[(size_t)b * DIM * NC + 2 * NC + oi] = lam2;
      if (A.u) A.u[(size_t)b * DIM * NC + 2 * NC + oi] = uo2;
    }
  }
  if (lane == 0) {
    A.res[b * 3 + 0] = sqrtf(mo);
    A.res[b * 3 + 1] = sqrtf(mv);
    A.res[b * 3 + 2] = sqrtf(ma);
    A.iters[b] = k;
    A.status[b] = st;
    if (st == 3) atomicOr(A.flags, 1);
  }
}

// ---- W warps per trajectory (W = 2 or 4) ---------------------------------------------
// The team's warps r = 0 .. W-1 own the 32-point blocks W m + r of the grid,
// t = 32 (W m + r) + lane: a slot holds 32 consecutive grid points, so the culled
// pair loop bounds it as tightly as one warp's, and every warp runs at most
// ceil(n_p / 32 W) slots, as an interleaved split would. Each evaluates, projects and
// contracts its timesteps; the partial contractions (after each warp's
// reduce-scatter) and the residual maxima are exchanged through double-buffered
// shared memory with one named barrier per iteration, and every warp adds them in
// the same order (r = 0, 1, ...), so all hold bitwise-identical u, lambda and xi
// and take the same decisions. The compensated QP step runs redundantly in each.
constexpr int XCH = 72; // floats per exchange slot: u (32 lanes), u of axis 2 (32), maxima, flag

__device__ __forceinline__ void team_bar(int id, int threads) {
  asm volatile("bar.sync %0, %1;" :: "r"(id), "r"(threads) : "memory");
}

template <int DIM, int NT, int W>
__device__ __noinline__ void solve_team(const SolveArgs &A, int b, const float *stab, int lane,
                                        int r, float *xch, int bar_id,
                                        unsigned long long deadline) {
  const int p = A.traj_problem[b];
  const ProblemDev pr = A.problems[p];
  const int n_p = pr.n_p;
  const float *Cb = A.constants + pr.const_off, *C = Cb;
  const float *tP = stab + pr.tbl_off;
  const float *tD = tP + n_p * ROW;
  const float *tA = tD + n_p * ROW;
  const float4 *obs = A.obstacles + (size_t)pr.pair_off * pair_vec(DIM);
  float rho = A.rho;
  const int oi = lane & 15, oa = lane >> 4;
  const int ri = oi < NC ? oi : NC - 1;
  const float *x0 = A.xi0 + (size_t)b * DIM * NC;
  float xo = x0[oa * NC + ri];
  float xo2 = DIM == 3 ? x0[2 * NC + ri] : 0.f;
  bool finite = isfinite(xo) && isfinite(xo2);
  finite = __all_sync(FULL, finite) && pr.nan_flag == 0;
  float *xout = A.xi + (size_t)b * DIM * NC;
  if (!finite) {
    if (r == 0) {
      if (oi < NC) {
        xout[oa * NC + oi] = xo;
        if (DIM == 3 && oa == 0) xout[2 * NC + oi] = xo2;
      }
      if (lane < 3) A.res[b * 3 + lane] = __int_as_float(0x7fc00000);
      if (lane == 0) { A.iters[b] = 0; A.status[b] = 2; atomicOr(A.flags, 2); }
    }
    return;
  }
  const float xs = xo, xs2 = xo2;
  float hq_hi, hq_lo, hq2_hi, hq2_lo;
  load_hq<DIM>(C, A.cost_mode, lane, xs, xs2, hq_hi, hq_lo, hq2_hi, hq2_lo);
  int level = 0;
  float lam = 0.f, lam2 = 0.f, uo = 0.f, uo2 = 0.f;
  float mo, mv, ma;
  int k = 0, par = 0;
  if (A.lam0) {
    resume_state<DIM>(A, b, oa, ri, lam, lam2, uo, uo2);
    k = A.u0 ? 1 : 0; // resume: the next step is a QP step; carry: project first
  }
  signed char st = 1;
  for (;; ++k) {
    if (k > 0) qp_step<DIM>(C, lane, rho, hq_hi, hq_lo, hq2_hi, hq2_lo, lam, lam2, uo, uo2, xo, xo2);
    float2 xp[DIM][6];
    broadcast_pairs<DIM>(xo, xo2, xp);
    float2 up[DIM][6];
    project_contract<DIM, NT, true>(xp, tP, tD, tA, obs, A.problems + p, n_p, NT, pr.dt, pr.invT,
                                    pr.invT2, A.vmax, A.amax, 32 * r + lane, up, mo, mv, ma, 32 * W);
    float part = 0.f, part2 = 0.f;
    scatter_pairs<DIM>(up, lane, part, part2);
    mo = warp_max(mo); mv = warp_max(mv); ma = warp_max(ma);
    // exchange with the partner warps
    float *mine = xch + (par * W + r) * XCH;
    mine[lane] = part;
    if (DIM == 3) mine[32 + lane] = part2;
    if (lane == 0) {
      mine[64] = mo; mine[65] = mv; mine[66] = ma;
      float late = 0.f;
      if (r == 0 && deadline && globaltimer_ns() > deadline) late = 1.f;
      mine[67] = late;
    }
    team_bar(bar_id, 32 * W);
    const float *s0 = xch + par * W * XCH;
    uo = s0[lane];
    if (DIM == 3) uo2 = s0[32 + lane];
    mo = s0[64]; mv = s0[65]; ma = s0[66];
#pragma unroll
    for (int w = 1; w < W; ++w) {
      const float *sw = s0 + w * XCH;
      uo += sw[lane];
      if (DIM == 3) uo2 += sw[32 + lane];
      mo = fmaxf(mo, sw[64]); mv = fmaxf(mv, sw[65]); ma = fmaxf(ma, sw[66]);
    }
    const bool late = s0[67] != 0.f;
    par ^= 1;
    if (k > 0) {
      lam -= rho * uo;
      if (DIM == 3) lam2 -= rho * uo2;
      if (A.tol >= 0.f && sqrtf(mo) <= A.tol && sqrtf(mv) <= A.tol && sqrtf(ma) <= A.tol) {
        st = 0;
        break;
      }
    }
    if (k >= A.max_iters) { st = 1; break; }
    if (late) { st = 3; break; }
    rho_step<DIM>(A, k, level, Cb, C, rho, lane, xs, xs2, hq_hi, hq_lo, hq2_hi, hq2_lo);
  }
  if (r == 0) {
    if (oi < NC) {
      xout[oa * NC + oi] = xo;
      if (A.lam) A.lam[(size_t)b * DIM * NC + oa * NC + oi] = lam;
      if (A.u) A.u[(size_t)b * DIM * NC + oa * NC + oi] = uo;
      if (DIM == 3 && oa == 0) {
        xout[2 * NC + oi] = xo2;
        if (A.lam) A.lam[(size_t)b * DIM * NC + 2 * NC + oi] = lam2;
        if (A.u) A.u[(size_t)b * DIM * NC + 2 * NC + oi] = uo2;
      }
    }
    if (lane == 0) {
      A.res[b * 3 + 0] = sqrtf(mo);
      A.res[b * 3 + 1] = sqrtf(mv);
      A.res[b * 3 + 2] = sqrtf(ma);
      A.iters[b] = k;
      A.status[b] = st;
      if (st == 3) atomicOr(A.flags, 1);
    }
  }
}

template <int DIM, int NT, int MAXNT, int W>
__device__ __forceinline__ void team_nt(const SolveArgs &A, int b, const float *stab, int lane,
                                        int r, float *xch, int bar_id,
                                        unsigned long long deadline, int nt) {
  if constexpr (NT >= MAXNT) {
    solve_team<DIM, MAXNT, W>(A, b, stab, lane, r, xch, bar_id, deadline);
  } else {
    if (nt <= NT) solve_team<DIM, NT, W>(A, b, stab, lane, r, xch, bar_id, deadline);
    else team_nt<DIM, NT + 1, MAXNT, W>(A, b, stab, lane, r, xch, bar_id, deadline, nt);
  }
}

template <int DIM, int MAXNT, int W>
__global__ void __launch_bounds__(MAX_WARPS_PER_BLOCK * 32, 2)
k_am_team(const __grid_constant__ SolveArgs A) {
  extern __shared__ float4 smem4[];
  const int nteam = blockDim.x / (32 * W);
  const float4 *g4 = reinterpret_cast<const float4 *>(A.tables);
  for (int i = threadIdx.x; i < A.table_floats_total / 4; i += blockDim.x) smem4[i] = g4[i];
  float *stab = reinterpret_cast<float *>(smem4);
  float *xch_all = stab + A.table_floats_total;          // [teams][2 parities][W warps][XCH]
  int *sitem = reinterpret_cast<int *>(xch_all + nteam * 2 * W * XCH);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int team = warp / W, r = warp % W, bar_id = 1 + team;
  float *xch = xch_all + team * 2 * W * XCH;

  unsigned long long deadline = 0;
  if (A.timeout_ns) {
    unsigned long long t0 = 0;
    if (lane == 0) {
      const unsigned long long now = globaltimer_ns();
      const unsigned long long prev = atomicCAS(A.t0, 0ull, now);
      t0 = prev ? prev : now;
    }
    deadline = __shfl_sync(FULL, t0, 0) + A.timeout_ns;
  }
  for (;;) {
    if (r == 0 && lane == 0) sitem[team] = atomicAdd(A.queue, 1);
    team_bar(bar_id, 32 * W);
    const int item = sitem[team];
    team_bar(bar_id, 32 * W);
    if (item >= A.n_traj) break;
    const int b = A.order[item];
    const int nt = (A.problems[A.traj_problem[b]].n_p + 32 * W - 1) / (32 * W);
    team_nt<DIM, 1, MAXNT, W>(A, b, stab, lane, r, xch, bar_id, deadline, nt);
  }
}

// Per-trajectory specialisation on the number of 32-step timestep slots, so a
// short horizon in an uneven batch does not pay for the longest one's slots.
template <int DIM, int NT, int MAXNT>
__device__ __forceinline__ void solve_nt(const SolveArgs &A, int b, const float *stab, int lane,
                                         unsigned long long deadline, int nt) {
  if constexpr (NT >= MAXNT) {
    solve_one<DIM, MAXNT>(A, b, stab, lane, deadline);
  } else {
    if (nt <= NT) solve_one<DIM, NT>(A, b, stab, lane, deadline);
    else solve_nt<DIM, NT + 1, MAXNT>(A, b, stab, lane, deadline, nt);
  }
}

// CAP: the occupancy build (at most 4 warps per block, 128 registers, four blocks
// per SM); otherwise registers are unrestricted (one block of up to 8 warps).
template <int DIM, int MAXNT, bool CAP = false>
__global__ void __launch_bounds__(CAP ? 128 : MAX_WARPS_PER_BLOCK * 32, CAP ? 4 : 1)
k_am_fp32(const __grid_constant__ SolveArgs A) {
  extern __shared__ float4 smem4[];
  const float4 *g4 = reinterpret_cast<const float4 *>(A.tables);
  for (int i = threadIdx.x; i < A.table_floats_total / 4; i += blockDim.x) smem4[i] = g4[i];
  __syncthreads();
  const float *stab = reinterpret_cast<const float *>(smem4);
  const int lane = threadIdx.x & 31;

  unsigned long long deadline = 0;
  if (A.timeout_ns) {
    unsigned long long t0 = 0;
    if (lane == 0) {
      const unsigned long long now = globaltimer_ns();
      const unsigned long long prev = atomicCAS(A.t0, 0ull, now);
      t0 = prev ? prev : now;
    }
    deadline = __shfl_sync(FULL, t0, 0) + A.timeout_ns;
  }
  for (;;) {
    int item = 0;
    if (lane == 0) item = atomicAdd(A.queue, 1);
    item = __shfl_sync(FULL, item, 0);
    if (item >= A.n_traj) break;
    const int b = A.order[item];
    const int nt = (A.problems[A.traj_problem[b]].n_p + 31) >> 5;
    solve_nt<DIM, 1, MAXNT>(A, b, stab, lane, deadline, nt);
  }
}

// Horizons beyond 32 * 8 grid points: one warp per trajectory, the timesteps
// streamed in chunks of long_cnt slots per iteration (256 grid points in 2D, 128
// in 3D, where eight slots would spill). Basis tables are staged in shared memory
// as in k_am_fp32 (at most 160 KB).
template <int DIM> __host__ __device__ constexpr int long_cnt() { return DIM == 2 ? 8 : 4; }

template <int DIM>
__global__ void __launch_bounds__(MAX_WARPS_PER_BLOCK * 32, 1)
k_am_long(const __grid_constant__ SolveArgs A) {
  extern __shared__ float4 smem4[];
  const float4 *g4 = reinterpret_cast<const float4 *>(A.tables);
  for (int i = threadIdx.x; i < A.table_floats_total / 4; i += blockDim.x) smem4[i] = g4[i];
  __syncthreads();
  const float *stab = reinterpret_cast<const float *>(smem4);
  const int lane = threadIdx.x & 31;
  unsigned long long deadline = 0;
  if (A.timeout_ns) {
    unsigned long long t0 = 0;
    if (lane == 0) {
      const unsigned long long now = globaltimer_ns();
      const unsigned long long prev = atomicCAS(A.t0, 0ull, now);
      t0 = prev ? prev : now;
    }
    deadline = __shfl_sync(FULL, t0, 0) + A.timeout_ns;
  }
  for (;;) {
    int item = 0;
    if (lane == 0) item = atomicAdd(A.queue, 1);
    item = __shfl_sync(FULL, item, 0);
    if (item >= A.n_traj) break;
    solve_one<DIM, long_cnt<DIM>(), true>(A, A.order[item], stab, lane, deadline);
  }
}

template <int W> struct TeamKernel {
  template <int DIM, int MAXNT, bool CAP> static constexpr auto get() { return k_am_team<DIM, (MAXNT + W - 1) / W, W>; }
};
template <> struct TeamKernel<1> {
  template <int DIM, int MAXNT, bool CAP> static constexpr auto get() { return k_am_fp32<DIM, MAXNT, CAP>; }
};

template <int DIM, int MAXNT, int W, bool CAP = false>
static cudaError_t launch_t(const SolveArgs &a, const LaunchShape &shape, int n_sm,
                            cudaStream_t s, LaunchShape *used) {
  auto kern = TeamKernel<W>::template get<DIM, MAXNT, CAP>();
  const int warps = shape.warps_per_block > 0 ? shape.warps_per_block : 4;
  if (warps > (CAP ? 4 : MAX_WARPS_PER_BLOCK) || warps % W != 0) return cudaErrorInvalidValue;
  const size_t smem = sizeof(float) * (size_t)a.table_floats_total +
                      (W > 1 ? (size_t)(warps / W) * (2 * W * XCH * sizeof(float) + sizeof(int)) : 0);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, warps * 32, smem);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  if (shape.blocks_per_sm > 0 && shape.blocks_per_sm < occ) occ = shape.blocks_per_sm;
  long long want = ((long long)a.n_traj * W + warps - 1) / warps;
  long long grid = (long long)n_sm * occ;
  if (want < grid) grid = want;
  if (grid < 1) grid = 1;
  if (used) {
    used->warps_per_block = warps; used->blocks_per_sm = occ; used->grid = (int)grid; used->team = W;
    used->occupancy = CAP ? 1 : 0;
    cudaFuncAttributes fa{};
    used->regs = cudaFuncGetAttributes(&fa, kern) == cudaSuccess ? fa.numRegs : 0;
    used->smem = (int)smem;
  }
  kern<<<(unsigned)grid, warps * 32, smem, s>>>(a);
  return cudaGetLastError();
}

// k_am_long: the shape's warps per block and blocks per SM apply; the team is one warp.
// Default warps per block (0): the fewest that still hold the whole batch in one wave
// of resident blocks, so that a batch with large tables (one block per SM) is spread
// over every SM rather than packed into fewer, fuller ones.
template <int DIM>
static cudaError_t launch_long(const SolveArgs &a, const LaunchShape &shape, int n_sm,
                               cudaStream_t s, LaunchShape *used) {
  int warps = shape.warps_per_block > 0 ? shape.warps_per_block : MAX_WARPS_PER_BLOCK;
  if (warps > MAX_WARPS_PER_BLOCK) return cudaErrorInvalidValue;
  const size_t smem = sizeof(float) * (size_t)a.table_floats_total;
  cudaError_t e = cudaFuncSetAttribute(k_am_long<DIM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  auto resident = [&](int w, int &occ) -> cudaError_t {
    cudaError_t r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_am_long<DIM>, w * 32, smem);
    if (r == cudaSuccess && shape.blocks_per_sm > 0 && shape.blocks_per_sm < occ) occ = shape.blocks_per_sm;
    return r;
  };
  int occ = 0;
  if ((e = resident(warps, occ)) != cudaSuccess) return e;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  while (shape.warps_per_block <= 0 && warps > 1) {
    int occ_less = 0;
    if ((e = resident(warps - 1, occ_less)) != cudaSuccess) return e;
    if ((long long)n_sm * occ_less * (warps - 1) < a.n_traj) break;
    --warps;
    occ = occ_less;
  }
  long long want = ((long long)a.n_traj + warps - 1) / warps;
  long long grid = (long long)n_sm * occ;
  if (want < grid) grid = want;
  if (grid < 1) grid = 1;
  if (used) { used->warps_per_block = warps; used->blocks_per_sm = occ; used->grid = (int)grid; used->team = 1; used->occupancy = 0; }
  k_am_long<DIM><<<(unsigned)grid, warps * 32, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_am_solve(int dim, int max_np, int precision, const SolveArgs &a,
                            const LaunchShape &shape, int n_sm, cudaStream_t s, LaunchShape *used) {
  if (precision == 1 || precision == 2)
    return launch_am_mixed(dim, max_np, precision == 2, a, shape, n_sm, s, used);
  const int nt = (max_np + 31) / 32;
  if (nt > 8) { // long horizons: chunked, one warp per trajectory
    if (shape.team != 0 && shape.team != 1) return cudaErrorInvalidValue;
    return dim == 2 ? launch_long<2>(a, shape, n_sm, s, used) : launch_long<3>(a, shape, n_sm, s, used);
  }
  const int team = shape.team;
  if (team != 0 && team != 1 && team != 2 && team != 4) return cudaErrorInvalidValue;
  if (shape.occupancy) { // the register-capped build: one warp per trajectory, n_p <= 160
    if (team > 1 || nt > 5) return cudaErrorInvalidValue;
    if (dim == 2) return nt <= 4 ? launch_t<2, 4, 1, true>(a, shape, n_sm, s, used)
                                 : launch_t<2, 5, 1, true>(a, shape, n_sm, s, used);
    return nt <= 4 ? launch_t<3, 4, 1, true>(a, shape, n_sm, s, used)
                   : launch_t<3, 5, 1, true>(a, shape, n_sm, s, used);
  }
#define TB_PICK(D, N)                                                                   \
  return team == 4 ? launch_t<D, N, 4>(a, shape, n_sm, s, used)                         \
       : team == 2 ? launch_t<D, N, 2>(a, shape, n_sm, s, used)                         \
                   : launch_t<D, N, 1>(a, shape, n_sm, s, used)
  if (dim == 2) {
    if (nt <= 4) TB_PICK(2, 4);
    if (nt <= 5) TB_PICK(2, 5);
    TB_PICK(2, 8);
  }
  if (nt <= 4) TB_PICK(3, 4);
  if (nt <= 5) TB_PICK(3, 5);
  TB_PICK(3, 8);
#undef TB_PICK
}

} // namespace tb

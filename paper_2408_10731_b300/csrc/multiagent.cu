// multiagent.cu -- the joint multi-agent trajectory optimizer of Paper IV
// (Algorithm 5) for a batch of independent scenes, one CTA per scene.
//
// Per scene: N agents (degree-10 Bernstein coefficients per axis), each pair
// (i, j) kept apart by x_i - x_j = d_ij e(alpha_ij, beta_ij), d_ij >= 1, with
// e on the spheroid (a, a, b) (eq. sphere_proposed), and static spheres kept
// out the same way. Cost 1/2 sum_i xi_i^T Pdd^T Pdd xi_i; start and goal fixed
// with zero velocity and acceleration (eqs. eq_multiagent_start/final).
//
// The x-step (eq. kkt_step_x) couples all agents of a scene through
// A_fo^T A_fo = 2 (N I - 1 1^T) (x) P^T P (+ n_o I (x) P^T P for the static
// spheres). That matrix is diagonal in the agent-mean / deviation basis, so the
// (11 N)-variable KKT system splits into two 17 x 17 ones, formed and inverted
// in FP64 once per scene and penalty (k_ma_setup):
//   mean      xi_bar: [Pdd^T Pdd + rho n_o S, A^T; A, 0]
//   deviation xi_i - xi_bar: [Pdd^T Pdd + rho (n_o + 2N) S, A^T; A, 0]   (S = P^T P).
// With the pair targets written as delta - r (r the residual of the d-step), the
// x-step becomes an increment on the previous iterate:
//   xi_bar' = G_m xi_bar - H_m u_bar + E_m e_bar
//   dlt_i'  = G_d dlt_i  - H_d (u_i - u_bar) + E_d (e_i - e_bar)
// with u_i = P^T w_i, w_i = sum_j 2 (r_ij + lambda_ij / rho') + sum_o (r_io +
// lambda_io / rho'), and the constants and the iterate (xi_bar, dlt) kept as
// FP32 (hi, lo) pairs: the joint problem amplifies rounding of the iterate, so a
// plain FP32 iterate drifts from the FP64 result by ~1e-5 m within tens of
// iterations on crowded scenes.
//
// The pair pass takes each unordered pair (i < j) once per grid point: e from
// the closed form of eqs. com_alpha_i / com_beta_i (e = delta / R with R the
// spheroid norm of delta; e = (0, 0, b), or (a, 0) in 2D, at delta = 0), d from
// eq. com_d_i with d >= 1, and lambda += rho r (eqs. update_lamda_*). The
// multipliers of agent pairs live in shared memory when they fit, otherwise in
// device memory; w is rebuilt from the new and old multiplier sums, since
// r = (lambda' - lambda) / rho.
#include "trajbatch.h"
#include "internal.cuh"
#include "nvtx_range.h"
#include "basis.cuh"
#include "linalg.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

namespace tb {
namespace {

constexpr int MA_NE = 6;             // boundary rows: p, p', p'' at both ends
constexpr int MA_NK = NC + MA_NE;    // 17
constexpr int MA_MAX_AGENTS = 64;
constexpr int MA_THREADS = 1024;
// constants of one scene and penalty level (floats): six (hi, lo) matrices
constexpr int MA_G_M = 0, MA_H_M = 242, MA_E_M = 484, MA_G_D = 616, MA_H_D = 858, MA_E_D = 1100;
constexpr int MA_LEVEL_FLOATS = 1232;
constexpr int MA_FREE_FLOATS = 132; // free-init E (hi, lo)

struct MaArgs {
  int n_scenes, N, n_p, npairs, levels, rho_every, max_iters, lam_in_smem;
  float tol;
  const float *rho_ladder;  // [levels]
  const float *P;           // [n_p][ROW] position basis
  const float *consts;      // [S][levels][MA_LEVEL_FLOATS]
  const float *consts_free; // [S][MA_FREE_FLOATS]
  const float *start, *goal; // [S][N][dim]
  const float2 *shape;      // [S] (r, h) of the agents
  const int *obs_off;       // [S + 1]
  const float4 *obs;        // [n_obs] (centre, radius)
  float *lam_ag;            // [S][npairs][dim][n_p] (when not in shared memory)
  float *lam_ob;            // [n_obs][N][dim][n_p]
  float *xi_out;            // [S][N][dim][NC]
  float *res_out;           // [S]
  int *iters_out;           // [S]
};

// shared-memory carve-up in floats (identical on host and device)
struct MaSmem {
  int P, xbar, xbar_n, dlt0, dlt1, u, ubar, pos, w, Lold, lam, se, red, total;
};

__host__ __device__ inline MaSmem ma_smem(int dim, int N, int n_p, int npairs, bool lam_in_smem) {
  MaSmem m;
  int o = 0;
  auto take = [&](int n) { int r = o; o += (n + 3) & ~3; return r; };
  m.P = take(n_p * ROW);
  m.xbar = take(2 * dim * NC); // (hi, lo) halves
  m.xbar_n = take(2 * dim * NC);
  m.dlt0 = take(2 * N * dim * NC);
  m.dlt1 = take(2 * N * dim * NC);
  m.u = take(N * dim * NC);
  m.ubar = take(dim * NC);
  m.pos = take(N * dim * n_p);
  m.w = take(N * dim * n_p);
  m.Lold = take(N * dim * n_p);
  m.lam = lam_in_smem ? take(npairs * dim * n_p) : 0;
  m.se = take(2 * N * dim + 4 * (N + 1) * dim); // start, goal; deviations and means (hi, lo)
  m.red = take(64);
  m.total = o;
  return m;
}

// ---- set-up: FP64 KKT inverses per scene and penalty level ------------------------
// grid (scene, level); dynamic shared memory 3 n_p NC doubles
__global__ void k_ma_setup(int N, int n_p, const double *Tarr, const int *obs_off,
                           const float *rho_ladder, float *consts, float *consts_free, int *err) {
  extern __shared__ double smd[];
  __shared__ double S[NC * NC], Q0[NC * NC], Arow[MA_NE * NC], K11[NC * NC];
  __shared__ double W[MA_NK * 2 * MA_NK];
  __shared__ int piv, bad;
  const int s = blockIdx.x, l = blockIdx.y, levels = gridDim.y;
  const double T = Tarr[s], iT = 1.0 / T, iT2 = iT * iT;
  const int n_o = obs_off[s + 1] - obs_off[s];
  const double rho = (double)rho_ladder[l];
  double *P = smd, *Pd = smd + n_p * NC, *Pdd = smd + 2 * n_p * NC;
  if (threadIdx.x == 0) bad = 0;
  for (int t = threadIdx.x; t < n_p; t += blockDim.x) {
    double a[NC], b[NC], c[NC];
    basis_row(n_p, t, a, b, c);
    for (int i = 0; i < NC; ++i) {
      P[t * NC + i] = a[i];
      Pd[t * NC + i] = b[i] * iT;
      Pdd[t * NC + i] = c[i] * iT2;
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < NC * NC; e += blockDim.x) {
    const int a = e / NC, b = e % NC;
    double ss = 0.0, qq = 0.0;
    for (int t = 0; t < n_p; ++t) {
      ss += P[t * NC + a] * P[t * NC + b];
      qq += Pdd[t * NC + a] * Pdd[t * NC + b];
    }
    S[e] = ss;
    Q0[e] = qq;
  }
  for (int e = threadIdx.x; e < MA_NE * NC; e += blockDim.x) {
    const int r = e / NC, i = e % NC, t = r < 3 ? 0 : n_p - 1;
    const double *src = (r % 3) == 0 ? P : (r % 3) == 1 ? Pd : Pdd;
    Arow[e] = src[t * NC + i];
  }
  __syncthreads();
  // modes: 0 mean, 1 deviation, 2 free initialisation (level 0 only)
  for (int mode = 0; mode < (l == 0 ? 3 : 2); ++mode) {
    const double cS = mode == 0 ? rho * n_o : mode == 1 ? rho * (n_o + 2.0 * N) : 0.0;
    for (int e = threadIdx.x; e < MA_NK * 2 * MA_NK; e += blockDim.x) {
      const int r = e / (2 * MA_NK), c = e % (2 * MA_NK);
      double v = 0.0;
      if (c >= MA_NK) v = (c - MA_NK == r) ? 1.0 : 0.0;
      else if (r < NC && c < NC) v = Q0[r * NC + c] + cS * S[r * NC + c];
      else if (r < NC) v = Arow[(c - NC) * NC + r];
      else if (c < NC) v = Arow[(r - NC) * NC + c];
      W[e] = v;
    }
    __syncthreads();
    gj_invert(W, MA_NK, &piv, &bad);
    for (int e = threadIdx.x; e < NC * NC; e += blockDim.x)
      K11[e] = W[(e / NC) * 2 * MA_NK + MA_NK + (e % NC)];
    __syncthreads();
    if (mode == 2) {
      float *F = consts_free + (size_t)s * MA_FREE_FLOATS;
      for (int e = threadIdx.x; e < NC * MA_NE; e += blockDim.x)
        split2(&F[e], &F[66 + e], W[(e / MA_NE) * 2 * MA_NK + MA_NK + NC + (e % MA_NE)]);
    } else {
      float *C = consts + ((size_t)s * levels + l) * MA_LEVEL_FLOATS;
      const int oG = mode == 0 ? MA_G_M : MA_G_D, oH = mode == 0 ? MA_H_M : MA_H_D,
                oE = mode == 0 ? MA_E_M : MA_E_D;
      for (int e = threadIdx.x; e < NC * NC; e += blockDim.x) {
        const int a = e / NC, b = e % NC;
        double g = 0.0;
        for (int k = 0; k < NC; ++k) g += K11[a * NC + k] * S[k * NC + b];
        split2(&C[oG + e], &C[oG + 121 + e], cS * g);
        split2(&C[oH + e], &C[oH + 121 + e], rho * K11[e]);
      }
      for (int e = threadIdx.x; e < NC * MA_NE; e += blockDim.x)
        split2(&C[oE + e], &C[oE + 66 + e], W[(e / MA_NE) * 2 * MA_NK + MA_NK + NC + (e % MA_NE)]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && bad) atomicOr(err, 1);
}

// ---- solve --------------------------------------------------------------------
// One pair at one grid point: e of eqs. com_alpha_i / com_beta_i in closed form,
// e = delta / R with R the spheroid norm of delta (R^2 = (dx^2 + dy^2) / a^2 +
// dz^2 / b^2); the d-step of eq. com_d_i, d = max(1, e.(delta + lambda / rho) / e.e)
// = max(1, R delta.(delta + lambda / rho) / |delta|^2); the residual
// r = delta - d e = delta (1 - d / R); and the multiplier update lambda += rho r in
// place (the initial pass, lambda = 0, leaves r instead). At delta = 0 the angles
// are 0: e = (0, 0, b) in 3D, (a, 0) in 2D. ia2 = 1 / a^2, ib2 = 1 / b^2.
// Returns ||r||^2.
template <int DIM, bool INIT>
__device__ __forceinline__ float ma_pair(const float (&dl)[DIM], float a, float b, float ia2,
                                         float ib2, float (&lm)[DIM], float rho, float irho) {
  if (INIT) {
#pragma unroll
    for (int k = 0; k < DIM; ++k) lm[k] = 0.f;
  }
  float n2 = 0.f, num = 0.f;
#pragma unroll
  for (int k = 0; k < DIM; ++k) {
    n2 = fmaf(dl[k], dl[k], n2);
    num = fmaf(dl[k], fmaf(lm[k], irho, dl[k]), num);
  }
  float r[DIM];
  if (n2 > 0.f) {
    float R2;
    if constexpr (DIM == 3) R2 = fmaf(dl[2] * dl[2], ib2, (dl[0] * dl[0] + dl[1] * dl[1]) * ia2);
    else R2 = n2 * ia2;
    const float R = sqrtf(R2);
    const float d = fmaxf(__fdividef(R * num, n2), 1.f); // 2-ulp quotients (MUFU reciprocal)
    const float f = 1.f - __fdividef(d, R);
#pragma unroll
    for (int k = 0; k < DIM; ++k) r[k] = dl[k] * f;
  } else {
    const int ax = DIM == 3 ? 2 : 0;
    const float ee = DIM == 3 ? b : a;
    const float d = fmaxf(lm[ax] * irho / ee, 1.f);
#pragma unroll
    for (int k = 0; k < DIM; ++k) r[k] = k == ax ? -d * ee : 0.f;
  }
  float rr = 0.f;
#pragma unroll
  for (int k = 0; k < DIM; ++k) {
    rr = fmaf(r[k], r[k], rr);
    lm[k] = INIT ? r[k] : fmaf(rho, r[k], lm[k]);
  }
  return rr;
}

// The pair pass of one thread: rows of the pair triangle (agent i with every j > i)
// in snake order over the slots, so that each slot gets about npairs / nslot pairs,
// at grid point t_me; the row owner also takes agent i's obstacles and leaves
// 2 sum_{j>i} lambda_ij + sum_o lambda_io (the part of agent i's multiplier sum it
// can form alone) in w. Returns the largest ||r||^2 (NaN as +inf).
template <int DIM, bool INIT>
__device__ __forceinline__ float pair_rows(int N, int n_p, int nslot, int slot, int t_me,
                                           const float *pos, float *lam, float *lamo,
                                           const float4 *obs, int n_o, float2 shp, float rho,
                                           float irho, float *w) {
  const int plane = DIM * n_p;
  const float a_ag = 2.f * shp.x, b_ag = 2.f * shp.y;
  const float ia2 = 1.f / (a_ag * a_ag), ib2 = 1.f / (b_ag * b_ag);
  float rmax = 0.f;
  for (int kb = 0; kb * nslot < N; ++kb) {
    const int i = kb * nslot + ((kb & 1) ? nslot - 1 - slot : slot);
    if (i >= N) continue;
    const float *pin = pos + i * plane + t_me;
    float pi[DIM], part[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) { pi[a] = pin[a * n_p]; part[a] = 0.f; }
    const int np_row = N - 1 - i;
    float *lp = lam + (size_t)(i * (2 * N - i - 1) / 2) * plane + t_me;
    const float *pj = pin + plane;
    float nxt[DIM] = {};
    if (!INIT && np_row > 0)
#pragma unroll
      for (int a = 0; a < DIM; ++a) nxt[a] = lp[a * n_p];
    for (int jj = 0; jj < np_row; ++jj, lp += plane, pj += plane) {
      float lm[DIM], dl[DIM];
#pragma unroll
      for (int a = 0; a < DIM; ++a) lm[a] = nxt[a];
      if (!INIT && jj + 1 < np_row) // the next pair's multipliers, loaded early
#pragma unroll
        for (int a = 0; a < DIM; ++a) nxt[a] = lp[plane + a * n_p];
#pragma unroll
      for (int a = 0; a < DIM; ++a) dl[a] = pi[a] - pj[a * n_p];
      const float rr = ma_pair<DIM, INIT>(dl, a_ag, b_ag, ia2, ib2, lm, rho, irho);
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        lp[a * n_p] = lm[a];
        part[a] += lm[a];
      }
      rmax = fmaxf(rmax, rr != rr ? __int_as_float(0x7f800000) : rr);
    }
#pragma unroll
    for (int a = 0; a < DIM; ++a) part[a] *= 2.f;
    float *lo = lamo + (size_t)i * plane + t_me;
    for (int o = 0; o < n_o; ++o, lo += (size_t)N * plane) {
      const float4 ob = obs[o];
      const float ctr[3] = {ob.x, ob.y, ob.z};
      float dl[DIM], lm[DIM];
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        dl[a] = pi[a] - ctr[a];
        lm[a] = INIT ? 0.f : lo[a * n_p];
      }
      const float ao = shp.x + ob.w, bo = shp.y + ob.w;
      const float rr = ma_pair<DIM, INIT>(dl, ao, bo, 1.f / (ao * ao), 1.f / (bo * bo), lm, rho, irho);
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        lo[a * n_p] = lm[a];
        part[a] += lm[a];
      }
      rmax = fmaxf(rmax, rr != rr ? __int_as_float(0x7f800000) : rr);
    }
#pragma unroll
    for (int a = 0; a < DIM; ++a) w[i * plane + a * n_p + t_me] = part[a];
  }
  return rmax;
}

// (s, e) with s + e = a + b exactly (Knuth's TwoSum)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void block_max(float v, float *red, float *out) {
  // v >= 0 or +inf; NaN is mapped to +inf by the caller
  for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    float m = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) *out = m;
  }
  __syncthreads();
}

template <int DIM>
__global__ void __launch_bounds__(MA_THREADS, 1) k_ma_solve(MaArgs A) {
  extern __shared__ float4 sm4[];
  float *sm = reinterpret_cast<float *>(sm4);
  const int s = blockIdx.x, N = A.N, n_p = A.n_p, npairs = A.npairs;
  const MaSmem L = ma_smem(DIM, N, n_p, npairs, A.lam_in_smem != 0);
  float *Ps = sm + L.P, *xbar = sm + L.xbar, *xbar_n = sm + L.xbar_n;
  float *u = sm + L.u, *ubar = sm + L.ubar;
  float *pos = sm + L.pos, *w = sm + L.w, *Lold = sm + L.Lold, *red = sm + L.red;
  // bv[(i DIM + a) 4 + {0,1,2,3}]: (start hi, lo, goal hi, lo) of agent i's deviation from
  // the agent mean (i < N) and of the mean itself (i = N), as exact float pairs
  float *st = sm + L.se, *gl = st + N * DIM, *bv = gl + N * DIM;
  float *dlt = sm + L.dlt0, *dlt_n = sm + L.dlt1;
  const int xsz = DIM * NC, dsz = N * DIM * NC; // offsets of the lo halves
  const int tid = threadIdx.x, nth = blockDim.x;
  const int plane = DIM * n_p;
  // grid-point-major work split: thread -> (grid point t_me, slot); nslot slots per point
  const int nslot = nth / n_p, t_me = tid % n_p, slot = tid / n_p;
  const bool on = slot < nslot;
  float *lam = A.lam_in_smem ? sm + L.lam : A.lam_ag + (size_t)s * npairs * plane;
  const int ob0 = A.obs_off[s], n_o = A.obs_off[s + 1] - ob0;
  float *lamo = A.lam_ob + (size_t)ob0 * N * plane;
  const float2 shp = A.shape[s];

  // tables, boundary values, pair list
  for (int e = tid; e < n_p * ROW; e += nth) Ps[e] = A.P[e];
  for (int e = tid; e < N * DIM; e += nth) {
    st[e] = A.start[(size_t)s * N * DIM + e];
    gl[e] = A.goal[(size_t)s * N * DIM + e];
  }
  __syncthreads();
  float Prow[NC]; // position basis at this thread's grid point
#pragma unroll
  for (int q = 0; q < NC; ++q) Prow[q] = Ps[t_me * ROW + q];
  for (int e = tid; e < 2 * DIM; e += nth) { // compensated agent means
    const int a = e % DIM;
    const float *src = e < DIM ? st : gl;
    float sh = 0.f, sl = 0.f;
    for (int i = 0; i < N; ++i) {
      float t, er;
      two_sum(sh, src[i * DIM + a], t, er);
      sh = t;
      sl += er;
    }
    const float q = sh / N;
    const float ql = (fmaf(-q, (float)N, sh) + sl) / N;
    bv[(N * DIM + a) * 4 + (e < DIM ? 0 : 2)] = q;
    bv[(N * DIM + a) * 4 + (e < DIM ? 1 : 3)] = ql;
  }
  __syncthreads();
  for (int e = tid; e < 2 * N * DIM; e += nth) { // deviations from the means
    const int ia = e % (N * DIM), a = ia % DIM, c = e < N * DIM ? 0 : 2;
    const float *src = c == 0 ? st : gl;
    float h, l;
    two_sum(src[ia], -bv[(N * DIM + a) * 4 + c], h, l);
    bv[ia * 4 + c] = h;
    bv[ia * 4 + c + 1] = l - bv[(N * DIM + a) * 4 + c + 1];
  }
  __syncthreads();
  // xi^0: the free optimum, split into the agent mean and the deviations (reading M3)
  {
    const float *F = A.consts_free + (size_t)s * MA_FREE_FLOATS;
    for (int e = tid; e < (N + 1) * DIM * NC; e += nth) {
      const int i = e / (DIM * NC), a = (e / NC) % DIM, k = e % NC;
      const float *b4 = bv + (i * DIM + a) * 4;
      float hi = 0.f, lo = 0.f;
      df_fma(hi, lo, F[k * MA_NE + 0], F[66 + k * MA_NE + 0], b4[0]);
      lo = fmaf(F[k * MA_NE + 0], b4[1], lo);
      df_fma(hi, lo, F[k * MA_NE + 3], F[66 + k * MA_NE + 3], b4[2]);
      lo = fmaf(F[k * MA_NE + 3], b4[3], lo);
      float sh, sl;
      two_sum(hi, lo, sh, sl);
      if (i < N) { dlt[(i * DIM + a) * NC + k] = sh; dlt[dsz + (i * DIM + a) * NC + k] = sl; }
      else { xbar[a * NC + k] = sh; xbar[xsz + a * NC + k] = sl; }
    }
  }
  __syncthreads();

  int level = 0, k_done = 0;
  float res = 0.f;
  for (int k = 0; k <= A.max_iters; ++k) {
    const bool init = k == 0;
    const int next = (!init && A.levels > 1 && A.rho_every > 0 && k % A.rho_every == 0 &&
                      level < A.levels - 1) ? level + 1 : level;
    const float rho = A.rho_ladder[level], rho_n = A.rho_ladder[next];
    if (!init) {
      // x-step (eq. kkt_step_x) as the increment on the mean / deviation split
      const float *C = A.consts + ((size_t)s * A.levels + level) * MA_LEVEL_FLOATS;
      for (int e = tid; e < N * DIM * NC; e += nth) {
        const int ia = e / NC, kk = e % NC;
        const float *wr = w + ia * n_p;
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f; // four chains for latency
        int t = 0;
        for (; t + 3 < n_p; t += 4) {
          a0 = fmaf(Ps[t * ROW + kk], wr[t], a0);
          a1 = fmaf(Ps[(t + 1) * ROW + kk], wr[t + 1], a1);
          a2 = fmaf(Ps[(t + 2) * ROW + kk], wr[t + 2], a2);
          a3 = fmaf(Ps[(t + 3) * ROW + kk], wr[t + 3], a3);
        }
        for (; t < n_p; ++t) a0 = fmaf(Ps[t * ROW + kk], wr[t], a0);
        u[e] = (a0 + a1) + (a2 + a3);
      }
      __syncthreads();
      for (int e = tid; e < DIM * NC; e += nth) {
        const int a = e / NC, kk = e % NC;
        float acc = 0.f;
        for (int i = 0; i < N; ++i) acc += u[(i * DIM + a) * NC + kk];
        ubar[e] = acc / N;
      }
      __syncthreads();
      for (int e = tid; e < (N + 1) * DIM * NC; e += nth) {
        const int i = e / (DIM * NC), a = (e / NC) % DIM, kk = e % NC;
        const bool mean = i == N;
        const int oG = mean ? MA_G_M : MA_G_D, oH = mean ? MA_H_M : MA_H_D,
                  oE = mean ? MA_E_M : MA_E_D;
        const float *x = mean ? xbar + a * NC : dlt + (i * DIM + a) * NC;
        const float *xl = x + (mean ? xsz : dsz);
        const float *uu = mean ? ubar + a * NC : u + (i * DIM + a) * NC;
        const float *ub = ubar + a * NC;
        float hi = 0.f, lo = 0.f, h2 = 0.f, l2 = 0.f; // two chains: G x and H u
#pragma unroll
        for (int q = 0; q < NC; ++q) {
          df_fma(hi, lo, C[oG + kk * NC + q], C[oG + 121 + kk * NC + q], x[q]);
          lo = fmaf(C[oG + kk * NC + q], xl[q], lo);
          const float uq = mean ? -uu[q] : ub[q] - uu[q];
          df_fma(h2, l2, C[oH + kk * NC + q], C[oH + 121 + kk * NC + q], uq);
        }
        {
          float sh, sl;
          two_sum(hi, h2, sh, sl);
          hi = sh;
          lo = lo + (l2 + sl);
        }
        const float *b4 = bv + (i * DIM + a) * 4; // i = N: the mean
        df_fma(hi, lo, C[oE + kk * MA_NE + 0], C[oE + 66 + kk * MA_NE + 0], b4[0]);
        lo = fmaf(C[oE + kk * MA_NE + 0], b4[1], lo);
        df_fma(hi, lo, C[oE + kk * MA_NE + 3], C[oE + 66 + kk * MA_NE + 3], b4[2]);
        lo = fmaf(C[oE + kk * MA_NE + 3], b4[3], lo);
        float sh, sl;
        two_sum(hi, lo, sh, sl);
        if (mean) { xbar_n[e - dsz] = sh; xbar_n[xsz + e - dsz] = sl; }
        else { dlt_n[e] = sh; dlt_n[dsz + e] = sl; }
      }
      __syncthreads();
      for (int e = tid; e < 2 * DIM * NC; e += nth) xbar[e] = xbar_n[e];
      float *tmp = dlt; dlt = dlt_n; dlt_n = tmp;
      __syncthreads();
    }
    // positions on the grid from xi = xi_bar + dlt as an exact float pair (cc, in the
    // free second iterate buffer)
    float *cc = dlt_n;
    for (int e = tid; e < dsz; e += nth) {
      const int a = (e / NC) % DIM, q = e % NC;
      float ch, cl;
      two_sum(xbar[a * NC + q], dlt[e], ch, cl);
      cc[e] = ch;
      cc[dsz + e] = cl + (xbar[xsz + a * NC + q] + dlt[dsz + e]);
    }
    __syncthreads();
    if (on)
      for (int ia = slot; ia < N * DIM; ia += nslot) {
        const float *ch = cc + ia * NC, *cl = cc + dsz + ia * NC;
        float acc = 0.f, acl = 0.f;
#pragma unroll
        for (int q = 0; q < NC; ++q) {
          acc = fmaf(Prow[q], ch[q], acc);
          acl = fmaf(Prow[q], cl[q], acl);
        }
        pos[ia * n_p + t_me] = acc + acl;
      }
    __syncthreads();
    // pair pass (eqs. com_alpha_i, com_beta_i, com_d_i, update_lamda_*)
    const float irho = 1.f / rho;
    float rmax = 0.f;
    if (on)
      rmax = init ? pair_rows<DIM, true>(N, n_p, nslot, slot, t_me, pos, lam, lamo, A.obs + ob0, n_o,
                                         shp, rho, irho, w)
                  : pair_rows<DIM, false>(N, n_p, nslot, slot, t_me, pos, lam, lamo, A.obs + ob0,
                                          n_o, shp, rho, irho, w);
    block_max(rmax, red, red + 32);
    res = sqrtf(red[32]);
    k_done = k;
    if (!init && res <= A.tol) break;
    if (k == A.max_iters) break;
    // w_i from the new and old multiplier sums: the row part left in w minus twice the
    // column sum sum_{j<i} lambda_ji (record j (2N - j - 1) / 2 + (i - j - 1))
    const float c1 = 1.f / rho + 1.f / rho_n, c0 = 1.f / rho;
    if (on)
      for (int i = slot; i < N; i += nslot) {
        float dn[DIM];
#pragma unroll
        for (int a = 0; a < DIM; ++a) dn[a] = 0.f;
        const float *lc = lam + (size_t)(i - 1) * plane + t_me; // pair (0, i)
        for (int j = 0; j < i; ++j) {
#pragma unroll
          for (int a = 0; a < DIM; ++a) dn[a] += lc[a * n_p];
          lc += (size_t)(N - j - 2) * plane; // to pair (j + 1, i)
        }
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
          const int e = (i * DIM + a) * n_p + t_me;
          const float acc = w[e] - 2.f * dn[a];
          w[e] = init ? acc : c1 * acc - c0 * Lold[e]; // Lold is not yet written at init
          Lold[e] = init ? 0.f : acc;
        }
      }
    __syncthreads();
    if (init) { // the initial pass stored r in the multiplier slots: lambda^0 = 0
      for (int e = tid; e < npairs * plane; e += nth) lam[e] = 0.f;
      for (int e = tid; e < N * n_o * plane; e += nth) lamo[e] = 0.f;
      __syncthreads();
    }
    level = next;
  }
  // results: xi = xi_bar + dlt
  for (int e = tid; e < N * DIM * NC; e += nth)
    A.xi_out[(size_t)s * N * DIM * NC + e] =
        (xbar[(e / NC) % DIM * NC + e % NC] + dlt[e]) +
        (xbar[xsz + (e / NC) % DIM * NC + e % NC] + dlt[dsz + e]);
  if (tid == 0) {
    A.res_out[s] = res;
    A.iters_out[s] = k_done;
  }
}

// position basis table [n_p][ROW] (FP64 evaluation stored as FP32)
__global__ void k_ma_table(int n_p, float *P) {
  for (int t = threadIdx.x + blockIdx.x * blockDim.x; t < n_p; t += blockDim.x * gridDim.x) {
    double a[NC], b[NC], c[NC];
    basis_row(n_p, t, a, b, c);
    for (int i = 0; i < ROW; ++i) P[t * ROW + i] = i < NC ? (float)a[i] : 0.f;
  }
}

} // namespace
} // namespace tb

// ---- C ABI ------------------------------------------------------------------------
using namespace tb;

struct traj_ma_batch {
  traj_ma_config cfg{};
  cudaStream_t stream = nullptr;
  std::string err;
  int n_scenes = 0, N = 0, n_obs = 0, levels = 1, lam_in_smem = 0;
  bool have_problems = false, have_result = false;
  size_t smem = 0;
  double *d_T = nullptr;
  float *d_P = nullptr, *d_rho = nullptr, *d_consts = nullptr, *d_free = nullptr;
  float *d_start = nullptr, *d_goal = nullptr, *d_lam = nullptr, *d_lamo = nullptr;
  float2 *d_shape = nullptr;
  int *d_obs_off = nullptr, *d_iters = nullptr, *d_err = nullptr;
  float4 *d_obs = nullptr;
  float *d_xi = nullptr, *d_res = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

namespace tb_ma {
thread_local std::string g_ma_error;

traj_status ma_fail(traj_ma_batch *b, traj_status s, const std::string &m) {
  if (b) b->err = m;
  else g_ma_error = m;
  return s;
}

#define MA_CK(b, expr)                                                                  \
  do {                                                                                  \
    cudaError_t e_ = (expr);                                                            \
    if (e_ != cudaSuccess) return ma_fail(b, TRAJ_ECUDA, std::string(#expr ": ") + cudaGetErrorString(e_)); \
  } while (0)

template <class T> cudaError_t ma_alloc(T **p, size_t n) {
  return cudaMalloc(reinterpret_cast<void **>(p), sizeof(T) * (n > 0 ? n : 1));
}

void ma_free_all(traj_ma_batch *b) {
  void *ptrs[] = {b->d_T, b->d_P, b->d_rho, b->d_consts, b->d_free, b->d_start, b->d_goal,
                  b->d_lam, b->d_lamo, b->d_shape, b->d_obs_off, b->d_iters, b->d_err, b->d_obs,
                  b->d_xi, b->d_res};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  if (b->ev0) cudaEventDestroy(b->ev0);
  if (b->ev1) cudaEventDestroy(b->ev1);
}

int max_optin_smem() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 0;
  return v;
}
} // namespace tb_ma
using namespace tb_ma;

extern "C" {

const char *traj_ma_last_error(traj_ma_batch *b) { return b ? b->err.c_str() : g_ma_error.c_str(); }

traj_status traj_ma_create(const traj_ma_config *cfg, void *cuda_stream, traj_ma_batch **out) {
  g_ma_error.clear();
  if (!cfg || !out) return ma_fail(nullptr, TRAJ_EINVAL, "NULL config or output pointer");
  const traj_ma_config &c = *cfg;
  if (c.dim != 2 && c.dim != 3) return ma_fail(nullptr, TRAJ_EINVAL, "dim must be 2 or 3");
  if (c.max_scenes < 1 || c.max_agents < 1 || c.max_agents > MA_MAX_AGENTS || c.max_obstacles < 0 ||
      c.n_steps < 2 || c.n_steps > MAX_STEPS)
    return ma_fail(nullptr, TRAJ_EINVAL, "capacities out of range (agents <= 64, n_steps in [2, 256])");
  if (!(c.rho > 0) || !std::isfinite(c.rho) || c.rho_levels < 0 || c.rho_levels > RHO_MAX_LEVELS ||
      (c.rho_levels > 1 && !(c.rho_growth > 0)) || c.rho_every < 0)
    return ma_fail(nullptr, TRAJ_EINVAL, "rho must be positive; rho_levels in [0, 10]; growth > 0");
  traj_ma_batch *b = new traj_ma_batch();
  b->cfg = c;
  b->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  b->levels = c.rho_levels > 1 ? c.rho_levels : 1;
  const size_t S = c.max_scenes, N = c.max_agents, D = c.dim, np_ = c.n_steps, O = c.max_obstacles;
  const size_t npairs = N * (N - 1) / 2;
  cudaError_t e;
  if ((e = ma_alloc(&b->d_T, S)) || (e = ma_alloc(&b->d_P, np_ * ROW)) ||
      (e = ma_alloc(&b->d_rho, RHO_MAX_LEVELS)) ||
      (e = ma_alloc(&b->d_consts, S * b->levels * MA_LEVEL_FLOATS)) ||
      (e = ma_alloc(&b->d_free, S * MA_FREE_FLOATS)) || (e = ma_alloc(&b->d_start, S * N * D)) ||
      (e = ma_alloc(&b->d_goal, S * N * D)) || (e = ma_alloc(&b->d_lam, S * npairs * D * np_)) ||
      (e = ma_alloc(&b->d_lamo, O * N * D * np_)) || (e = ma_alloc(&b->d_shape, S)) ||
      (e = ma_alloc(&b->d_obs_off, S + 1)) || (e = ma_alloc(&b->d_iters, S)) ||
      (e = ma_alloc(&b->d_err, 1)) || (e = ma_alloc(&b->d_obs, O)) ||
      (e = ma_alloc(&b->d_xi, S * N * D * NC)) || (e = ma_alloc(&b->d_res, S)) ||
      (e = cudaEventCreate(&b->ev0)) || (e = cudaEventCreate(&b->ev1))) {
    g_ma_error = std::string("allocation: ") + cudaGetErrorString(e);
    ma_free_all(b);
    delete b;
    return e == cudaErrorMemoryAllocation ? TRAJ_ENOMEM : TRAJ_ECUDA;
  }
  std::vector<float> ladder(RHO_MAX_LEVELS);
  for (int l = 0; l < RHO_MAX_LEVELS; ++l)
    ladder[l] = (float)(c.rho * std::pow((double)(c.rho_levels > 1 ? c.rho_growth : 1.f), l));
  k_ma_table<<<1, 256, 0, b->stream>>>(c.n_steps, b->d_P);
  if ((e = cudaGetLastError()) != cudaSuccess ||
      (e = cudaMemcpyAsync(b->d_rho, ladder.data(), sizeof(float) * RHO_MAX_LEVELS,
                           cudaMemcpyHostToDevice, b->stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(b->stream)) != cudaSuccess) {
    g_ma_error = std::string("set-up: ") + cudaGetErrorString(e);
    ma_free_all(b);
    delete b;
    return TRAJ_ECUDA;
  }
  *out = b;
  return TRAJ_OK;
}

traj_status traj_ma_destroy(traj_ma_batch *b) {
  if (!b) return TRAJ_EINVAL;
  cudaStreamSynchronize(b->stream);
  ma_free_all(b);
  delete b;
  return TRAJ_OK;
}

traj_status traj_ma_set_problems(traj_ma_batch *b, int n_scenes, int n_agents,
                                 const double *duration, const double *start, const double *goal,
                                 const float *radius, const float *height, const int *obs_offsets,
                                 const float *obs_centers, const float *obs_radii) {
  if (!b) return TRAJ_EINVAL;
  const traj_ma_config &c = b->cfg;
  const int D = c.dim;
  if (!duration || !start || !goal || !radius || !obs_offsets || (D == 3 && !height))
    return ma_fail(b, TRAJ_EINVAL, "NULL problem array");
  if (n_scenes < 1 || n_scenes > c.max_scenes || n_agents < 1 || n_agents > c.max_agents)
    return ma_fail(b, TRAJ_ESHAPE, "n_scenes / n_agents exceed the capacities");
  if (obs_offsets[0] != 0) return ma_fail(b, TRAJ_EINVAL, "obs_offsets[0] must be 0");
  for (int s = 0; s < n_scenes; ++s)
    if (obs_offsets[s + 1] < obs_offsets[s]) return ma_fail(b, TRAJ_EINVAL, "obs_offsets must not decrease");
  const int n_obs = obs_offsets[n_scenes];
  if (n_obs > c.max_obstacles) return ma_fail(b, TRAJ_ESHAPE, "more obstacles than max_obstacles");
  if (n_obs > 0 && (!obs_centers || !obs_radii)) return ma_fail(b, TRAJ_EINVAL, "NULL obstacle array");
  std::vector<float> st((size_t)n_scenes * n_agents * D), gl(st.size());
  std::vector<float2> shp(n_scenes);
  std::vector<float4> obs(std::max(n_obs, 1));
  for (int s = 0; s < n_scenes; ++s) {
    if (!(duration[s] > 0) || !std::isfinite(duration[s]))
      return ma_fail(b, TRAJ_EINVAL, "durations must be positive and finite");
    const float h = D == 3 ? height[s] : 1.f;
    if (!(radius[s] > 0) || !(h > 0) || !std::isfinite(radius[s]) || !std::isfinite(h))
      return ma_fail(b, TRAJ_EINVAL, "agent radius and height must be positive and finite");
    shp[s] = make_float2(radius[s], h);
  }
  for (size_t e = 0; e < st.size(); ++e) {
    if (!std::isfinite(start[e]) || !std::isfinite(goal[e]))
      return ma_fail(b, TRAJ_ENAN, "non-finite start or goal");
    st[e] = (float)start[e];
    gl[e] = (float)goal[e];
  }
  for (int o = 0; o < n_obs; ++o) {
    float cc[3] = {0.f, 0.f, 0.f};
    for (int a = 0; a < D; ++a) cc[a] = obs_centers[(size_t)o * D + a];
    if (!std::isfinite(cc[0]) || !std::isfinite(cc[1]) || !std::isfinite(cc[2]) ||
        !(obs_radii[o] >= 0) || !std::isfinite(obs_radii[o]))
      return ma_fail(b, TRAJ_EINVAL, "obstacle centres must be finite and radii >= 0");
    obs[o] = make_float4(cc[0], cc[1], cc[2], obs_radii[o]);
  }
  const int N = n_agents, npairs = N * (N - 1) / 2;
  const size_t smem_full = sizeof(float) * ma_smem(D, N, c.n_steps, npairs, true).total;
  const size_t smem_part = sizeof(float) * ma_smem(D, N, c.n_steps, npairs, false).total;
  const int optin = max_optin_smem();
  if (optin <= 0) return ma_fail(b, TRAJ_ECUDA, "no CUDA device");
  if ((int)smem_part > optin)
    return ma_fail(b, TRAJ_ESHAPE, "agents x grid points do not fit one CTA's shared memory");
  b->lam_in_smem = (int)smem_full <= optin ? 1 : 0;
  b->smem = b->lam_in_smem ? smem_full : smem_part;
  cudaStream_t s = b->stream;
  MA_CK(b, cudaMemcpyAsync(b->d_T, duration, sizeof(double) * n_scenes, cudaMemcpyHostToDevice, s));
  MA_CK(b, cudaMemcpyAsync(b->d_start, st.data(), sizeof(float) * st.size(), cudaMemcpyHostToDevice, s));
  MA_CK(b, cudaMemcpyAsync(b->d_goal, gl.data(), sizeof(float) * gl.size(), cudaMemcpyHostToDevice, s));
  MA_CK(b, cudaMemcpyAsync(b->d_shape, shp.data(), sizeof(float2) * n_scenes, cudaMemcpyHostToDevice, s));
  MA_CK(b, cudaMemcpyAsync(b->d_obs_off, obs_offsets, sizeof(int) * (n_scenes + 1), cudaMemcpyHostToDevice, s));
  MA_CK(b, cudaMemcpyAsync(b->d_obs, obs.data(), sizeof(float4) * obs.size(), cudaMemcpyHostToDevice, s));
  MA_CK(b, cudaMemsetAsync(b->d_err, 0, sizeof(int), s));
  const size_t smem_setup = sizeof(double) * 3 * c.n_steps * NC;
  MA_CK(b, cudaFuncSetAttribute(k_ma_setup, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_setup));
  k_ma_setup<<<dim3(n_scenes, b->levels), 128, smem_setup, s>>>(N, c.n_steps, b->d_T, b->d_obs_off,
                                                                b->d_rho, b->d_consts, b->d_free, b->d_err);
  MA_CK(b, cudaGetLastError());
  int herr = 0;
  MA_CK(b, cudaMemcpyAsync(&herr, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  MA_CK(b, cudaStreamSynchronize(s));
  if (herr & 1) return ma_fail(b, TRAJ_EINVAL, "a scene's KKT matrix is singular");
  b->n_scenes = n_scenes;
  b->N = N;
  b->n_obs = n_obs;
  b->have_problems = true;
  b->have_result = false;
  return TRAJ_OK;
}

traj_status traj_ma_solve(traj_ma_batch *b, int max_iters, float tol, traj_ma_stats *stats) {
  tb::NvtxRange nvtx_range("traj_ma_solve");
  if (!b) return TRAJ_EINVAL;
  if (!b->have_problems) return ma_fail(b, TRAJ_ESTATE, "traj_ma_set_problems must come first");
  if (max_iters < 0) return ma_fail(b, TRAJ_EINVAL, "max_iters must be >= 0");
  const traj_ma_config &c = b->cfg;
  MaArgs A{};
  A.n_scenes = b->n_scenes;
  A.N = b->N;
  A.n_p = c.n_steps;
  A.npairs = b->N * (b->N - 1) / 2;
  A.levels = b->levels;
  A.rho_every = c.rho_every;
  A.max_iters = max_iters;
  A.lam_in_smem = b->lam_in_smem;
  A.tol = tol;
  A.rho_ladder = b->d_rho;
  A.P = b->d_P;
  A.consts = b->d_consts;
  A.consts_free = b->d_free;
  A.start = b->d_start;
  A.goal = b->d_goal;
  A.shape = b->d_shape;
  A.obs_off = b->d_obs_off;
  A.obs = b->d_obs;
  A.lam_ag = b->d_lam;
  A.lam_ob = b->d_lamo;
  A.xi_out = b->d_xi;
  A.res_out = b->d_res;
  A.iters_out = b->d_iters;
  cudaStream_t s = b->stream;
  auto kern = c.dim == 3 ? k_ma_solve<3> : k_ma_solve<2>;
  MA_CK(b, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem));
  MA_CK(b, cudaEventRecord(b->ev0, s));
  kern<<<b->n_scenes, MA_THREADS, b->smem, s>>>(A);
  MA_CK(b, cudaGetLastError());
  MA_CK(b, cudaEventRecord(b->ev1, s));
  b->have_result = true;
  if (stats) {
    MA_CK(b, cudaEventSynchronize(b->ev1));
    float ms = 0.f;
    MA_CK(b, cudaEventElapsedTime(&ms, b->ev0, b->ev1));
    std::vector<float> res(b->n_scenes);
    std::vector<int> it(b->n_scenes);
    MA_CK(b, cudaMemcpy(res.data(), b->d_res, sizeof(float) * b->n_scenes, cudaMemcpyDeviceToHost));
    MA_CK(b, cudaMemcpy(it.data(), b->d_iters, sizeof(int) * b->n_scenes, cudaMemcpyDeviceToHost));
    int conv = 0, imax = 0;
    for (int k = 0; k < b->n_scenes; ++k) {
      conv += res[k] <= tol ? 1 : 0;
      imax = std::max(imax, it[k]);
    }
    stats->gpu_ms = ms;
    stats->n_converged = conv;
    stats->max_iters_run = imax;
    stats->lambda_in_shared = b->lam_in_smem;
  }
  return TRAJ_OK;
}

traj_status traj_ma_get_trajectories(traj_ma_batch *b, float *coeffs, float *residual, int *iters) {
  if (!b) return TRAJ_EINVAL;
  if (!b->have_result) return ma_fail(b, TRAJ_ESTATE, "traj_ma_solve must come first");
  const size_t n = (size_t)b->n_scenes * b->N * b->cfg.dim * NC;
  cudaStream_t s = b->stream;
  if (coeffs) MA_CK(b, cudaMemcpyAsync(coeffs, b->d_xi, sizeof(float) * n, cudaMemcpyDefault, s));
  if (residual) MA_CK(b, cudaMemcpyAsync(residual, b->d_res, sizeof(float) * b->n_scenes, cudaMemcpyDefault, s));
  if (iters) MA_CK(b, cudaMemcpyAsync(iters, b->d_iters, sizeof(int) * b->n_scenes, cudaMemcpyDefault, s));
  MA_CK(b, cudaStreamSynchronize(s));
  return TRAJ_OK;
}

} // extern "C"

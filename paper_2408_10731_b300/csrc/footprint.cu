// footprint.cu -- the batch optimizer for a robot with a multi-circle footprint
// and a heading (Paper II, Algorithm 2 with the heading variables), 2D.
//
// Per trajectory: x, y and the heading psi as degree-10 Bernstein polynomials,
// plus slack copies c, s of cos psi, sin psi with their own coefficients. Each
// half h in {x, y} has 22 coefficients (xi_h, xi_copy) and the rows of F
//   [Pdot 0] speed, [Pddot 0] acceleration, [P  r_m P] per circle m and
//   obstacle j, [0 P] the copy of cos / sin psi,
// so F^T F = [[Pd'Pd + Pdd'Pdd + n_o n_c S, n_o (sum r) S], [n_o (sum r) S,
// (n_o sum r^2 + 1) S]] (S = P^T P) is formed without F. One iteration:
//   xi-step   xi^k = hq + G xi^{k-1} + K11 (lambda - rho u), u = F^T (F xi - g),
//             per half, constants from the FP64 KKT inverse (eq. over_2),
//   psi-step  the convex surrogate (eq. compute_convex_surrogate) on
//             psi^ = psi + wrap(atan2(s, c) - psi), which with the multiplier
//             update is the increment xi_psi += rho_psi K_psi P^T (psi^ - psi),
//   alpha/d   closed forms: a footprint circle inside an (inflated) ellipse is
//             pushed out along its ray, speed and acceleration clipped,
//   lambda    lambda -= rho F^T (F xi - g) (lambda_psi is folded into the increment).
// One warp per trajectory; a lane owns grid points lane, lane + 32, ...
#include "trajbatch.h"
#include "internal.cuh"
#include "nvtx_range.h"
#include "basis.cuh"
#include "linalg.cuh"

#include <algorithm>
#include <climits>
#include <cmath>
#include <string>
#include <vector>

namespace tb {
namespace {

constexpr int FP_H = 22;         // coefficients per half
constexpr int FP_NK = FP_H + 4;  // half KKT size (4 boundary rows on xi_h)
constexpr int FP_PK = NC + 2;    // heading KKT size (heading at both ends)
constexpr int FP_MAX_CIRCLES = 8;
constexpr int FP_WARPS = 4;
// constants per problem (floats, each an FP32 hi/lo pair of an FP64 value)
constexpr int FC_K11 = 0, FC_G = 968, FC_HQ = 1936, FC_PK11 = 2024, FC_PG = 2266, FC_PHQ = 2508;
constexpr int FC_FLOATS = 2530;

struct FpProblemDev {
  int n_p, n_o, obs_off, tbl_off, const_off, pad0, pad1, pad2;
  float T, pad3, pad4, pad5;
};

struct FpArgs {
  int n_traj, n_c, max_iters;
  int mask_words;        // 32-obstacle mask words per warp: ceil(max obstacles per problem / 32)
  float tol, rho, rho_psi, vmax, amax, r_circle;
  float offs[FP_MAX_CIRCLES];
  const int *traj_problem;
  const FpProblemDev *problems;
  const float *tables;   // per problem [3][n_p][ROW]: P, Pdot, Pddot (time-scaled)
  const float *consts;   // per problem FC_FLOATS
  const float4 *obs;     // per obstacle (cx, cy, vx, vy)
  const float2 *obs_ax;  // per obstacle 1 / (a + r_circle), 1 / (b + r_circle)
  const float *xi0;      // [n_traj][3][11]: x, y, psi
  float *xi_out;         // [n_traj][5][11]: x, c, y, s, psi
  float *res_out;        // [n_traj][4]: obstacle, speed, acceleration, heading copy
  int *iters_out;
};

// ---- set-up (FP64, one CTA per problem) ------------------------------------------
__global__ void k_fp_setup(int n_c, float rho_f, float rho_psi_f, const float *offs,
                           const double *start, const double *goal, const double *psi_ends,
                           FpProblemDev *problems, float *tables, float *consts, int *err) {
  extern __shared__ double smd[];
  __shared__ double S[NC * NC], D[NC * NC], A2[NC * NC], W[FP_NK * 2 * FP_NK];
  __shared__ double K11[FP_H * FP_H], K12[FP_H * 4], Ab[4 * NC], qv[2 * NC];
  __shared__ int piv, bad;
  const int p = blockIdx.x;
  const FpProblemDev pr = problems[p];
  const int n_p = pr.n_p, n_o = pr.n_o;
  const double T = pr.T, iT = 1.0 / T, iT2 = iT * iT, rho = rho_f, rp = rho_psi_f;
  double sr = 0.0, sr2 = 0.0;
  for (int m = 0; m < n_c; ++m) { sr += offs[m]; sr2 += (double)offs[m] * offs[m]; }
  double *P = smd, *Pd = smd + n_p * NC, *Pdd = smd + 2 * n_p * NC;
  if (threadIdx.x == 0) bad = 0;
  float *tab = tables + pr.tbl_off;
  for (int t = threadIdx.x; t < n_p; t += blockDim.x) {
    double a[NC], b[NC], c[NC];
    basis_row(n_p, t, a, b, c);
    for (int i = 0; i < ROW; ++i) {
      const double va = i < NC ? a[i] : 0.0, vb = i < NC ? b[i] * iT : 0.0,
                   vc = i < NC ? c[i] * iT2 : 0.0;
      if (i < NC) { P[t * NC + i] = va; Pd[t * NC + i] = vb; Pdd[t * NC + i] = vc; }
      tab[(0 * n_p + t) * ROW + i] = (float)va;
      tab[(1 * n_p + t) * ROW + i] = (float)vb;
      tab[(2 * n_p + t) * ROW + i] = (float)vc;
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < NC * NC + 2 * NC; e += blockDim.x) {
    if (e < NC * NC) {
      const int a = e / NC, b = e % NC;
      double ss = 0.0, dd = 0.0, aa = 0.0;
      for (int t = 0; t < n_p; ++t) {
        ss += P[t * NC + a] * P[t * NC + b];
        dd += Pd[t * NC + a] * Pd[t * NC + b];
        aa += Pdd[t * NC + a] * Pdd[t * NC + b];
      }
      S[e] = ss; D[e] = dd; A2[e] = aa;
    } else { // q = -P^T x_des, x_des the constant-velocity line (eq. Q_matrix)
      const int k = e - NC * NC, ax = k / NC, i = k % NC;
      const double s0 = start[p * 2 + ax], g0 = goal[p * 2 + ax];
      double s = 0.0;
      for (int t = 0; t < n_p; ++t) s += P[t * NC + i] * (s0 + (g0 - s0) * (double)t / (double)(n_p - 1));
      qv[k] = -s;
    }
  }
  for (int e = threadIdx.x; e < 4 * NC; e += blockDim.x) {
    const int r = e / NC, i = e % NC;
    Ab[e] = r == 0 ? P[i] : r == 1 ? Pd[i] : r == 2 ? Pdd[i] : P[(n_p - 1) * NC + i];
  }
  __syncthreads();
  // half KKT: [[Q + rho F^T F, A^T], [A, 0]], Q = blockdiag(Pdd'Pdd + P'P, 0)
  auto FtF = [&](int r, int c) -> double { // F^T F of one half (22 x 22)
    const int br = r / NC, bc = c / NC, i = r % NC, j = c % NC;
    if (br == 0 && bc == 0) return D[i * NC + j] + A2[i * NC + j] + (double)n_o * n_c * S[i * NC + j];
    if (br != bc) return (double)n_o * sr * S[i * NC + j];
    return ((double)n_o * sr2 + 1.0) * S[i * NC + j];
  };
  for (int e = threadIdx.x; e < FP_NK * 2 * FP_NK; e += blockDim.x) {
    const int r = e / (2 * FP_NK), c = e % (2 * FP_NK);
    double v = 0.0;
    if (c >= FP_NK) v = (c - FP_NK == r) ? 1.0 : 0.0;
    else if (r < FP_H && c < FP_H) {
      v = rho * FtF(r, c);
      if (r < NC && c < NC) v += A2[r * NC + c] + S[r * NC + c];
    } else if (r < FP_H) v = r < NC ? Ab[(c - FP_H) * NC + r] : 0.0;
    else if (c < FP_H) v = c < NC ? Ab[(r - FP_H) * NC + c] : 0.0;
    W[e] = v;
  }
  __syncthreads();
  gj_invert(W, FP_NK, &piv, &bad);
  for (int e = threadIdx.x; e < FP_H * FP_H + FP_H * 4; e += blockDim.x) {
    if (e < FP_H * FP_H) K11[e] = W[(e / FP_H) * 2 * FP_NK + FP_NK + e % FP_H];
    else {
      const int k = e - FP_H * FP_H;
      K12[k] = W[(k / 4) * 2 * FP_NK + FP_NK + FP_H + k % 4];
    }
  }
  __syncthreads();
  float *C = consts + pr.const_off;
  for (int e = threadIdx.x; e < FP_H * FP_H; e += blockDim.x) {
    const int r = e / FP_H, c = e % FP_H;
    double g = 0.0;
    for (int k = 0; k < FP_H; ++k) g += K11[r * FP_H + k] * FtF(k, c);
    split2(&C[FC_K11 + e], &C[FC_K11 + 484 + e], K11[e]);
    split2(&C[FC_G + e], &C[FC_G + 484 + e], rho * g);
  }
  for (int e = threadIdx.x; e < 2 * FP_H; e += blockDim.x) { // hq = K11 (-q) + K12 b per half
    const int h = e / FP_H, i = e % FP_H;
    const double b[4] = {start[p * 2 + h], 0.0, 0.0, goal[p * 2 + h]};
    double v = 0.0;
    for (int k = 0; k < NC; ++k) v += K11[i * FP_H + k] * (-qv[h * NC + k]);
    for (int k = 0; k < 4; ++k) v += K12[i * 4 + k] * b[k];
    split2(&C[FC_HQ + e], &C[FC_HQ + 44 + e], v);
  }
  __syncthreads();
  // heading KKT: [[Pdd'Pdd + rho_psi S, A_psi^T], [A_psi, 0]], A_psi = (P_0; P_last)
  for (int e = threadIdx.x; e < FP_PK * 2 * FP_PK; e += blockDim.x) {
    const int r = e / (2 * FP_PK), c = e % (2 * FP_PK);
    double v = 0.0;
    if (c >= FP_PK) v = (c - FP_PK == r) ? 1.0 : 0.0;
    else if (r < NC && c < NC) v = A2[r * NC + c] + rp * S[r * NC + c];
    else if (r < NC) v = c == NC ? P[r] : P[(n_p - 1) * NC + r];
    else if (c < NC) v = r == NC ? P[c] : P[(n_p - 1) * NC + c];
    W[e] = v;
  }
  __syncthreads();
  gj_invert(W, FP_PK, &piv, &bad);
  for (int e = threadIdx.x; e < NC * NC; e += blockDim.x) {
    const int r = e / NC, c = e % NC;
    double g = 0.0;
    for (int k = 0; k < NC; ++k) g += W[r * 2 * FP_PK + FP_PK + k] * S[k * NC + c];
    split2(&C[FC_PK11 + e], &C[FC_PK11 + 121 + e], W[r * 2 * FP_PK + FP_PK + c]);
    split2(&C[FC_PG + e], &C[FC_PG + 121 + e], rp * g);
  }
  for (int e = threadIdx.x; e < NC; e += blockDim.x) {
    const double v = W[e * 2 * FP_PK + FP_PK + NC] * psi_ends[p * 2] +
                     W[e * 2 * FP_PK + FP_PK + NC + 1] * psi_ends[p * 2 + 1];
    split2(&C[FC_PHQ + e], &C[FC_PHQ + 11 + e], v);
  }
  if (threadIdx.x == 0 && bad) atomicOr(err, 1);
}

// ---- solve -------------------------------------------------------------------------
__device__ __forceinline__ float wrap_pi(float x) {
  const float TWO_PI = 6.28318530717958647692f, PI = 3.14159265358979323846f;
  return x - TWO_PI * ceilf((x - PI) / TWO_PI);
}

// speed / acceleration step (reading R5): the residual w - clip(w, bound)
__device__ __forceinline__ void bound_res(float wx, float wy, float bound, float &rx, float &ry) {
  const float n = sqrtf(wx * wx + wy * wy);
  const float f = n > bound ? 1.f - bound / n : 0.f;
  rx = wx * f;
  ry = wy * f;
}

// per-warp shared state (floats)
// (the iterate as exact float pairs: X / XL, XP / XPL)
constexpr int WS_X = 0, WS_XL = 44, WS_LAM = 88, WS_V = 132, WS_XP = 176, WS_XPL = 187,
              WS_UP = 198, WS_U = 209, WS_FLOATS = 256;

// dot of 11 coefficients (shared, broadcast) with a table row
__device__ __forceinline__ float dot11(const float *row, const float *c) {
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < NC; ++k) s = fmaf(row[k], c[k], s);
  return s;
}

// the same for coefficients held as exact pairs (hi at c, lo at c + off)
__device__ __forceinline__ float dot11p(const float *row, const float *c, int off) {
  float s = 0.f, l = 0.f;
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    s = fmaf(row[k], c[k], s);
    l = fmaf(row[k], c[off + k], l);
  }
  return s + l;
}

// (s, e) with s + e = a + b exactly (Knuth's TwoSum)
__device__ __forceinline__ void fp_two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ float warp_max(float v) {
  for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Order keys for warp min/max on the integer unit: k = bits ^ ((bits >> 31) & 0x7fffffff)
// orders as a signed integer as the floats do; the map is its own inverse.
__device__ __forceinline__ int fp_key(float f) {
  const int b = __float_as_int(f);
  return b ^ ((b >> 31) & 0x7fffffff);
}
__device__ __forceinline__ float fp_unkey(int k) { return __int_as_float(k ^ ((k >> 31) & 0x7fffffff)); }
__device__ __forceinline__ float fp_warp_min(float v, bool on) {
  return fp_unkey(__reduce_min_sync(0xffffffffu, on ? fp_key(v) : INT_MAX));
}
__device__ __forceinline__ float fp_warp_max(float v, bool on) {
  return fp_unkey(__reduce_max_sync(0xffffffffu, on ? fp_key(v) : INT_MIN));
}

template <int PPL>
__global__ void __launch_bounds__(FP_WARPS * 32) k_fp_solve(FpArgs A, int max_np) {
  extern __shared__ float smf[];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int traj = blockIdx.x * FP_WARPS + w;
  if (traj >= A.n_traj) return; // whole warp; no block-wide barrier follows
  float *ws = smf + w * (WS_FLOATS + A.mask_words);
  unsigned *keep = reinterpret_cast<unsigned *>(ws + WS_FLOATS); // this slot's kept obstacles
  const FpProblemDev pr = A.problems[A.traj_problem[traj]];
  const int n_p = pr.n_p, n_o = pr.n_o, n_c = A.n_c;
  const float *tP = A.tables + pr.tbl_off, *tD = tP + n_p * ROW, *tA = tD + n_p * ROW;
  const float *C = A.consts + pr.const_off;
  const float4 *ob = A.obs + pr.obs_off;
  const float2 *oax = A.obs_ax + pr.obs_off;
  const float rho = A.rho, rp = A.rho_psi;
  float *X = ws + WS_X, *LAM = ws + WS_LAM, *V = ws + WS_V, *XP = ws + WS_XP;
  float *UP = ws + WS_UP, *U = ws + WS_U;
  constexpr int XLO = WS_XL - WS_X, PLO = WS_XPL - WS_XP; // offsets of the lo halves

  // initial coefficients: x, y, psi given; the copy coefficients start as cos / sin
  // of the heading coefficients. The targets use cos / sin psi on the grid (reading
  // H5); the copy coefficients only set where F xi starts, and the first xi-step,
  // hq + G xi0 - rho K11 F^T (F xi0 - g0) = hq + rho K11 F^T g0, does not depend on
  // them: starting them near the copies keeps F xi0 - g0 small in FP32.
  for (int e = lane; e < 44; e += 32) {
    const int h = e / FP_H, i = e % FP_H;
    const float ps = A.xi0[((size_t)traj * 3 + 2) * NC + (i % NC)];
    X[e] = i < NC ? A.xi0[((size_t)traj * 3 + h) * NC + i] : (h == 0 ? cosf(ps) : sinf(ps));
    X[XLO + e] = 0.f;
    LAM[e] = 0.f;
  }
  if (lane < NC) { XP[lane] = A.xi0[((size_t)traj * 3 + 2) * NC + lane]; XP[PLO + lane] = 0.f; }
  __syncwarp();

  // Projections at the lane's points with this lane's residual maxima (obstacle,
  // speed, acceleration, copy). init: the footprint targets use cos / sin psi on the
  // grid while F xi uses the copy coefficients. The contraction u = F^T (F xi - g) is
  // accumulated per lane over its points (44 partial sums) and reduced across the
  // warp into U.
  // Culled and exact: per slot of 32 grid points the warp bounds every circle
  // centre of its valid lanes by a box [fx_lo, fx_hi] x [fy_lo, fy_hi] and the
  // times by [tA, tB]; lane j then bounds obstacle j's normalised offsets
  // ux = (fx - fma(vx, t, cx)) * iax (and uy) over the box with the same rounded
  // operations at its corners. Each is monotone (round-to-nearest, iax > 0), so an
  // obstacle with ux >= 1 or ux <= -1 (or uy) over the whole box has fma(ux, ux, uy^2)
  // >= 1 at every circle and point of the slot and cannot hold one; the circle loop
  // visits only the obstacles kept, in increasing order, and the sums are bitwise
  // those of visiting all of them.
  const int n_rounds = (n_o + 31) >> 5;
  auto project = [&](bool init, float (&rmax)[4]) {
    rmax[0] = rmax[1] = rmax[2] = rmax[3] = 0.f;
    float acc[44];
#pragma unroll
    for (int e = 0; e < 44; ++e) acc[e] = 0.f;
#pragma unroll
    for (int q = 0; q < PPL; ++q) {
      if (32 * q >= n_p) break; // warp-uniform: the slot holds at least one grid point
      const int t = lane + 32 * q;
      const bool valid = t < n_p;
      const int tv = valid ? t : n_p - 1; // idle lanes read the last row; results unused
      const float *rp_ = tP + tv * ROW, *rd = tD + tv * ROW, *ra = tA + tv * ROW;
      const float x = dot11p(rp_, X, XLO), y = dot11p(rp_, X + FP_H, XLO);
      const float vx = dot11(rd, X), vy = dot11(rd, X + FP_H); // bound tests: hi part
      const float axx = dot11(ra, X), ayy = dot11(ra, X + FP_H);
      const float psi = dot11p(rp_, XP, PLO);
      float sp, cp;
      sincosf(psi, &sp, &cp);
      // F xi uses the copy coefficients (cF, sF); the footprint targets use the copies,
      // or cos / sin psi in the initial pass (reading H5)
      const float cF = dot11p(rp_, X + NC, XLO), sF = dot11p(rp_, X + FP_H + NC, XLO);
      const float c = init ? cp : cF, s = init ? sp : sF;
      const float tt = (float)t * pr.T / (float)(n_p - 1);
      { // the slot's kept obstacles
        float flo = __int_as_float(0x7f800000), fhi = -flo, glo = flo, ghi = -flo;
        for (int m = 0; m < n_c; ++m) {
          const float r = A.offs[m];
          const float fx = fmaf(r, c, x), fy = fmaf(r, s, y);
          flo = fminf(flo, fx); fhi = fmaxf(fhi, fx);
          glo = fminf(glo, fy); ghi = fmaxf(ghi, fy);
        }
        flo = fp_warp_min(flo, valid); fhi = fp_warp_max(fhi, valid);
        glo = fp_warp_min(glo, valid); ghi = fp_warp_max(ghi, valid);
        const float ta = __int_as_float(__reduce_min_sync(0xffffffffu, valid ? __float_as_int(tt) : INT_MAX));
        const float tb = __int_as_float(__reduce_max_sync(0xffffffffu, valid ? __float_as_int(tt) : INT_MIN));
        for (int k = 0; k < n_rounds; ++k) {
          const int j = 32 * k + lane;
          bool kept = false;
          if (j < n_o) {
            const float4 o = ob[j];
            const float2 ia = oax[j];
            const float cA = fmaf(o.z, ta, o.x), cB = fmaf(o.z, tb, o.x);
            const float dA = fmaf(o.w, ta, o.y), dB = fmaf(o.w, tb, o.y);
            const float uxl = (flo - fmaxf(cA, cB)) * ia.x, uxh = (fhi - fminf(cA, cB)) * ia.x;
            const float uyl = (glo - fmaxf(dA, dB)) * ia.y, uyh = (ghi - fminf(dA, dB)) * ia.y;
            kept = !(uxl >= 1.f || uxh <= -1.f || uyl >= 1.f || uyh <= -1.f);
          }
          const unsigned msk = __ballot_sync(0xffffffffu, kept);
          if (lane == 0) keep[k] = msk;
        }
        __syncwarp();
      }
      if (valid) {
      float rvx, rvy, rax, ray;
      bound_res(vx, vy, A.vmax, rvx, rvy);
      bound_res(axx, ayy, A.amax, rax, ray);
      rmax[1] = fmaxf(rmax[1], sqrtf(rvx * rvx + rvy * rvy));
      rmax[2] = fmaxf(rmax[2], sqrtf(rax * rax + ray * ray));
      float Rox = 0.f, Roy = 0.f, Rcx = 0.f, Rcy = 0.f;
      for (int m = 0; m < n_c; ++m) {
        const float r = A.offs[m];
        const float fx = fmaf(r, c, x), fy = fmaf(r, s, y);
        float sx = 0.f, sy = 0.f; // sum over obstacles of the circle's residuals
        for (int k = 0; k < n_rounds; ++k) {
          unsigned bits = keep[k];
          while (bits) {
            const int j = 32 * k + __ffs(bits) - 1;
            bits &= bits - 1u;
            const float4 o = ob[j];
            const float2 ia = oax[j]; // reciprocal inflated semi-axes
            const float dx = fx - fmaf(o.z, tt, o.x), dy = fy - fmaf(o.w, tt, o.y);
            const float ux = dx * ia.x, uy = dy * ia.y;
            const float u2 = fmaf(ux, ux, uy * uy);
            if (u2 < 1.f) { // inside: pushed out along the ray (d = 1)
              float ex, ey;
              if (u2 > 0.f) {
                const float f = 1.f - 1.f / sqrtf(u2);
                ex = dx * f;
                ey = dy * f;
              } else { ex = -1.f / ia.x; ey = 0.f; } // atan2(0, 0) = 0
              rmax[0] = fmaxf(rmax[0], sqrtf(ex * ex + ey * ey));
              sx += ex;
              sy += ey;
            }
          }
        }
        // F xi - g for the collision rows: (x + r cF) - target = e - r (c - cF)
        const float ox = sx - (float)n_o * r * (c - cF), oy = sy - (float)n_o * r * (s - sF);
        Rox += ox; Roy += oy;
        Rcx = fmaf(r, ox, Rcx); Rcy = fmaf(r, oy, Rcy);
      }
      // copies: F xi - g = cF - cos psi
      const float rcx = cF - cp, rcy = sF - sp;
      if (!init) rmax[3] = fmaxf(rmax[3], sqrtf((c - cp) * (c - cp) + (s - sp) * (s - sp)));
      const float qx = Rcx + rcx, qy = Rcy + rcy;
#pragma unroll
      for (int kk = 0; kk < NC; ++kk) {
        const float p0 = rp_[kk], d0 = rd[kk], a0 = ra[kk];
        acc[kk] = fmaf(p0, Rox, fmaf(a0, rax, fmaf(d0, rvx, acc[kk])));
        acc[NC + kk] = fmaf(p0, qx, acc[NC + kk]);
        acc[FP_H + kk] = fmaf(p0, Roy, fmaf(a0, ray, fmaf(d0, rvy, acc[FP_H + kk])));
        acc[FP_H + NC + kk] = fmaf(p0, qy, acc[FP_H + NC + kk]);
      }
      } // valid
      __syncwarp(); // the next slot rewrites the masks
    }
#pragma unroll
    for (int e = 0; e < 44; ++e) {
      float v = acc[e];
      for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == (e & 31)) U[e] = v;
    }
    __syncwarp();
  };

  float rmax[4];
  project(true, rmax);
  for (int e = lane; e < 44; e += 32) V[e] = -rho * U[e];
  __syncwarp();
  float res[4] = {rmax[0], rmax[1], rmax[2], rmax[3]};
  int k_done = 0;
  for (int k = 1; k <= A.max_iters; ++k) {
    // xi-step per half (eq. zeta_1_sepration_1 as an increment)
    float xn[2], xl[2];
#pragma unroll
    for (int pass = 0; pass < 2; ++pass) {
      const int e = lane + 32 * pass;
      xn[pass] = 0.f;
      xl[pass] = 0.f;
      if (e < 44) {
        const int h = e / FP_H, i = e % FP_H;
        const float *xh = X + h * FP_H, *vh = V + h * FP_H;
        float hi = C[FC_HQ + e], lo = C[FC_HQ + 44 + e];
        for (int j = 0; j < FP_H; ++j) {
          df_fma(hi, lo, C[FC_G + i * FP_H + j], C[FC_G + 484 + i * FP_H + j], xh[j]);
          lo = fmaf(C[FC_G + i * FP_H + j], xh[XLO + j], lo);
          df_fma(hi, lo, C[FC_K11 + i * FP_H + j], C[FC_K11 + 484 + i * FP_H + j], vh[j]);
        }
        fp_two_sum(hi, lo, xn[pass], xl[pass]);
      }
    }
    __syncwarp();
    X[lane] = xn[0];
    X[XLO + lane] = xl[0];
    if (lane + 32 < 44) { X[lane + 32] = xn[1]; X[XLO + lane + 32] = xl[1]; }
    __syncwarp();
    // psi-step: psi^ - psi from the new copies (reading H2), then the surrogate QP.
    // With lambda_psi^{k-1} = lambda_psi^{k-2} - rho_psi P^T (psi^{k-1} - psi^^{k-1})
    // the surrogate's solution is an increment: xi_psi^k = xi_psi^{k-1} +
    // rho_psi K_psi P^T (psi^^k - psi^{k-1}) for k >= 2; the first step is
    // hq_psi + G_psi xi_psi^0 + rho_psi K_psi P^T (psi^^1 - psi^0) (lambda_psi^0 = 0).
    {
      float up[NC];
#pragma unroll
      for (int kk = 0; kk < NC; ++kk) up[kk] = 0.f;
#pragma unroll
      for (int q = 0; q < PPL; ++q) {
        const int t = lane + 32 * q;
        if (t >= n_p) break;
        const float *rp_ = tP + t * ROW;
        const float c = dot11p(rp_, X + NC, XLO), s = dot11p(rp_, X + FP_H + NC, XLO);
        const float psi = dot11p(rp_, XP, PLO);
        const float dpsi = wrap_pi(atan2f(s, c) - psi);
#pragma unroll
        for (int kk = 0; kk < NC; ++kk) up[kk] = fmaf(rp_[kk], dpsi, up[kk]);
      }
#pragma unroll
      for (int kk = 0; kk < NC; ++kk) {
        float v = up[kk];
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == kk) UP[kk] = rp * v;
      }
      __syncwarp();
    }
    float xph = 0.f, xpl = 0.f;
    if (lane < NC) {
      float hi, lo;
      if (k == 1) {
        hi = C[FC_PHQ + lane];
        lo = C[FC_PHQ + 11 + lane];
        for (int j = 0; j < NC; ++j) {
          df_fma(hi, lo, C[FC_PG + lane * NC + j], C[FC_PG + 121 + lane * NC + j], XP[j]);
          lo = fmaf(C[FC_PG + lane * NC + j], XP[PLO + j], lo);
        }
      } else {
        hi = XP[lane];
        lo = XP[PLO + lane];
      }
      for (int j = 0; j < NC; ++j)
        df_fma(hi, lo, C[FC_PK11 + lane * NC + j], C[FC_PK11 + 121 + lane * NC + j], UP[j]);
      fp_two_sum(hi, lo, xph, xpl);
    }
    __syncwarp();
    if (lane < NC) { XP[lane] = xph; XP[PLO + lane] = xpl; }
    __syncwarp();
    // alpha / d steps, residual maxima and u at the new iterate
    project(false, rmax);
    // multipliers (eq. update_lambda2_1) and v = lambda - rho u
    for (int e = lane; e < 44; e += 32) {
      const float l = LAM[e] - rho * U[e];
      LAM[e] = l;
      V[e] = l - rho * U[e];
    }
    __syncwarp();
#pragma unroll
    for (int r = 0; r < 4; ++r) res[r] = warp_max(rmax[r] != rmax[r] ? __int_as_float(0x7f800000) : rmax[r]);
    k_done = k;
    if (A.tol >= 0.f && res[0] <= A.tol && res[1] <= A.tol && res[2] <= A.tol && res[3] <= A.tol) break;
  }
  // outputs: (x, c, y, s, psi)
  for (int e = lane; e < 5 * NC; e += 32)
    A.xi_out[(size_t)traj * 5 * NC + e] = e < 44 ? X[e] + X[XLO + e] : XP[e - 44] + XP[PLO + e - 44];
  if (lane < 4) A.res_out[(size_t)traj * 4 + lane] = res[lane];
  if (lane == 0) A.iters_out[traj] = k_done;
}

} // namespace
} // namespace tb

// ---- C ABI -------------------------------------------------------------------------
using namespace tb;

struct traj_fp_batch {
  traj_fp_config cfg{};
  cudaStream_t stream = nullptr;
  std::string err;
  int n_problems = 0, n_traj = 0, max_np = 0, max_no = 0;
  bool have_problems = false, have_initial = false, have_result = false;
  FpProblemDev *d_problems = nullptr;
  float *d_tables = nullptr, *d_consts = nullptr, *d_offs = nullptr;
  double *d_start = nullptr, *d_goal = nullptr, *d_psi = nullptr;
  float4 *d_obs = nullptr;
  float2 *d_ax = nullptr;
  int *d_traj_problem = nullptr, *d_iters = nullptr, *d_err = nullptr;
  float *d_xi0 = nullptr, *d_xi = nullptr, *d_res = nullptr;
  size_t tables_cap = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

namespace tb_fp {
thread_local std::string g_fp_error;

traj_status fp_fail(traj_fp_batch *b, traj_status s, const std::string &m) {
  if (b) b->err = m;
  else g_fp_error = m;
  return s;
}

#define FP_CK(b, expr)                                                                  \
  do {                                                                                  \
    cudaError_t e_ = (expr);                                                            \
    if (e_ != cudaSuccess) return fp_fail(b, TRAJ_ECUDA, std::string(#expr ": ") + cudaGetErrorString(e_)); \
  } while (0)

template <class T> cudaError_t fp_alloc(T **p, size_t n) {
  return cudaMalloc(reinterpret_cast<void **>(p), sizeof(T) * (n > 0 ? n : 1));
}

void fp_free_all(traj_fp_batch *b) {
  void *ptrs[] = {b->d_problems, b->d_tables, b->d_consts, b->d_offs, b->d_start, b->d_goal,
                  b->d_psi, b->d_obs, b->d_ax, b->d_traj_problem, b->d_iters, b->d_err,
                  b->d_xi0, b->d_xi, b->d_res};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  if (b->ev0) cudaEventDestroy(b->ev0);
  if (b->ev1) cudaEventDestroy(b->ev1);
}
} // namespace tb_fp
using namespace tb_fp;

extern "C" {

const char *traj_fp_last_error(traj_fp_batch *b) { return b ? b->err.c_str() : g_fp_error.c_str(); }

traj_status traj_fp_create(const traj_fp_config *cfg, void *cuda_stream, traj_fp_batch **out) {
  g_fp_error.clear();
  if (!cfg || !out) return fp_fail(nullptr, TRAJ_EINVAL, "NULL config or output pointer");
  const traj_fp_config &c = *cfg;
  if (c.max_problems < 1 || c.max_traj < 1 || c.max_obstacles < 0 || c.max_steps < 2 ||
      c.max_steps > MAX_STEPS || c.n_circles < 1 || c.n_circles > FP_MAX_CIRCLES)
    return fp_fail(nullptr, TRAJ_EINVAL, "capacities out of range (n_circles 1..8, max_steps 2..256)");
  if (!(c.vmax > 0) || !(c.amax > 0) || !(c.rho > 0) || !(c.rho_psi > 0) || !(c.r_circle >= 0) ||
      !std::isfinite(c.vmax) || !std::isfinite(c.amax) || !std::isfinite(c.rho) ||
      !std::isfinite(c.rho_psi) || !std::isfinite(c.r_circle))
    return fp_fail(nullptr, TRAJ_EINVAL, "vmax, amax, rho, rho_psi must be positive; r_circle >= 0");
  for (int m = 0; m < c.n_circles; ++m)
    if (!std::isfinite(c.circle_offsets[m])) return fp_fail(nullptr, TRAJ_EINVAL, "non-finite circle offset");
  traj_fp_batch *b = new traj_fp_batch();
  b->cfg = c;
  b->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  const size_t P = c.max_problems, B = c.max_traj, O = c.max_obstacles;
  cudaError_t e;
  if ((e = fp_alloc(&b->d_problems, P)) || (e = fp_alloc(&b->d_consts, P * FC_FLOATS)) ||
      (e = fp_alloc(&b->d_offs, FP_MAX_CIRCLES)) || (e = fp_alloc(&b->d_start, P * 2)) ||
      (e = fp_alloc(&b->d_goal, P * 2)) || (e = fp_alloc(&b->d_psi, P * 2)) ||
      (e = fp_alloc(&b->d_obs, O)) || (e = fp_alloc(&b->d_ax, O)) ||
      (e = fp_alloc(&b->d_traj_problem, B)) || (e = fp_alloc(&b->d_iters, B)) ||
      (e = fp_alloc(&b->d_err, 1)) || (e = fp_alloc(&b->d_xi0, B * 3 * NC)) ||
      (e = fp_alloc(&b->d_xi, B * 5 * NC)) || (e = fp_alloc(&b->d_res, B * 4)) ||
      (e = cudaEventCreate(&b->ev0)) || (e = cudaEventCreate(&b->ev1)) ||
      (e = cudaMemcpy(b->d_offs, c.circle_offsets, sizeof(float) * FP_MAX_CIRCLES, cudaMemcpyHostToDevice))) {
    g_fp_error = std::string("allocation: ") + cudaGetErrorString(e);
    fp_free_all(b);
    delete b;
    return e == cudaErrorMemoryAllocation ? TRAJ_ENOMEM : TRAJ_ECUDA;
  }
  *out = b;
  return TRAJ_OK;
}

traj_status traj_fp_destroy(traj_fp_batch *b) {
  if (!b) return TRAJ_EINVAL;
  cudaStreamSynchronize(b->stream);
  fp_free_all(b);
  delete b;
  return TRAJ_OK;
}

traj_status traj_fp_set_problems(traj_fp_batch *b, int n_problems, const int *n_steps,
                                 const double *duration, const double *start, const double *goal,
                                 const double *heading_start, const double *heading_goal,
                                 const int *obs_offsets, const float *centers,
                                 const float *semi_axes, const float *velocities) {
  if (!b) return TRAJ_EINVAL;
  const traj_fp_config &c = b->cfg;
  if (!n_steps || !duration || !start || !goal || !heading_start || !heading_goal || !obs_offsets)
    return fp_fail(b, TRAJ_EINVAL, "NULL problem array");
  if (n_problems < 1 || n_problems > c.max_problems) return fp_fail(b, TRAJ_ESHAPE, "n_problems out of range");
  if (obs_offsets[0] != 0) return fp_fail(b, TRAJ_EINVAL, "obs_offsets[0] must be 0");
  std::vector<FpProblemDev> recs(n_problems);
  std::vector<double> psi(2 * n_problems);
  size_t tbl = 0;
  int max_np = 0, max_no = 0;
  for (int p = 0; p < n_problems; ++p) {
    if (n_steps[p] < 2 || n_steps[p] > c.max_steps) return fp_fail(b, TRAJ_ESHAPE, "n_steps out of range");
    if (!(duration[p] > 0) || !std::isfinite(duration[p])) return fp_fail(b, TRAJ_EINVAL, "bad duration");
    if (obs_offsets[p + 1] < obs_offsets[p]) return fp_fail(b, TRAJ_EINVAL, "obs_offsets must not decrease");
    for (int a = 0; a < 2; ++a)
      if (!std::isfinite(start[p * 2 + a]) || !std::isfinite(goal[p * 2 + a]))
        return fp_fail(b, TRAJ_ENAN, "non-finite start or goal");
    if (!std::isfinite(heading_start[p]) || !std::isfinite(heading_goal[p]))
      return fp_fail(b, TRAJ_ENAN, "non-finite heading");
    FpProblemDev r{};
    r.n_p = n_steps[p];
    r.n_o = obs_offsets[p + 1] - obs_offsets[p];
    r.obs_off = obs_offsets[p];
    r.tbl_off = (int)tbl;
    r.const_off = p * FC_FLOATS;
    r.T = (float)duration[p];
    recs[p] = r;
    tbl += (size_t)3 * n_steps[p] * ROW;
    max_np = std::max(max_np, n_steps[p]);
    max_no = std::max(max_no, r.n_o);
    psi[2 * p] = heading_start[p];
    psi[2 * p + 1] = heading_goal[p];
  }
  const int n_obs = obs_offsets[n_problems];
  if (n_obs > c.max_obstacles) return fp_fail(b, TRAJ_ESHAPE, "more obstacles than max_obstacles");
  if (n_obs > 0 && (!centers || !semi_axes || !velocities)) return fp_fail(b, TRAJ_EINVAL, "NULL obstacle array");
  std::vector<float4> obs(std::max(n_obs, 1));
  std::vector<float2> ax(std::max(n_obs, 1));
  for (int j = 0; j < n_obs; ++j) {
    const float v[6] = {centers[2 * j], centers[2 * j + 1], velocities[2 * j], velocities[2 * j + 1],
                        semi_axes[2 * j], semi_axes[2 * j + 1]};
    for (float x : v)
      if (!std::isfinite(x)) return fp_fail(b, TRAJ_ENAN, "non-finite obstacle data");
    if (!(v[4] > 0) || !(v[5] > 0)) return fp_fail(b, TRAJ_EINVAL, "semi-axes must be positive");
    obs[j] = make_float4(v[0], v[1], v[2], v[3]);
    ax[j] = make_float2((float)(1.0 / ((double)v[4] + c.r_circle)), (float)(1.0 / ((double)v[5] + c.r_circle)));
  }
  if (tbl > b->tables_cap) {
    if (b->d_tables) cudaFree(b->d_tables);
    b->d_tables = nullptr;
    b->tables_cap = 0;
    FP_CK(b, fp_alloc(&b->d_tables, tbl));
    b->tables_cap = tbl;
  }
  cudaStream_t s = b->stream;
  FP_CK(b, cudaMemcpyAsync(b->d_problems, recs.data(), sizeof(FpProblemDev) * n_problems, cudaMemcpyHostToDevice, s));
  FP_CK(b, cudaMemcpyAsync(b->d_start, start, sizeof(double) * 2 * n_problems, cudaMemcpyHostToDevice, s));
  FP_CK(b, cudaMemcpyAsync(b->d_goal, goal, sizeof(double) * 2 * n_problems, cudaMemcpyHostToDevice, s));
  FP_CK(b, cudaMemcpyAsync(b->d_psi, psi.data(), sizeof(double) * 2 * n_problems, cudaMemcpyHostToDevice, s));
  FP_CK(b, cudaMemcpyAsync(b->d_obs, obs.data(), sizeof(float4) * obs.size(), cudaMemcpyHostToDevice, s));
  FP_CK(b, cudaMemcpyAsync(b->d_ax, ax.data(), sizeof(float2) * ax.size(), cudaMemcpyHostToDevice, s));
  FP_CK(b, cudaMemsetAsync(b->d_err, 0, sizeof(int), s));
  const size_t smem = sizeof(double) * 3 * max_np * NC;
  FP_CK(b, cudaFuncSetAttribute(k_fp_setup, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_fp_setup<<<n_problems, 128, smem, s>>>(c.n_circles, c.rho, c.rho_psi, b->d_offs, b->d_start,
                                           b->d_goal, b->d_psi, b->d_problems, b->d_tables,
                                           b->d_consts, b->d_err);
  FP_CK(b, cudaGetLastError());
  int herr = 0;
  FP_CK(b, cudaMemcpyAsync(&herr, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  FP_CK(b, cudaStreamSynchronize(s));
  if (herr & 1) return fp_fail(b, TRAJ_EINVAL, "a problem's KKT matrix is singular");
  b->n_problems = n_problems;
  b->max_np = max_np;
  b->max_no = max_no;
  b->have_problems = true;
  b->have_initial = false;
  b->have_result = false;
  return TRAJ_OK;
}

traj_status traj_fp_set_initial(traj_fp_batch *b, int n_traj, const int *traj_problem, const float *xi0) {
  if (!b) return TRAJ_EINVAL;
  if (!b->have_problems) return fp_fail(b, TRAJ_ESTATE, "traj_fp_set_problems must come first");
  if (!traj_problem || !xi0) return fp_fail(b, TRAJ_EINVAL, "NULL initial array");
  if (n_traj < 1 || n_traj > b->cfg.max_traj) return fp_fail(b, TRAJ_ESHAPE, "n_traj out of range");
  for (int k = 0; k < n_traj; ++k)
    if (traj_problem[k] < 0 || traj_problem[k] >= b->n_problems)
      return fp_fail(b, TRAJ_EINVAL, "traj_problem out of range");
  for (size_t e = 0; e < (size_t)n_traj * 3 * NC; ++e)
    if (!std::isfinite(xi0[e])) return fp_fail(b, TRAJ_ENAN, "non-finite initial coefficients");
  cudaStream_t s = b->stream;
  FP_CK(b, cudaMemcpyAsync(b->d_traj_problem, traj_problem, sizeof(int) * n_traj, cudaMemcpyHostToDevice, s));
  FP_CK(b, cudaMemcpyAsync(b->d_xi0, xi0, sizeof(float) * n_traj * 3 * NC, cudaMemcpyHostToDevice, s));
  FP_CK(b, cudaStreamSynchronize(s));
  b->n_traj = n_traj;
  b->have_initial = true;
  b->have_result = false;
  return TRAJ_OK;
}

traj_status traj_fp_solve(traj_fp_batch *b, int max_iters, float tol, traj_fp_stats *stats) {
  tb::NvtxRange nvtx_range("traj_fp_solve");
  if (!b) return TRAJ_EINVAL;
  if (!b->have_initial) return fp_fail(b, TRAJ_ESTATE, "traj_fp_set_initial must come first");
  if (max_iters < 0) return fp_fail(b, TRAJ_EINVAL, "max_iters must be >= 0");
  const traj_fp_config &c = b->cfg;
  FpArgs A{};
  A.n_traj = b->n_traj;
  A.n_c = c.n_circles;
  A.max_iters = max_iters;
  A.tol = tol;
  A.rho = c.rho;
  A.rho_psi = c.rho_psi;
  A.vmax = c.vmax;
  A.amax = c.amax;
  A.r_circle = c.r_circle;
  for (int m = 0; m < FP_MAX_CIRCLES; ++m) A.offs[m] = m < c.n_circles ? c.circle_offsets[m] : 0.f;
  A.traj_problem = b->d_traj_problem;
  A.problems = b->d_problems;
  A.tables = b->d_tables;
  A.consts = b->d_consts;
  A.obs = b->d_obs;
  A.obs_ax = b->d_ax;
  A.xi0 = b->d_xi0;
  A.xi_out = b->d_xi;
  A.res_out = b->d_res;
  A.iters_out = b->d_iters;
  const int max_np = b->max_np;
  A.mask_words = std::max(1, (b->max_no + 31) / 32);
  const size_t smem = sizeof(float) * FP_WARPS * (WS_FLOATS + A.mask_words);
  if (smem > 227 * 1024) // one 32-bit mask word per 32 obstacles of a problem, per warp
    return fp_fail(b, TRAJ_ESHAPE, "a problem has more obstacles than the solve's shared memory covers (456 704)");
  const int grid = (b->n_traj + FP_WARPS - 1) / FP_WARPS;
  cudaStream_t s = b->stream;
  auto kern = max_np <= 64 ? k_fp_solve<2> : max_np <= 128 ? k_fp_solve<4> : k_fp_solve<8>;
  FP_CK(b, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  FP_CK(b, cudaEventRecord(b->ev0, s));
  kern<<<grid, FP_WARPS * 32, smem, s>>>(A, max_np);
  FP_CK(b, cudaGetLastError());
  FP_CK(b, cudaEventRecord(b->ev1, s));
  b->have_result = true;
  if (stats) {
    FP_CK(b, cudaEventSynchronize(b->ev1));
    float ms = 0.f;
    FP_CK(b, cudaEventElapsedTime(&ms, b->ev0, b->ev1));
    std::vector<float> res((size_t)b->n_traj * 4);
    std::vector<int> it(b->n_traj);
    FP_CK(b, cudaMemcpy(res.data(), b->d_res, sizeof(float) * res.size(), cudaMemcpyDeviceToHost));
    FP_CK(b, cudaMemcpy(it.data(), b->d_iters, sizeof(int) * it.size(), cudaMemcpyDeviceToHost));
    int solved = 0, imax = 0;
    for (int k = 0; k < b->n_traj; ++k) {
      bool ok = true;
      for (int r = 0; r < 4; ++r) ok = ok && res[(size_t)k * 4 + r] <= tol;
      solved += ok ? 1 : 0;
      imax = std::max(imax, it[k]);
    }
    stats->gpu_ms = ms;
    stats->n_solved = solved;
    stats->max_iters_run = imax;
  }
  return TRAJ_OK;
}

traj_status traj_fp_get_trajectories(traj_fp_batch *b, float *coeffs, float *residual, int *iters) {
  if (!b) return TRAJ_EINVAL;
  if (!b->have_result) return fp_fail(b, TRAJ_ESTATE, "traj_fp_solve must come first");
  cudaStream_t s = b->stream;
  if (coeffs) FP_CK(b, cudaMemcpyAsync(coeffs, b->d_xi, sizeof(float) * b->n_traj * 5 * NC, cudaMemcpyDefault, s));
  if (residual) FP_CK(b, cudaMemcpyAsync(residual, b->d_res, sizeof(float) * b->n_traj * 4, cudaMemcpyDefault, s));
  if (iters) FP_CK(b, cudaMemcpyAsync(iters, b->d_iters, sizeof(int) * b->n_traj, cudaMemcpyDefault, s));
  FP_CK(b, cudaStreamSynchronize(s));
  return TRAJ_OK;
}

} // extern "C"

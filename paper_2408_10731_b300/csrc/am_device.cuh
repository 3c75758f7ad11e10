// am_device.cuh -- device building blocks of the AM iteration shared by the
// FP32 solve kernels (am_solve.cu) and the tensor-core form (am_mixed.cu):
// warp reductions, basis-row loads, the compensated QP step (Algorithm 2 line 2),
// the obstacle pair loop and the fused evaluate / project / contract pass
// (Algorithm 2 lines 4-6).
//
// Packed arithmetic: the 11 coefficients of an axis are held as six two-lane pairs
// (2i, 2i + 1), the twelfth lane zero, so that evaluation and contraction run on
// the f32x2 FMA (__ffma2_rn: two IEEE fmas per instruction), and the obstacle
// test runs on the two obstacles of a pair record at once.
#pragma once
#include <climits>

#include "internal.cuh"

namespace tb {

constexpr unsigned FULL = 0xffffffffu;

// Reduce-scatter of 32 per-lane values: afterwards lane L holds the warp sum of
// slot L (recursive halving; slot order preserved).
__device__ __forceinline__ float reduce_scatter32(float (&v)[32], int lane) {
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    const bool upper = (lane & s) != 0;
#pragma unroll
    for (int k = 0; k < s; ++k) {
      float send = upper ? v[k] : v[k + s];
      float keep = upper ? v[k + s] : v[k];
      v[k] = keep + __shfl_xor_sync(FULL, send, s);
    }
  }
  return v[0];
}

// 16 slots: plain reduction over lane halves, then reduce-scatter; lane L holds
// the warp sum of slot (L & 15).
__device__ __forceinline__ float reduce_scatter16(float (&v)[16], int lane) {
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] += __shfl_xor_sync(FULL, v[k], 16);
#pragma unroll
  for (int s = 8; s >= 1; s >>= 1) {
    const bool upper = (lane & s) != 0;
#pragma unroll
    for (int k = 0; k < s; ++k) {
      float send = upper ? v[k] : v[k + s];
      float keep = upper ? v[k + s] : v[k];
      v[k] = keep + __shfl_xor_sync(FULL, send, s);
    }
  }
  return v[0];
}

// Warp maximum of a non-negative float (a squared residual norm). Non-negative
// IEEE floats order as their bit patterns do as unsigned integers, so one
// redux.sync unsigned max gives the exact maximum (a NaN, whose pattern is above
// every finite one, is kept rather than dropped as fmaxf would).
__device__ __forceinline__ float warp_max(float x) {
  return __uint_as_float(__reduce_max_sync(FULL, __float_as_uint(x)));
}

__device__ __forceinline__ void load_row(const float *row, float (&r)[12]) {
  const float4 *r4 = reinterpret_cast<const float4 *>(row);
  float4 a = r4[0], b = r4[1], c = r4[2];
  r[0] = a.x; r[1] = a.y; r[2] = a.z; r[3] = a.w;
  r[4] = b.x; r[5] = b.y; r[6] = b.z; r[7] = b.w;
  r[8] = c.x; r[9] = c.y; r[10] = c.z; r[11] = c.w;
}

// Coefficient pairs of the iterate: xp[a][j] = (xi_a[2j], xi_a[2j+1]), xp[a][5].y = 0.
// Lane 16 a + i owns coefficient i of axis a < 2; axis 2 is owned by lanes i (< 11).
template <int DIM>
__device__ __forceinline__ void broadcast_pairs(float xo, float xo2, float2 (&xp)[DIM][6]) {
#pragma unroll
  for (int j = 0; j < 6; ++j) {
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      xp[a][j].x = __shfl_sync(FULL, xo, 16 * a + 2 * j);
      xp[a][j].y = j < 5 ? __shfl_sync(FULL, xo, 16 * a + 2 * j + 1) : 0.f;
    }
    if constexpr (DIM == 3) {
      xp[2][j].x = __shfl_sync(FULL, xo2, 2 * j);
      xp[2][j].y = j < 5 ? __shfl_sync(FULL, xo2, 2 * j + 1) : 0.f;
    }
  }
}

// Row (12 floats, column 11 zero) dotted with a coefficient-pair vector: six
// packed fmas over the pairs, then the two lanes added.
__device__ __forceinline__ float dot11(const float (&r)[12], const float2 (&xp)[6]) {
  float2 acc = __fmul2_rn(make_float2(r[0], r[1]), xp[0]);
#pragma unroll
  for (int j = 1; j < 6; ++j) acc = __ffma2_rn(make_float2(r[2 * j], r[2 * j + 1]), xp[j], acc);
  return acc.x + acc.y;
}

// up[j] += (r[2j], r[2j+1]) * R, the fmas of every coefficient in the order
// R_a (acceleration), R_v (velocity), R_o (obstacles).
__device__ __forceinline__ void contract_row3(float2 (&up)[6], const float (&rp)[12],
                                              const float (&rd)[12], const float (&ra)[12],
                                              float Ro, float Rv, float Ra) {
  const float2 o2 = make_float2(Ro, Ro), v2 = make_float2(Rv, Rv), a2 = make_float2(Ra, Ra);
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    float2 t = __ffma2_rn(make_float2(ra[2 * j], ra[2 * j + 1]), a2, up[j]);
    t = __ffma2_rn(make_float2(rd[2 * j], rd[2 * j + 1]), v2, t);
    up[j] = __ffma2_rn(make_float2(rp[2 * j], rp[2 * j + 1]), o2, t);
  }
}

// Reduce-scatter of the per-lane partial contraction (coefficient pairs) over the
// warp: afterwards lane 16 a + i holds u_a[i] (axis 2 of 3D: lanes i and 16 + i).
template <int DIM>
__device__ __forceinline__ void scatter_pairs(const float2 (&up)[DIM][6], int lane, float &uo,
                                              float &uo2) {
  float v32[32];
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    v32[i] = i < NC ? ((i & 1) ? up[0][i >> 1].y : up[0][i >> 1].x) : 0.f;
    v32[16 + i] = i < NC ? ((i & 1) ? up[1][i >> 1].y : up[1][i >> 1].x) : 0.f;
  }
  uo = reduce_scatter32(v32, lane);
  if constexpr (DIM == 3) {
    float v16[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) v16[i] = i < NC ? ((i & 1) ? up[2][i >> 1].y : up[2][i >> 1].x) : 0.f;
    uo2 = reduce_scatter16(v16, lane);
  } else {
    uo2 = 0.f;
  }
}

// hq of the QP step at the owner lanes from a constants block C: smoothness/tracking
// mode reads K11 (-q) + K12 b; projection mode forms K12 b + K11 xi_sample from the
// trajectory's own sample coefficients (xs, xs2 at the owner lanes), compensated.
template <int DIM>
__device__ __forceinline__ void load_hq(const float *C, int cost_mode, int lane, float xs, float xs2,
                                        float &hq_hi, float &hq_lo, float &hq2_hi, float &hq2_lo) {
  const int oa = lane >> 4, oi = lane & 15;
  const int ri = oi < NC ? oi : NC - 1;
  hq2_hi = 0.f; hq2_lo = 0.f;
  if (cost_mode == 0) {
    hq_hi = C[C_HQ_HI + oa * ROW + ri]; hq_lo = C[C_HQ_LO + oa * ROW + ri];
    if (DIM == 3) { hq2_hi = C[C_HQ_HI + 2 * ROW + ri]; hq2_lo = C[C_HQ_LO + 2 * ROW + ri]; }
    return;
  }
  hq_hi = C[C_C_HI + oa * ROW + ri]; hq_lo = C[C_C_LO + oa * ROW + ri];
  if (DIM == 3) { hq2_hi = C[C_C_HI + 2 * ROW + ri]; hq2_lo = C[C_C_LO + 2 * ROW + ri]; }
#pragma unroll
  for (int q = 0; q < NC; ++q) {
    const float xk = __shfl_sync(FULL, xs, (lane & 16) + q);
    df_fma(hq_hi, hq_lo, C[C_K11_HI + ri * ROW + q], C[C_K11_LO + ri * ROW + q], xk);
    if (DIM == 3) {
      const float xk2 = __shfl_sync(FULL, xs2, q);
      df_fma(hq2_hi, hq2_lo, C[C_K11_HI + ri * ROW + q], C[C_K11_LO + ri * ROW + q], xk2);
    }
  }
  // hq = c + K11 xi_sample: fold lo into hi once (both stay exact pairs)
  const float s = hq_hi + hq_lo; hq_lo = hq_lo - (s - hq_hi); hq_hi = s;
  if (DIM == 3) { const float s2 = hq2_hi + hq2_lo; hq2_lo = hq2_lo - (s2 - hq2_hi); hq2_hi = s2; }
}

// Penalty continuation: after iteration k, if the trajectory has not converged and k
// is a multiple of rho_every, move to the next rho of the ladder (its constants block
// and hq); returns true when the level changed.
template <int DIM>
__device__ __forceinline__ bool rho_step(const SolveArgs &A, int k, int &level, const float *Cb,
                                         const float *&C, float &rho, int lane, float xs, float xs2,
                                         float &hq_hi, float &hq_lo, float &hq2_hi, float &hq2_lo) {
  if (k == 0 || A.rho_every <= 0 || level + 1 >= A.rho_levels || (k % A.rho_every) != 0) return false;
  ++level;
  C = Cb + (size_t)level * CONST_FLOATS;
  rho = A.rho_ladder[level];
  load_hq<DIM>(C, A.cost_mode, lane, xs, xs2, hq_hi, hq_lo, hq2_hi, hq2_lo);
  return true;
}

// Resume or carry: the owner lanes' multipliers of trajectory b from the imported
// state, and its last contraction when one was imported (resume; a carried start
// forms u with its initial projection) (lane 16 a + i: axis a, coefficient i; axis 2
// at lanes i, 16 + i).
template <int DIM>
__device__ __forceinline__ void resume_state(const SolveArgs &A, int b, int oa, int ri, float &lam,
                                             float &lam2, float &uo, float &uo2) {
  const size_t base = (size_t)b * DIM * NC;
  lam = A.lam0[base + oa * NC + ri];
  if (A.u0) uo = A.u0[base + oa * NC + ri];
  if constexpr (DIM == 3) {
    lam2 = A.lam0[base + 2 * NC + ri];
    if (A.u0) uo2 = A.u0[base + 2 * NC + ri];
  }
}

// Algorithm 2 line 2 at the owner lanes, compensated FP32:
// xi^k = hq + G xi^{k-1} + K11 (lambda^{k-1} - rho u^{k-1}).
template <int DIM>
__device__ __forceinline__ void qp_step(const float *C, int lane, float rho, float hq_hi,
                                        float hq_lo, float hq2_hi, float hq2_lo, float lam,
                                        float lam2, float uo, float uo2, float &xo, float &xo2) {
  const int oi = lane & 15;
  const int ri = oi < NC ? oi : NC - 1;
  const float vo = lam - rho * uo, vo2 = lam2 - rho * uo2;
  float hi = hq_hi, lo = hq_lo, hi2 = hq2_hi, lo2 = hq2_lo;
  const float x_own = xo, x_own2 = xo2;
#pragma unroll
  for (int q = 0; q < NC; ++q) {
    const float xk = __shfl_sync(FULL, x_own, (lane & 16) + q);
    const float vk = __shfl_sync(FULL, vo, (lane & 16) + q);
    const float g_hi = C[C_G_HI + ri * ROW + q], g_lo = C[C_G_LO + ri * ROW + q];
    const float k_hi = C[C_K11_HI + ri * ROW + q], k_lo = C[C_K11_LO + ri * ROW + q];
    df_fma(hi, lo, g_hi, g_lo, xk);
    df_fma(hi, lo, k_hi, k_lo, vk);
    if constexpr (DIM == 3) {
      const float xk2 = __shfl_sync(FULL, x_own2, q);
      const float vk2 = __shfl_sync(FULL, vo2, q);
      df_fma(hi2, lo2, g_hi, g_lo, xk2);
      df_fma(hi2, lo2, k_hi, k_lo, vk2);
    }
  }
  xo = hi + lo;
  if constexpr (DIM == 3) xo2 = hi2 + lo2;
}

// ---- obstacles (Algorithm 2 lines 4-5 for the obstacle groups) ---------------------
// ||u||^2 - 1 of both obstacles of a record at one timestep (packed), with
// u = p * ia + (nc + nv t): negative inside the ellipse / ellipsoid.
template <int DIM>
__device__ __forceinline__ float2 pair_sm1(const float4 (&o)[pair_vec(DIM)], const float2 (&p2)[DIM],
                                           float2 t2) {
  constexpr int IA = DIM; // record index of {iax0, iax1, iay0, iay1}
  float2 ux = __ffma2_rn(make_float2(o[0].z, o[0].w), t2, make_float2(o[0].x, o[0].y));
  ux = __ffma2_rn(make_float2(o[IA].x, o[IA].y), p2[0], ux);
  float2 uy = __ffma2_rn(make_float2(o[1].z, o[1].w), t2, make_float2(o[1].x, o[1].y));
  uy = __ffma2_rn(make_float2(o[IA].z, o[IA].w), p2[1], uy);
  float2 s = __ffma2_rn(ux, ux, make_float2(-1.f, -1.f));
  s = __ffma2_rn(uy, uy, s);
  if constexpr (DIM == 3) {
    float2 uz = __ffma2_rn(make_float2(o[2].z, o[2].w), t2, make_float2(o[2].x, o[2].y));
    uz = __ffma2_rn(make_float2(o[4].x, o[4].y), p2[2], uz);
    s = __ffma2_rn(uz, uz, s);
  }
  return s;
}

// Projection of one timestep onto both obstacles of a record, packed: each half
// with sm < 0 (the point is inside) contributes g - p = (u * a) (1/||u|| - 1),
// the alpha and d steps giving g - o = Delta * max(1, 1/||u||) with Delta = u * a;
// at the centre atan2(0, 0) = 0 pushes along +x by the x semi-axis (3D: beta = 0,
// +z). A half with sm >= 0 contributes exactly zero. acc accumulates the halves in
// order; mo takes the max of ||g - p||^2.
template <int DIM>
__device__ __forceinline__ void pair_project(const float4 (&o)[pair_vec(DIM)], const float2 (&p2)[DIM],
                                             float2 t2, float2 sm, float (&acc)[DIM], float &mo) {
  constexpr int IA = DIM;
  float2 ux = __ffma2_rn(make_float2(o[0].z, o[0].w), t2, make_float2(o[0].x, o[0].y));
  ux = __ffma2_rn(make_float2(o[IA].x, o[IA].y), p2[0], ux);
  float2 uy = __ffma2_rn(make_float2(o[1].z, o[1].w), t2, make_float2(o[1].x, o[1].y));
  uy = __ffma2_rn(make_float2(o[IA].z, o[IA].w), p2[1], uy);
  float2 s = __ffma2_rn(uy, uy, __fmul2_rn(ux, ux));
  float2 uz = make_float2(0.f, 0.f), ax, ay, az = make_float2(0.f, 0.f);
  if constexpr (DIM == 3) {
    uz = __ffma2_rn(make_float2(o[2].z, o[2].w), t2, make_float2(o[2].x, o[2].y));
    uz = __ffma2_rn(make_float2(o[4].x, o[4].y), p2[2], uz);
    s = __ffma2_rn(uz, uz, s);
    ax = make_float2(o[4].z, o[4].w); ay = make_float2(o[5].x, o[5].y); az = make_float2(o[5].z, o[5].w);
  } else {
    ax = make_float2(o[3].x, o[3].y); ay = make_float2(o[3].z, o[3].w);
  }
  const bool in0 = sm.x < 0.f, in1 = sm.y < 0.f;
  const float w0 = (in0 && s.x > 0.f) ? fmaxf(rsqrtf(s.x) - 1.f, 0.f) : 0.f;
  const float w1 = (in1 && s.y > 0.f) ? fmaxf(rsqrtf(s.y) - 1.f, 0.f) : 0.f;
  const float2 w = make_float2(w0, w1);
  float2 ex = __fmul2_rn(__fmul2_rn(ux, ax), w);
  float2 ey = __fmul2_rn(__fmul2_rn(uy, ay), w);
  float2 ez = make_float2(0.f, 0.f);
  if constexpr (DIM == 3) ez = __fmul2_rn(__fmul2_rn(uz, az), w);
  const bool c0 = in0 && !(s.x > 0.f), c1 = in1 && !(s.y > 0.f); // at the centre
  if constexpr (DIM == 2) {
    if (c0) ex.x = ax.x;
    if (c1) ex.y = ax.y;
  } else {
    if (c0) ez.x = az.x;
    if (c1) ez.y = az.y;
  }
  acc[0] = (acc[0] + ex.x) + ex.y;
  acc[1] = (acc[1] + ey.x) + ey.y;
  float2 n2 = __ffma2_rn(ey, ey, __fmul2_rn(ex, ex));
  if constexpr (DIM == 3) {
    acc[2] = (acc[2] + ez.x) + ez.y;
    n2 = __ffma2_rn(ez, ez, n2);
  }
  mo = fmaxf(mo, fmaxf(n2.x, n2.y));
}

// The projections of one record whose test found a point inside: the semi-axes
// (the record's last float4) are loaded here, and only the timestep slots with a
// point inside are projected.
template <int DIM, int MAXNT>
__device__ __forceinline__ void project_record(float4 (&o)[pair_vec(DIM)], const float4 *rec,
                                               const float2 (&p2)[MAXNT][DIM],
                                               const float2 (&t2)[MAXNT], const float2 (&sm)[MAXNT],
                                               float (&acc)[MAXNT][DIM], float &mo) {
  constexpr int PV = pair_vec(DIM), PT = pair_test_vec(DIM);
#pragma unroll
  for (int k = PT; k < PV; ++k) o[k] = __ldg(&rec[k]);
#pragma unroll
  for (int m = 0; m < MAXNT; ++m)
    if ((int)(__float_as_uint(sm[m].x) | __float_as_uint(sm[m].y)) < 0)
      pair_project<DIM>(o, p2[m], t2[m], sm[m], acc[m], mo);
}

// Dense pair loop: all of the lane's timesteps against every obstacle-pair record
// of the problem, two records (four obstacles) per step, each with its own test.
// The tests are branch-free and packed; the sign bits of all ||u||^2 - 1 of a
// record are OR-ed, and only when one is negative (a point inside, a few percent of
// the tests) does the warp take that record's projection branch.
// acc accumulates sum_j (g_j - p) (= -sum_j r_j); mo is the lane's max ||r_j||^2.
template <int DIM, int MAXNT>
__device__ __forceinline__ void pair_loop_dense(const float (&pos)[MAXNT][DIM], const float (&tm)[MAXNT],
                                          const float4 *obs, int n_o, float (&acc)[MAXNT][DIM],
                                          float &mo) {
  constexpr int PV = pair_vec(DIM), PT = pair_test_vec(DIM);
  const int n_pairs = pair_count(n_o);
  float2 p2[MAXNT][DIM], t2[MAXNT];
#pragma unroll
  for (int m = 0; m < MAXNT; ++m) {
    t2[m] = make_float2(tm[m], tm[m]);
#pragma unroll
    for (int a = 0; a < DIM; ++a) p2[m][a] = make_float2(pos[m][a], pos[m][a]);
  }
  mo = 0.f;
  int q = 0;
  for (; q + 1 < n_pairs; q += 2) {
    float4 oa[PV], ob[PV];
#pragma unroll
    for (int k = 0; k < PT; ++k) {
      oa[k] = __ldg(&obs[PV * q + k]);
      ob[k] = __ldg(&obs[PV * (q + 1) + k]);
    }
    float2 sa[MAXNT], sb[MAXNT];
    unsigned ga = 0u, gb = 0u;
#pragma unroll
    for (int m = 0; m < MAXNT; ++m) {
      sa[m] = pair_sm1<DIM>(oa, p2[m], t2[m]);
      sb[m] = pair_sm1<DIM>(ob, p2[m], t2[m]);
      ga |= __float_as_uint(sa[m].x) | __float_as_uint(sa[m].y);
      gb |= __float_as_uint(sb[m].x) | __float_as_uint(sb[m].y);
    }
    if ((int)ga < 0) project_record<DIM, MAXNT>(oa, obs + PV * q, p2, t2, sa, acc, mo);
    if ((int)gb < 0) project_record<DIM, MAXNT>(ob, obs + PV * (q + 1), p2, t2, sb, acc, mo);
  }
  if (q < n_pairs) {
    float4 o[PV];
#pragma unroll
    for (int k = 0; k < PT; ++k) o[k] = __ldg(&obs[PV * q + k]);
    float2 sm[MAXNT];
    unsigned g = 0u;
#pragma unroll
    for (int m = 0; m < MAXNT; ++m) {
      sm[m] = pair_sm1<DIM>(o, p2[m], t2[m]);
      g |= __float_as_uint(sm[m].x) | __float_as_uint(sm[m].y);
    }
    if ((int)g < 0) project_record<DIM, MAXNT>(o, obs + PV * q, p2, t2, sm, acc, mo);
  }
}

// Order keys of floats for warp min/max reductions on the integer unit: the key
// k = bits ^ ((bits >> 31) & 0x7fffffff) orders as a signed integer as the floats
// do (the magnitude bits of a negative float reversed); the map is its own inverse.
__device__ __forceinline__ int float_key(float f) {
  const int b = __float_as_int(f);
  return b ^ ((b >> 31) & 0x7fffffff);
}
__device__ __forceinline__ float key_float(int k) { return __int_as_float(k ^ ((k >> 31) & 0x7fffffff)); }

// Culled pair loop: all of the lane's timesteps against the problem's obstacle-pair
// records, culled and exact: the records are taken 32 at a time, one per lane, and
// for every timestep slot the lane first bounds its record's normalised coordinate
// u = fma(ia, p, fma(nv, t, nc)) over the slot's box (the warp's least and greatest
// position per axis and time, over the slots' valid lanes) by evaluating that same
// expression at the box's corners: round-to-nearest is monotone and ia > 0, so the
// corner values bound the u that each lane's own test computes. Where u >= 1 or
// u <= -1 on some axis for both obstacles of a record, no lane's ||u||^2 - 1 can come
// out negative, so the record is left out of that slot (a ballot per slot). The
// records kept are then tested as before, two per step: packed and branch-free,
// and only when a sign bit is set (a point inside) does the warp take the
// projection branch. The results are bitwise those of testing every record; the
// records of a slot are visited in increasing order.
// acc accumulates sum_j (g_j - p) (= -sum_j r_j); mo is the lane's max ||r_j||^2.
template <int DIM, int MAXNT>
__device__ __forceinline__ void pair_loop_culled(const float (&pos)[MAXNT][DIM], const float (&tm)[MAXNT],
                                                 unsigned valid, const float4 *obs, int n_o,
                                                 float (&acc)[MAXNT][DIM], float &mo) {
  constexpr int PV = pair_vec(DIM), PT = pair_test_vec(DIM), IA = DIM;
  const int n_pairs = pair_count(n_o);
  const int lane = threadIdx.x & 31;
  float2 p2[MAXNT][DIM], t2[MAXNT];
#pragma unroll
  for (int m = 0; m < MAXNT; ++m) {
    t2[m] = make_float2(tm[m], tm[m]);
#pragma unroll
    for (int a = 0; a < DIM; ++a) p2[m][a] = make_float2(pos[m][a], pos[m][a]);
  }
  mo = 0.f;
  for (int k0 = 0; k0 < n_pairs; k0 += 32) {
    const int r = k0 + lane;
    float4 o[PT];
#pragma unroll
    for (int k = 0; k < PT; ++k)
      o[k] = r < n_pairs ? __ldg(&obs[PV * r + k]) : make_float4(0.f, 0.f, 0.f, 0.f);
    unsigned keep[MAXNT];
#pragma unroll
    for (int m = 0; m < MAXNT; ++m) {
      const bool v = (valid >> m) & 1u;
      const int kt0 = __reduce_min_sync(0xffffffffu, v ? __float_as_int(tm[m]) : INT_MAX);
      const int kt1 = __reduce_max_sync(0xffffffffu, v ? __float_as_int(tm[m]) : INT_MIN);
      const float2 ta = make_float2(__int_as_float(kt0), __int_as_float(kt0));
      const float2 tb = make_float2(__int_as_float(kt1), __int_as_float(kt1));
      bool out0 = false, out1 = false;
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        const int key = float_key(pos[m][a]);
        const float lo = key_float(__reduce_min_sync(0xffffffffu, v ? key : INT_MAX));
        const float hi = key_float(__reduce_max_sync(0xffffffffu, v ? key : INT_MIN));
        const float2 nc = make_float2(o[a].x, o[a].y), nv = make_float2(o[a].z, o[a].w);
        float2 ia;
        if constexpr (DIM == 2) ia = a == 0 ? make_float2(o[IA].x, o[IA].y) : make_float2(o[IA].z, o[IA].w);
        else ia = a == 0 ? make_float2(o[IA].x, o[IA].y)
                         : (a == 1 ? make_float2(o[IA].z, o[IA].w) : make_float2(o[IA + 1].x, o[IA + 1].y));
        const float2 i0 = __ffma2_rn(nv, ta, nc), i1 = __ffma2_rn(nv, tb, nc);
        const float2 umin = __ffma2_rn(ia, make_float2(lo, lo),
                                       make_float2(fminf(i0.x, i1.x), fminf(i0.y, i1.y)));
        const float2 umax = __ffma2_rn(ia, make_float2(hi, hi),
                                       make_float2(fmaxf(i0.x, i1.x), fmaxf(i0.y, i1.y)));
        out0 = out0 || umin.x >= 1.f || umax.x <= -1.f;
        out1 = out1 || umin.y >= 1.f || umax.y <= -1.f;
      }
      // an empty slot (no valid lane) keeps nothing
      keep[m] = __ballot_sync(0xffffffffu, kt0 != INT_MAX && r < n_pairs && !(out0 && out1));
    }
#pragma unroll
    for (int m = 0; m < MAXNT; ++m) {
      unsigned bits = keep[m];
      while (bits) {
        const int ra = k0 + __ffs(bits) - 1;
        bits &= bits - 1u;
        const bool two = bits != 0u;
        const int rb = two ? k0 + __ffs(bits) - 1 : ra; // a lone last record pairs with itself
        bits &= bits - 1u;
        float4 oa[PV], ob[PV];
#pragma unroll
        for (int k = 0; k < PT; ++k) {
          oa[k] = __ldg(&obs[PV * ra + k]);
          ob[k] = __ldg(&obs[PV * rb + k]);
        }
        const float2 sa = pair_sm1<DIM>(oa, p2[m], t2[m]);
        const float2 sb = pair_sm1<DIM>(ob, p2[m], t2[m]);
        if ((int)(__float_as_uint(sa.x) | __float_as_uint(sa.y)) < 0) {
#pragma unroll
          for (int k = PT; k < PV; ++k) oa[k] = __ldg(&obs[PV * ra + k]);
          pair_project<DIM>(oa, p2[m], t2[m], sa, acc[m], mo);
        }
        if (two && (int)(__float_as_uint(sb.x) | __float_as_uint(sb.y)) < 0) {
#pragma unroll
          for (int k = PT; k < PV; ++k) ob[k] = __ldg(&obs[PV * rb + k]);
          pair_project<DIM>(ob, p2[m], t2[m], sb, acc[m], mo);
        }
      }
    }
  }
}

// Which loop a kernel runs is fixed when it is compiled. The cull's fixed cost per
// timestep slot (the slot box's warp reductions, one record bound per lane and a
// ballot, about 50 instructions) pays for itself where a slot's 32 lanes hold 32
// consecutive grid points and the problem has more than about 12 records (24
// obstacles): each record a slot skips saves a packed test (about 8 instructions).
// The one-warp and team kernels run the culled loop; the long-horizon chunks serve
// problems with few obstacles (n_o = 10 in Paper I) and run the dense one.
template <int DIM, int MAXNT, bool CULL>
__device__ __forceinline__ void pair_loop(const float (&pos)[MAXNT][DIM], const float (&tm)[MAXNT],
                                          unsigned valid, const float4 *obs, int n_o,
                                          float (&acc)[MAXNT][DIM], float &mo) {
  if constexpr (CULL)
    pair_loop_culled<DIM, MAXNT>(pos, tm, valid, obs, n_o, acc, mo);
  else
    pair_loop_dense<DIM, MAXNT>(pos, tm, obs, n_o, acc, mo);
}

// Workspace bounds (PRIEST's G xi <= tau, G = [-P; P] per axis, slack s = max(0, tau -
// G xi)): the residual rows are max(lo - p, 0) and max(p - hi, 0), i.e. the point's
// offset from the box, p - clamp(p, lo, hi), which joins the obstacle group's sum
// (P^T G^T r has the basis P) and its maximum norm.
template <int DIM, int MAXNT>
__device__ __forceinline__ void box_residuals(const ProblemDev *pr, const float (&pos)[MAXNT][DIM],
                                              int t0, int ts, int n_p, int nt,
                                              float (&acc)[MAXNT][DIM], float &mo) {
  float lo[DIM], hi[DIM];
#pragma unroll
  for (int a = 0; a < DIM; ++a) { lo[a] = pr->lo[a]; hi[a] = pr->hi[a]; }
#pragma unroll
  for (int m = 0; m < MAXNT; ++m) {
    if (m < nt && t0 + ts * m < n_p) {
      float n2 = 0.f;
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        const float r = pos[m][a] - fminf(fmaxf(pos[m][a], lo[a]), hi[a]);
        acc[m][a] -= r;
        n2 = fmaf(r, r, n2);
      }
      mo = fmaxf(mo, n2);
    }
  }
}

// ---- evaluate / project / contract ---------------------------------------------------
// Positions p(t) = P xi at the lane's timesteps t = t0 + ts m (padding slots get a far
// sentinel, which is outside every obstacle); bit m of valid is set for a slot that
// holds a grid point.
template <int DIM, int MAXNT>
__device__ __forceinline__ void eval_positions(const float2 (&xp)[DIM][6], const float *tP, int n_p,
                                               int nt, float dt, int t0, int ts,
                                               float (&pos)[MAXNT][DIM], float (&tm)[MAXNT],
                                               unsigned &valid) {
  valid = 0u;
#pragma unroll
  for (int m = 0; m < MAXNT; ++m) {
    const int t = t0 + ts * m;
    tm[m] = dt * (float)t;
#pragma unroll
    for (int a = 0; a < DIM; ++a) pos[m][a] = 1.0e18f;
    if (m < nt && t < n_p) {
      valid |= 1u << m;
      float r[12];
      load_row(tP + t * ROW, r);
#pragma unroll
      for (int a = 0; a < DIM; ++a) pos[m][a] = dot11(r, xp[a]);
    }
  }
}

// Velocity / acceleration at one timestep and their projections onto the bound
// balls: r = w max(0, 1 - bound/||w||). Returns the time-scaled residuals
// Rv = r_v / T and Ra = r_a / T^2 (so that Pd^T r_v = dB^T Rv) and raises the maxima.
template <int DIM>
__device__ __forceinline__ void bound_residuals(const float2 (&xp)[DIM][6], const float (&rd)[12],
                                                const float (&ra)[12], float invT, float invT2,
                                                float vmax, float amax, float (&Rv)[DIM],
                                                float (&Ra)[DIM], float &mv, float &ma) {
  float vel[DIM], ac[DIM], nv2 = 0.f, na2 = 0.f;
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    vel[a] = dot11(rd, xp[a]) * invT;
    ac[a] = dot11(ra, xp[a]) * invT2;
    nv2 = fmaf(vel[a], vel[a], nv2);
    na2 = fmaf(ac[a], ac[a], na2);
  }
  float fv = 0.f, fa = 0.f;
  if (nv2 > vmax * vmax) { fv = 1.f - vmax * rsqrtf(nv2); mv = fmaxf(mv, nv2 * fv * fv); }
  if (na2 > amax * amax) { fa = 1.f - amax * rsqrtf(na2); ma = fmaxf(ma, na2 * fa * fa); }
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    Rv[a] = vel[a] * fv * invT;
    Ra[a] = ac[a] * fa * invT2;
  }
}

// Evaluate, project and contract one iterate (Algorithm 2 lines 4-6, minus the
// multiplier update). The lane's timesteps are t = t0 + ts m (ts = 32 when one warp
// owns a trajectory; the culled pair loop wants that). Returns the per-lane partial
// contraction u = F^T r as coefficient pairs up[DIM][6] and the lane maxima of
// ||r_j||^2, ||r_v||^2, ||r_a||^2.
template <int DIM, int MAXNT, bool CULL>
__device__ __forceinline__ void project_contract(
    const float2 (&xp)[DIM][6], const float *tP, const float *tD, const float *tA,
    const float4 *obs, const ProblemDev *pr, int n_p, int nt, float dt, float invT, float invT2,
    float vmax, float amax, int t0, float2 (&up)[DIM][6], float &mo, float &mv, float &ma,
    int ts = 32) {
  float pos[MAXNT][DIM], acc[MAXNT][DIM], tm[MAXNT];
  unsigned valid;
  eval_positions<DIM, MAXNT>(xp, tP, n_p, nt, dt, t0, ts, pos, tm, valid);
#pragma unroll
  for (int m = 0; m < MAXNT; ++m)
#pragma unroll
    for (int a = 0; a < DIM; ++a) acc[m][a] = 0.f;
  pair_loop<DIM, MAXNT, CULL>(pos, tm, valid, obs, pr->n_o, acc, mo);
  if (pr->box) box_residuals<DIM, MAXNT>(pr, pos, t0, ts, n_p, nt, acc, mo);
#pragma unroll
  for (int a = 0; a < DIM; ++a)
#pragma unroll
    for (int j = 0; j < 6; ++j) up[a][j] = make_float2(0.f, 0.f);
  mv = 0.f; ma = 0.f;
#pragma unroll
  for (int m = 0; m < MAXNT; ++m) {
    const int t = t0 + ts * m;
    if (m < nt && t < n_p) {
      float rp[12], rd[12], ra[12];
      load_row(tP + t * ROW, rp);
      load_row(tD + t * ROW, rd);
      load_row(tA + t * ROW, ra);
      float Rv[DIM], Ra[DIM];
      bound_residuals<DIM>(xp, rd, ra, invT, invT2, vmax, amax, Rv, Ra, mv, ma);
#pragma unroll
      for (int a = 0; a < DIM; ++a) contract_row3(up[a], rp, rd, ra, -acc[m][a], Rv[a], Ra[a]);
    }
  }
}

// Long horizons (more grid points than a lane holds in registers): the lane's
// timesteps t = c0 + lane + 32 m, m < CNT, one chunk of 32 CNT grid points at a
// time, each chunk evaluated, projected onto every obstacle and the bounds, and
// contracted; the contraction and the residual maxima accumulate over the chunks.
template <int DIM, int CNT>
__device__ __forceinline__ void project_contract_chunked(
    const float2 (&xp)[DIM][6], const float *tP, const float *tD, const float *tA,
    const float4 *obs, const ProblemDev *pr, int n_p, float dt, float invT, float invT2,
    float vmax, float amax, int lane, float2 (&up)[DIM][6], float &mo, float &mv, float &ma) {
#pragma unroll
  for (int a = 0; a < DIM; ++a)
#pragma unroll
    for (int j = 0; j < 6; ++j) up[a][j] = make_float2(0.f, 0.f);
  mo = 0.f; mv = 0.f; ma = 0.f;
  for (int c0 = 0; c0 < n_p; c0 += 32 * CNT) {
    const int nt = min(CNT, (n_p - c0 + 31) >> 5);
    float pos[CNT][DIM], acc[CNT][DIM], tm[CNT];
    unsigned valid;
    eval_positions<DIM, CNT>(xp, tP, n_p, nt, dt, c0 + lane, 32, pos, tm, valid);
#pragma unroll
    for (int m = 0; m < CNT; ++m)
#pragma unroll
      for (int a = 0; a < DIM; ++a) acc[m][a] = 0.f;
    float moc;
    pair_loop<DIM, CNT, false>(pos, tm, valid, obs, pr->n_o, acc, moc);
    mo = fmaxf(mo, moc);
    if (pr->box) box_residuals<DIM, CNT>(pr, pos, c0 + lane, 32, n_p, nt, acc, mo);
#pragma unroll
    for (int m = 0; m < CNT; ++m) {
      const int t = c0 + lane + 32 * m;
      if (m < nt && t < n_p) {
        float rp[12], rd[12], ra[12];
        load_row(tP + t * ROW, rp);
        load_row(tD + t * ROW, rd);
        load_row(tA + t * ROW, ra);
        float Rv[DIM], Ra[DIM];
        bound_residuals<DIM>(xp, rd, ra, invT, invT2, vmax, amax, Rv, Ra, mv, ma);
#pragma unroll
        for (int a = 0; a < DIM; ++a) contract_row3(up[a], rp, rd, ra, -acc[m][a], Rv[a], Ra[a]);
      }
    }
  }
}

// Evaluate and project one iterate without the contraction (the tensor-core form
// contracts on the MMA; one warp per trajectory, the culled pair loop): per lane and
// timestep slot, the residual vectors
// Ro = sum_j r_j, Rv = r_v / T and Ra = r_a / T^2 (zero past the horizon) and the
// lane maxima of ||r_j||^2, ||r_v||^2, ||r_a||^2.
template <int DIM, int NT>
__device__ __forceinline__ void project_only(
    const float2 (&xp)[DIM][6], const float *tP, const float *tD, const float *tA,
    const float4 *obs, const ProblemDev *pr, int n_p, float dt, float invT, float invT2,
    float vmax, float amax, int t0, float (&Ro)[NT][DIM], float (&Rv)[NT][DIM],
    float (&Ra)[NT][DIM], float &mo, float &mv, float &ma, int ts = 32) {
  float pos[NT][DIM], acc[NT][DIM], tm[NT];
  unsigned valid;
  eval_positions<DIM, NT>(xp, tP, n_p, NT, dt, t0, ts, pos, tm, valid);
#pragma unroll
  for (int m = 0; m < NT; ++m)
#pragma unroll
    for (int a = 0; a < DIM; ++a) acc[m][a] = 0.f;
  pair_loop<DIM, NT, true>(pos, tm, valid, obs, pr->n_o, acc, mo);
  if (pr->box) box_residuals<DIM, NT>(pr, pos, t0, ts, n_p, NT, acc, mo);
  mv = 0.f; ma = 0.f;
#pragma unroll
  for (int m = 0; m < NT; ++m) {
    const int t = t0 + ts * m;
#pragma unroll
    for (int a = 0; a < DIM; ++a) { Ro[m][a] = 0.f; Rv[m][a] = 0.f; Ra[m][a] = 0.f; }
    if (t < n_p) {
      float rd[12], ra[12];
      load_row(tD + t * ROW, rd);
      load_row(tA + t * ROW, ra);
      bound_residuals<DIM>(xp, rd, ra, invT, invT2, vmax, amax, Rv[m], Ra[m], mv, ma);
#pragma unroll
      for (int a = 0; a < DIM; ++a) Ro[m][a] = -acc[m][a];
    }
  }
}

// FP32 contraction of residuals produced by project_only: per-lane partial
// u = P^T Ro + dB^T Rv + d2B^T Ra over the lane's timesteps, as coefficient pairs.
template <int DIM, int NT>
__device__ __forceinline__ void contract_fp32(const float (&Ro)[NT][DIM], const float (&Rv)[NT][DIM],
                                              const float (&Ra)[NT][DIM], const float *tP,
                                              const float *tD, const float *tA, int n_p, int t0,
                                              float2 (&up)[DIM][6], int ts = 32) {
#pragma unroll
  for (int a = 0; a < DIM; ++a)
#pragma unroll
    for (int j = 0; j < 6; ++j) up[a][j] = make_float2(0.f, 0.f);
#pragma unroll
  for (int m = 0; m < NT; ++m) {
    const int t = t0 + ts * m;
    if (t < n_p) {
      float rp[12], rd[12], ra[12];
      load_row(tP + t * ROW, rp);
      load_row(tD + t * ROW, rd);
      load_row(tA + t * ROW, ra);
#pragma unroll
      for (int a = 0; a < DIM; ++a) contract_row3(up[a], rp, rd, ra, Ro[m][a], Rv[m][a], Ra[m][a]);
    }
  }
}

} // namespace tb

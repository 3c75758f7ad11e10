// am_device.cuh -- device building blocks of the AM iteration shared by the
// FP32 solve kernel (am_solve.cu) and the tensor-core form (am_mixed.cu):
// warp reductions, basis-row loads, the obstacle pair loop and the fused
// evaluate / project / contract pass (Algorithm 2 lines 4-6).
#pragma once
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

__device__ __forceinline__ float warp_max(float x) {
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) x = fmaxf(x, __shfl_xor_sync(FULL, x, s));
  return x;
}

__device__ __forceinline__ void load_row(const float *row, float (&r)[12]) {
  const float4 *r4 = reinterpret_cast<const float4 *>(row);
  float4 a = r4[0], b = r4[1], c = r4[2];
  r[0] = a.x; r[1] = a.y; r[2] = a.z; r[3] = a.w;
  r[4] = b.x; r[5] = b.y; r[6] = b.z; r[7] = b.w;
  r[8] = c.x; r[9] = c.y; r[10] = c.z; r[11] = c.w;
}

// Pair loop over obstacles (Algorithm 2 lines 4-5 for the obstacle groups): acc
// accumulates sum_j Delta_j * w_j (r_j = -Delta_j w_j) at each of the lane's
// timesteps; mo is the lane's max ||r_j||^2.
template <int DIM, int MAXNT>
__device__ __forceinline__ void pair_loop(const float (&pos)[MAXNT][DIM], const float (&tm)[MAXNT],
                                          const float4 *obs, int n_o, float (&acc)[MAXNT][DIM],
                                          float &mo) {
  constexpr int OV = obs_vec(DIM);
  // The containment tests of a pair of obstacles against all of a lane's
  // timesteps are computed branch-free (x and y packed in f32x2 lanes) and
  // combined with one min; only when one of them contains a point does the
  // warp take the projection branch (rare once the iterates are outside).
  mo = 0.f;
  for (int j = 0; j < n_o; j += 2) {
    float4 o[2][OV];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (j + h < n_o) {
#pragma unroll
        for (int q = 0; q < OV; ++q) o[h][q] = __ldg(&obs[OV * (j + h) + q]);
      } else { // tail sentinel: static, 1e18 m away, unit axes: never inside
        if constexpr (DIM == 2) {
          o[h][0] = make_float4(1.0e18f, 1.0e18f, 0.f, 0.f);
          o[h][1] = make_float4(1.f, 1.f, 1.f, 1.f);
        } else {
          o[h][0] = make_float4(1.0e18f, 1.0e18f, 1.0e18f, 1.f);
          o[h][1] = make_float4(0.f, 0.f, 0.f, 1.f);
          o[h][2] = make_float4(1.f, 1.f, 1.f, 1.f);
        }
      }
    }
    float d[2][MAXNT][DIM], s[2][MAXNT];
    float smin = 3.0e38f;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
#pragma unroll
      for (int m = 0; m < MAXNT; ++m) {
        if constexpr (DIM == 2) {
          const float2 nc = make_float2(o[h][0].x, o[h][0].y), nv = make_float2(o[h][0].z, o[h][0].w);
          const float2 ia = make_float2(o[h][1].x, o[h][1].y);
          const float2 pc = __fadd2_rn(make_float2(pos[m][0], pos[m][1]), nc);
          const float2 dd = __ffma2_rn(nv, make_float2(tm[m], tm[m]), pc);
          const float2 uu = __fmul2_rn(dd, ia);
          d[h][m][0] = dd.x; d[h][m][1] = dd.y;
          s[h][m] = fmaf(uu.y, uu.y, uu.x * uu.x);
        } else {
          const float2 nc = make_float2(o[h][0].x, o[h][0].y), nv = make_float2(o[h][1].x, o[h][1].y);
          const float2 ia = make_float2(o[h][0].w, o[h][1].w);
          const float2 pc = __fadd2_rn(make_float2(pos[m][0], pos[m][1]), nc);
          const float2 dd = __ffma2_rn(nv, make_float2(tm[m], tm[m]), pc);
          const float2 uu = __fmul2_rn(dd, ia);
          const float dz = fmaf(o[h][1].z, tm[m], pos[m][2] + o[h][0].z);
          const float uz = dz * o[h][2].w;
          d[h][m][0] = dd.x; d[h][m][1] = dd.y; d[h][m][2] = dz;
          s[h][m] = fmaf(uz, uz, fmaf(uu.y, uu.y, uu.x * uu.x));
        }
        smin = fminf(smin, s[h][m]);
      }
    }
    if (smin < 1.f) { // some timestep is inside one of the two ellipses
#pragma unroll
      for (int h = 0; h < 2; ++h) {
#pragma unroll
        for (int m = 0; m < MAXNT; ++m) {
          if (s[h][m] < 1.f) {
            float e[DIM];
            if (s[h][m] > 0.f) { // project along the ray: target offset Delta / ||u||
              const float w = rsqrtf(s[h][m]) - 1.f;
#pragma unroll
              for (int a = 0; a < DIM; ++a) e[a] = d[h][m][a] * w;
            } else { // at the centre: atan2(0, 0) = 0 pushes along +x (3D: beta = 0, +z)
#pragma unroll
              for (int a = 0; a < DIM; ++a) e[a] = 0.f;
              if constexpr (DIM == 2) e[0] = o[h][1].z; else e[2] = o[h][2].z;
            }
            float n2 = 0.f;
#pragma unroll
            for (int a = 0; a < DIM; ++a) { acc[m][a] += e[a]; n2 = fmaf(e[a], e[a], n2); }
            mo = fmaxf(mo, n2);
          }
        }
      }
    }
  }
}

// Evaluate, project and contract one iterate (Algorithm 2 lines 4-6, minus the
// multiplier update). The lane's timesteps are t = lane + ts * m (the caller
// passes its first timestep as `lane`; ts = 32 when one warp owns a trajectory). xa: the iterate's coefficients (all lanes hold all).
// Returns the per-lane partial contraction in up[DIM][11] and per-lane maxima
// of ||r_j||^2, ||r_v||^2, ||r_a||^2.
template <int DIM, int MAXNT>
__device__ __forceinline__ void project_contract(
    const float (&xa)[DIM][NC], const float *tP, const float *tD, const float *tA,
    const float4 *obs, int n_o, int n_p, int nt, float dt, float invT, float invT2, float vmax,
    float amax, int lane, float (&up)[DIM][NC], float &mo, float &mv, float &ma, int ts = 32) {
  constexpr int OV = obs_vec(DIM);
  float pos[MAXNT][DIM], acc[MAXNT][DIM], tm[MAXNT];
  // positions p(t) = P xi at this lane's timesteps; padding lanes get a far sentinel
#pragma unroll
  for (int m = 0; m < MAXNT; ++m) {
    const int t = lane + ts * m;
    tm[m] = dt * (float)t;
#pragma unroll
    for (int a = 0; a < DIM; ++a) { pos[m][a] = 1.0e18f; acc[m][a] = 0.f; }
    if (m < nt && t < n_p) {
      float r[12];
      load_row(tP + t * ROW, r);
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        float s = 0.f;
#pragma unroll
        for (int i = 0; i < NC; ++i) s = fmaf(r[i], xa[a][i], s);
        pos[m][a] = s;
      }
    }
  }
  pair_loop<DIM, MAXNT>(pos, tm, obs, n_o, acc, mo);
  // velocity / acceleration projections and the contraction u = F^T r
#pragma unroll
  for (int a = 0; a < DIM; ++a)
#pragma unroll
    for (int i = 0; i < NC; ++i) up[a][i] = 0.f;
  mv = 0.f; ma = 0.f;
  const float vmax2 = vmax * vmax, amax2 = amax * amax;
#pragma unroll
  for (int m = 0; m < MAXNT; ++m) {
    const int t = lane + ts * m;
    if (m < nt && t < n_p) {
      float rp[12], rd[12], ra[12];
      load_row(tP + t * ROW, rp);
      load_row(tD + t * ROW, rd);
      load_row(tA + t * ROW, ra);
      float vel[DIM], ac[DIM], nv2 = 0.f, na2 = 0.f;
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        float sv = 0.f, sa = 0.f;
#pragma unroll
        for (int i = 0; i < NC; ++i) { sv = fmaf(rd[i], xa[a][i], sv); sa = fmaf(ra[i], xa[a][i], sa); }
        vel[a] = sv * invT; ac[a] = sa * invT2;
        nv2 = fmaf(vel[a], vel[a], nv2); na2 = fmaf(ac[a], ac[a], na2);
      }
      float fv = 0.f, fa = 0.f;
      if (nv2 > vmax2) { fv = 1.f - vmax * rsqrtf(nv2); mv = fmaxf(mv, nv2 * fv * fv); }
      if (na2 > amax2) { fa = 1.f - amax * rsqrtf(na2); ma = fmaxf(ma, na2 * fa * fa); }
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        const float Ro = -acc[m][a];              // sum_j r_j at t
        const float Rv = vel[a] * fv * invT;      // Pd^T r_v = dB^T (r_v / T)
        const float Ra = ac[a] * fa * invT2;      // Pdd^T r_a = d2B^T (r_a / T^2)
#pragma unroll
        for (int i = 0; i < NC; ++i) up[a][i] = fmaf(rp[i], Ro, fmaf(rd[i], Rv, fmaf(ra[i], Ra, up[a][i])));
      }
    }
  }
}

// Evaluate and project one iterate without the contraction (the tensor-core form
// contracts on the MMA): per lane and timestep slot, the residual vectors
// Ro = sum_j r_j, Rv = r_v / T and Ra = r_a / T^2 (the time scaling folded in,
// zero past the horizon) and the lane maxima of ||r_j||^2, ||r_v||^2, ||r_a||^2.
template <int DIM, int NT>
__device__ __forceinline__ void project_only(
    const float (&xa)[DIM][NC], const float *tP, const float *tD, const float *tA,
    const float4 *obs, int n_o, int n_p, float dt, float invT, float invT2, float vmax, float amax,
    int lane, float (&Ro)[NT][DIM], float (&Rv)[NT][DIM], float (&Ra)[NT][DIM], float &mo,
    float &mv, float &ma, int ts = 32) {
  float pos[NT][DIM], acc[NT][DIM], tm[NT];
#pragma unroll
  for (int m = 0; m < NT; ++m) {
    const int t = lane + ts * m;
    tm[m] = dt * (float)t;
#pragma unroll
    for (int a = 0; a < DIM; ++a) { pos[m][a] = 1.0e18f; acc[m][a] = 0.f; }
    if (t < n_p) {
      float r[12];
      load_row(tP + t * ROW, r);
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        float s = 0.f;
#pragma unroll
        for (int i = 0; i < NC; ++i) s = fmaf(r[i], xa[a][i], s);
        pos[m][a] = s;
      }
    }
  }
  pair_loop<DIM, NT>(pos, tm, obs, n_o, acc, mo);
  mv = 0.f; ma = 0.f;
  const float vmax2 = vmax * vmax, amax2 = amax * amax;
#pragma unroll
  for (int m = 0; m < NT; ++m) {
    const int t = lane + ts * m;
#pragma unroll
    for (int a = 0; a < DIM; ++a) { Ro[m][a] = 0.f; Rv[m][a] = 0.f; Ra[m][a] = 0.f; }
    if (t < n_p) {
      float rd[12], rA[12];
      load_row(tD + t * ROW, rd);
      load_row(tA + t * ROW, rA);
      float vel[DIM], ac[DIM], nv2 = 0.f, na2 = 0.f;
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        float sv = 0.f, sa = 0.f;
#pragma unroll
        for (int i = 0; i < NC; ++i) { sv = fmaf(rd[i], xa[a][i], sv); sa = fmaf(rA[i], xa[a][i], sa); }
        vel[a] = sv * invT; ac[a] = sa * invT2;
        nv2 = fmaf(vel[a], vel[a], nv2); na2 = fmaf(ac[a], ac[a], na2);
      }
      float fv = 0.f, fa = 0.f;
      if (nv2 > vmax2) { fv = 1.f - vmax * rsqrtf(nv2); mv = fmaxf(mv, nv2 * fv * fv); }
      if (na2 > amax2) { fa = 1.f - amax * rsqrtf(na2); ma = fmaxf(ma, na2 * fa * fa); }
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        Ro[m][a] = -acc[m][a];
        Rv[m][a] = vel[a] * fv * invT;
        Ra[m][a] = ac[a] * fa * invT2;
      }
    }
  }
}

// FP32 contraction of residuals produced by project_only: per-lane partial
// u = P^T Ro + dB^T Rv + d2B^T Ra over the lane's timesteps.
template <int DIM, int NT>
__device__ __forceinline__ void contract_fp32(const float (&Ro)[NT][DIM], const float (&Rv)[NT][DIM],
                                              const float (&Ra)[NT][DIM], const float *tP,
                                              const float *tD, const float *tA, int n_p, int lane,
                                              float (&up)[DIM][NC], int ts = 32) {
#pragma unroll
  for (int a = 0; a < DIM; ++a)
#pragma unroll
    for (int i = 0; i < NC; ++i) up[a][i] = 0.f;
#pragma unroll
  for (int m = 0; m < NT; ++m) {
    const int t = lane + ts * m;
    if (t < n_p) {
      float rp[12], rd[12], rA[12];
      load_row(tP + t * ROW, rp);
      load_row(tD + t * ROW, rd);
      load_row(tA + t * ROW, rA);
#pragma unroll
      for (int a = 0; a < DIM; ++a)
#pragma unroll
        for (int i = 0; i < NC; ++i)
          up[a][i] = fmaf(rp[i], Ro[m][a], fmaf(rd[i], Rv[m][a], fmaf(rA[i], Ra[m][a], up[a][i])));
    }
  }
}

} // namespace tb

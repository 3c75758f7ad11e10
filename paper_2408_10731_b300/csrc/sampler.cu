// sampler.cu -- the projection-guided sampler of Paper III (PRIEST, Algorithm 3)
// around the batched projection optimizer.
//
// One outer iteration l (traj_sampler_step):
//   1. Cholesky of Sigma + eps I (one CTA) and N_b samples xi_i = mu + L z_i,
//      z from an own Philox4x32-10 generator (Salmon et al., SC'11) with the
//      Box-Muller transform, or from caller-supplied normal draws;
//   2. the AM solve kernel in projection mode (Q = I, q = -xi_i, eq.
//      matrix_vec) for n_inner iterations;
//   3. residual r_i (worst of the three L-infinity residuals) and augmented
//      cost c_aug = c_1 + w_r r with c_1 = sum_t ||p''(t)||^2 (Algorithm 3), plus
//      optional curvature and path-distance terms (the BARN cost of Section 5);
//   4. ConstraintEliteSet: the N_proj lowest r; EliteSet: the N_elite lowest
//      c_aug among them (deterministic bitonic sorts on (key, index));
//   5. weights c_m = exp(-(c_aug,m - delta)/gamma), delta = min c_aug, and the
//      updates of eqs. update_mean and update_covariance (the covariance uses
//      the new mean). The sign of the exponent follows the reading that good
//      samples weigh more.
// Decentralised form (D-PRIEST): the batch splits into n_dist contiguous groups
// of B / n_dist samples, each with its own mean and covariance. The Cholesky,
// selection and refit kernels take one CTA per group, so every stage is one
// launch for all distributions; the projection solve is one launch as before.
#include "internal.cuh"
#include <math.h>

namespace tb {

// ---- Philox4x32-10 ----------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
    const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += W0; k.y += W1;
  }
  return c;
}

// 32-bit integer -> uniform in (0, 1): (x + 0.5) / 2^32
__device__ __forceinline__ float u01(uint32_t x) { return ((float)x + 0.5f) * 2.3283064365386963e-10f; }

// ---- kernels ----------------------------------------------------------------
// Cholesky of Sigma_g + eps I (D x D, D <= 48) into L_g (lower, row-major). One
// CTA per distribution g = blockIdx.x.
__global__ void k_cholesky(const float *sigma, int D, float eps, float *L, int *flag) {
  __shared__ float A[48 * 48];
  sigma += (size_t)blockIdx.x * D * D;
  L += (size_t)blockIdx.x * D * D;
  for (int e = threadIdx.x; e < D * D; e += blockDim.x) {
    const int i = e / D, j = e % D;
    A[e] = 0.5f * (sigma[i * D + j] + sigma[j * D + i]) + (i == j ? eps : 0.f);
  }
  __syncthreads();
  for (int j = 0; j < D; ++j) {
    if (threadIdx.x == 0) {
      float d = A[j * D + j];
      for (int k = 0; k < j; ++k) d -= A[j * D + k] * A[j * D + k];
      if (!(d > 0.f)) { atomicOr(flag, 4); d = 1e-30f; }
      A[j * D + j] = sqrtf(d);
    }
    __syncthreads();
    for (int i = j + 1 + threadIdx.x; i < D; i += blockDim.x) {
      float s = A[i * D + j];
      for (int k = 0; k < j; ++k) s -= A[i * D + k] * A[j * D + k];
      A[i * D + j] = s / A[j * D + j];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < D * D; e += blockDim.x) {
    const int i = e / D, j = e % D;
    L[e] = j <= i ? A[e] : 0.f;
  }
}

// xi_i = mu_g + L_g z_i for sample i of group g = i / Bg. z from `z` ([B][D]) or,
// when z == nullptr, Philox with counter (i, iteration, pair, 0) and key (seed lo,
// seed hi); Box-Muller pairs.
// One warp per sample (SAMPLE_WARPS per block): the lanes share its Philox calls (lane l
// takes the call of counter q = 2 l), then its output rows (d = lane, lane + 32),
// each row summed in the same order as a single thread would.
constexpr int SAMPLE_WARPS = 4;
__global__ void k_sample(const float *mu, const float *L, int D, int B, int Bg, const float *z,
                         unsigned long long seed, int iteration, float *xi0, float *samples_out) {
  __shared__ float zs[SAMPLE_WARPS][48];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * SAMPLE_WARPS + w;
  if (i >= B) return; // whole warps
  const int g = i / Bg;
  mu += (size_t)g * D;
  L += (size_t)g * D * D;
  float *zz = zs[w];
  if (z) {
    for (int d = lane; d < D; d += 32) zz[d] = z[(size_t)i * D + d];
  } else {
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    const int q = 2 * lane; // one Philox call -> two Box-Muller pairs
    if (2 * q < D) {
      const uint4 r = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)iteration, (uint32_t)q, 0u), key);
      const uint32_t wv[4] = {r.x, r.y, r.z, r.w};
      for (int h = 0; h < 2; ++h) {
        const float rad = sqrtf(-2.f * logf(u01(wv[2 * h])));
        float sn, cs;
        sincospif(2.f * u01(wv[2 * h + 1]), &sn, &cs);
        const int d0 = 2 * (q + h);
        if (d0 < D) zz[d0] = rad * cs;
        if (d0 + 1 < D) zz[d0 + 1] = rad * sn;
      }
    }
  }
  __syncwarp();
  for (int d = lane; d < D; d += 32) {
    float s = mu[d];
    for (int k = 0; k <= d; ++k) s = fmaf(L[d * D + k], zz[k], s);
    xi0[(size_t)i * D + d] = s;
    if (samples_out) samples_out[(size_t)i * D + d] = s;
  }
}

// r_i = max of the three residuals; c_aug = c_1 + w_r r with
// c_1 = sum_t ||p''||^2 + w_curv c_kappa + w_path c_p on the grid (PRIEST's BARN cost):
// c_kappa = ||p' x p''||^2 / ||p'||^6, the squared curvature (0 below a speed of 1e-3 m/s),
// c_p = distance of p(t) from its projection onto the segment start -> goal of the
// problem (start, goal: FP64 [dim]). One warp per sample: the lanes take the grid
// points t = lane + 32 m and the warp sums their terms (butterfly order).
__global__ void k_cost(const float *xi, const float *res, const float *tables, int tbl_off,
                       int n_p, float invT, float invT2, int dim, int B, float w_r, float w_curv,
                       float w_path, const double *start, const double *goal, float *r_out,
                       float *caug_out) {
  const int i = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= B) return; // whole warps
  const float *tP = tables + tbl_off, *tD = tP + n_p * ROW, *tA = tD + n_p * ROW;
  float sv[3] = {0.f, 0.f, 0.f}, gv[3] = {0.f, 0.f, 0.f};
  for (int a = 0; a < dim; ++a) {
    sv[a] = (float)start[a];
    gv[a] = (float)(goal[a] - start[a]);
  }
  float L2 = 0.f;
  for (int a = 0; a < dim; ++a) L2 = fmaf(gv[a], gv[a], L2);
  float x[3][NC];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int k = 0; k < NC; ++k) x[a][k] = a < dim ? xi[((size_t)i * dim + a) * NC + k] : 0.f;
  float c1 = 0.f;
  for (int t = lane; t < n_p; t += 32) {
    float pos[3] = {0.f, 0.f, 0.f}, vel[3] = {0.f, 0.f, 0.f}, acc[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (a >= dim) break;
      float sp = 0.f, sd = 0.f, sa = 0.f;
#pragma unroll
      for (int k = 0; k < NC; ++k) {
        sp = fmaf(tP[t * ROW + k], x[a][k], sp);
        sd = fmaf(tD[t * ROW + k], x[a][k], sd);
        sa = fmaf(tA[t * ROW + k], x[a][k], sa);
      }
      pos[a] = sp; vel[a] = sd * invT; acc[a] = sa * invT2;
    }
    float a2 = 0.f;
    for (int a = 0; a < dim; ++a) a2 = fmaf(acc[a], acc[a], a2);
    float c = a2;
    if (w_curv != 0.f) {
      const float cx = vel[1] * acc[2] - vel[2] * acc[1], cy = vel[2] * acc[0] - vel[0] * acc[2],
                  cz = vel[0] * acc[1] - vel[1] * acc[0];
      const float v2 = vel[0] * vel[0] + vel[1] * vel[1] + vel[2] * vel[2];
      if (v2 > 1e-6f) c += w_curv * (cx * cx + cy * cy + cz * cz) / (v2 * v2 * v2);
    }
    if (w_path != 0.f) {
      float u = 0.f;
      if (L2 > 0.f) {
        for (int a = 0; a < dim; ++a) u = fmaf(pos[a] - sv[a], gv[a], u);
        u = fminf(fmaxf(u / L2, 0.f), 1.f);
      }
      float d2 = 0.f;
      for (int a = 0; a < dim; ++a) {
        const float d = pos[a] - (sv[a] + u * gv[a]);
        d2 = fmaf(d, d, d2);
      }
      c += w_path * sqrtf(d2);
    }
    c1 += c;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) c1 += __shfl_xor_sync(0xffffffffu, c1, o);
  if (lane == 0) {
    float r = fmaxf(res[i * 3 + 0], fmaxf(res[i * 3 + 1], res[i * 3 + 2]));
    if (!(r == r)) r = __int_as_float(0x7f800000); // NaN ranks last
    r_out[i] = r;
    caug_out[i] = c1 + w_r * r;
  }
}

// Ascending bitonic sort of (key, index) pairs in shared memory; ties by index.
__device__ void bitonic(float *key, int *idx, int n) {
  for (int k = 2; k <= n; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const int p = t ^ j;
        if (p > t) {
          const bool up = (t & k) == 0;
          const float a = key[t], b = key[p];
          const int ia = idx[t], ib = idx[p];
          const bool gt = (a > b) || (a == b && ia > ib);
          if (gt == up) { key[t] = b; key[p] = a; idx[t] = ib; idx[p] = ia; }
        }
      }
      __syncthreads();
    }
}

// Two-stage top-k: the n_proj lowest r, then the n_elite lowest c_aug among them.
// One CTA per group g = blockIdx.x over its B samples (B <= 8192, padded to a power
// of two with +inf keys); indices are local to the group.
__global__ void k_select(const float *r, const float *caug, int B, int n_proj, int n_elite,
                         int *proj_idx, int *elite_idx) {
  extern __shared__ unsigned char sm_raw[];
  r += (size_t)blockIdx.x * B;
  caug += (size_t)blockIdx.x * B;
  proj_idx += (size_t)blockIdx.x * n_proj;
  elite_idx += (size_t)blockIdx.x * n_elite;
  int n = 1;
  while (n < B) n <<= 1;
  float *key = reinterpret_cast<float *>(sm_raw);
  int *idx = reinterpret_cast<int *>(key + n);
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    key[t] = t < B ? r[t] : __int_as_float(0x7f800000);
    idx[t] = t < B ? t : 0x7fffffff;
  }
  __syncthreads();
  bitonic(key, idx, n);
  for (int t = threadIdx.x; t < n_proj; t += blockDim.x) proj_idx[t] = idx[t];
  __syncthreads();
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    const int id = t < n_proj ? proj_idx[t] : 0x7fffffff;
    key[t] = t < n_proj ? caug[id] : __int_as_float(0x7f800000);
    idx[t] = id;
  }
  __syncthreads();
  bitonic(key, idx, n);
  for (int t = threadIdx.x; t < n_elite; t += blockDim.x) elite_idx[t] = idx[t];
}

// Weighted refit (eqs. update_mean, update_covariance) and the best elite. One CTA
// per group g = blockIdx.x of Bg samples. stage: the elites' coefficients are first
// copied to dynamic shared memory ([n_elite][D]), so that the sums over the elites read
// them there (same order of operations either way).
__global__ void k_refit(const float *xi, const float *caug, const int *elite, int Bg, int n_elite,
                        int D, float gamma, float sig, float *mu, float *sigma, float *best,
                        int stage) {
  __shared__ float w_s[8192];
  extern __shared__ float xs[];
  const size_t g = blockIdx.x;
  xi += g * Bg * D;
  caug += g * Bg;
  elite += g * n_elite;
  mu += g * D;
  sigma += g * D * D;
  best += g * (D + 1);
  __shared__ float mu_new[48];
  __shared__ float red[32];
  const float delta = caug[elite[0]];
  float part = 0.f;
  for (int m = threadIdx.x; m < n_elite; m += blockDim.x) {
    const float w = expf(-(caug[elite[m]] - delta) / gamma);
    w_s[m] = w;
    part += w;
  }
  for (int o = 16; o; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
  __syncthreads();
  float S = 0.f;
  for (int k = 0; k < (int)(blockDim.x + 31) / 32; ++k) S += red[k];
  if (stage) {
    for (int e = threadIdx.x; e < n_elite * D; e += blockDim.x)
      xs[e] = xi[(size_t)elite[e / D] * D + e % D];
    __syncthreads();
  }
  for (int d = threadIdx.x; d < D; d += blockDim.x) {
    float s = 0.f;
    for (int m = 0; m < n_elite; ++m)
      s = fmaf(w_s[m], stage ? xs[m * D + d] : xi[(size_t)elite[m] * D + d], s);
    mu_new[d] = (1.f - sig) * mu[d] + sig * (s / S);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < D * D; e += blockDim.x) {
    const int i = e / D, j = e % D;
    float s = 0.f;
    for (int m = 0; m < n_elite; ++m) {
      const float *x = stage ? xs + m * D : xi + (size_t)elite[m] * D;
      s = fmaf(w_s[m] * (x[i] - mu_new[i]), x[j] - mu_new[j], s);
    }
    sigma[e] = (1.f - sig) * sigma[e] + sig * (s / S);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < D; d += blockDim.x) {
    mu[d] = mu_new[d];
    best[d] = xi[(size_t)elite[0] * D + d];
  }
  if (threadIdx.x == 0) best[D] = delta;
}

// c_1 = sum_t ||p''(t)||^2 of every trajectory of a batch (each with its own problem).
__global__ void k_accel_cost(const float *xi, const int *traj_problem, const ProblemDev *problems,
                             const float *tables, int dim, int B, float *out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B) return;
  const ProblemDev pr = problems[traj_problem[i]];
  const float *tA = tables + pr.tbl_off + 2 * pr.n_p * ROW;
  float c1 = 0.f;
  for (int t = 0; t < pr.n_p; ++t) {
    float a2 = 0.f;
    for (int a = 0; a < dim; ++a) {
      float s = 0.f;
      for (int k = 0; k < NC; ++k) s = fmaf(tA[t * ROW + k], xi[((size_t)i * dim + a) * NC + k], s);
      s *= pr.invT2;
      a2 = fmaf(s, s, a2);
    }
    c1 += a2;
  }
  out[i] = c1;
}

cudaError_t launch_accel_cost(const float *xi, const int *traj_problem, const ProblemDev *problems,
                              const float *tables, int dim, int B, float *out, cudaStream_t s) {
  k_accel_cost<<<(B + 127) / 128, 128, 0, s>>>(xi, traj_problem, problems, tables, dim, B, out);
  return cudaGetLastError();
}

cudaError_t launch_sampler_front(const float *mu, const float *sigma, int D, int B, int n_dist,
                                 float eps, const float *z, unsigned long long seed, int iteration,
                                 float *L_scratch, int *flag, float *xi0, float *samples_out,
                                 cudaStream_t s) {
  k_cholesky<<<n_dist, 64, 0, s>>>(sigma, D, eps, L_scratch, flag);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_sample<<<(B + SAMPLE_WARPS - 1) / SAMPLE_WARPS, 32 * SAMPLE_WARPS, 0, s>>>(
      mu, L_scratch, D, B, B / n_dist, z, seed, iteration, xi0, samples_out);
  return cudaGetLastError();
}

cudaError_t launch_sampler_back(const float *xi, const float *res, const float *tables,
                                int tbl_off, int n_p, float invT, float invT2, int dim, int B,
                                int n_dist, const SamplerCost &cost, int n_proj, int n_elite,
                                float gamma, float sig, float *r_out, float *caug_out,
                                int *proj_idx, int *elite_idx, float *mu, float *sigma,
                                float *best, cudaStream_t s) {
  k_cost<<<(unsigned)(((long long)B * 32 + 255) / 256), 256, 0, s>>>(xi, res, tables, tbl_off, n_p,
                                                                     invT, invT2, dim, B,
                                         cost.w_res, cost.w_curv, cost.w_path, cost.start,
                                         cost.goal, r_out, caug_out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int Bg = B / n_dist;
  int n = 1;
  while (n < Bg) n <<= 1;
  const size_t smem = (size_t)n * (sizeof(float) + sizeof(int));
  e = cudaFuncSetAttribute(k_select, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_select<<<n_dist, 1024, smem, s>>>(r_out, caug_out, Bg, n_proj, n_elite, proj_idx, elite_idx);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // the elites' coefficients in shared memory when they fit beside the 32 KB of weights
  const size_t xs_bytes = sizeof(float) * (size_t)n_elite * dim * NC;
  const int stage = xs_bytes <= 160 * 1024 ? 1 : 0;
  if (stage && (e = cudaFuncSetAttribute(k_refit, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)xs_bytes)) != cudaSuccess)
    return e;
  k_refit<<<n_dist, 1024, stage ? xs_bytes : 0, s>>>(xi, caug_out, elite_idx, Bg, n_elite, dim * NC,
                                                     gamma, sig, mu, sigma, best, stage);
  return cudaGetLastError();
}

} // namespace tb

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
//      c_aug among them (exact ranks of the (key, index) pairs, counted over
//      many CTAs);
//   5. weights c_m = exp(-(c_aug,m - delta)/gamma), delta = min c_aug, and the
//      updates of eqs. update_mean and update_covariance (the covariance uses
//      the new mean). The sign of the exponent follows the reading that good
//      samples weigh more.
// Decentralised form (D-PRIEST): the batch splits into n_dist contiguous groups
// of B / n_dist samples, each with its own mean and covariance. The Cholesky and
// refit kernels take one CTA per group and the selections one row of CTAs per
// group, so every stage is one launch for all distributions; the projection solve
// is one launch as before.
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
// Cholesky of Sigma_g + eps I (D x D, D = 11 dim) into L_g (lower, row-major). One
// CTA per distribution g = blockIdx.x.
template <int D>
__global__ void k_cholesky(const float *sigma, float eps, float *L, int *flag) {
  // thread i holds row i in registers (loops unrolled to D, so every index is a
  // constant); the finished entries of each row are published in shared memory for the
  // rows below. The sums run in the column-by-column order of the textbook algorithm.
  __shared__ float Ls[D * D];
  sigma += (size_t)blockIdx.x * D * D;
  L += (size_t)blockIdx.x * D * D;
  const int i = threadIdx.x;
  const bool mine = i < D;
  float row[D];
#pragma unroll
  for (int k = 0; k < D; ++k)
    row[k] = mine ? 0.5f * (sigma[i * D + k] + sigma[k * D + i]) + (i == k ? eps : 0.f) : 0.f;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    if (i == j) {
      float d = row[j];
#pragma unroll
      for (int k = 0; k < j; ++k) d -= row[k] * row[k];
      if (!(d > 0.f)) { atomicOr(flag, 4); d = 1e-30f; }
      row[j] = sqrtf(d);
      Ls[j * D + j] = row[j];
    }
    __syncthreads();
    if (mine && i > j) {
      float s = row[j];
#pragma unroll
      for (int k = 0; k < j; ++k) s -= row[k] * Ls[j * D + k];
      row[j] = s / Ls[j * D + j];
      Ls[i * D + j] = row[j];
    }
    __syncthreads();
  }
  if (mine)
#pragma unroll
    for (int k = 0; k < D; ++k) L[i * D + k] = k <= i ? row[k] : 0.f;
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
constexpr int COST_WARPS = 16;

__global__ void __launch_bounds__(32 * COST_WARPS) k_cost(const float *xi, const float *res,
                                                          const float *tables, int tbl_off,
                                                          int n_p, float invT, float invT2,
                                                          int dim, int B, float w_r,
                                                          float w_curv, float w_path,
                                                          const double *start,
                                                          const double *goal, float *r_out,
                                                          float *caug_out, int stage) {
  // stage: the three basis tables are first copied to shared memory as [3][n_p][NC] (an
  // odd row stride, so that the lanes' different grid points fall in different banks)
  extern __shared__ float tab_s[];
  const float *tab = tables + tbl_off;
  int rs = ROW;
  if (stage) {
    for (int e = threadIdx.x; e < 3 * n_p * NC; e += blockDim.x)
      tab_s[e] = tab[(e / NC) * ROW + e % NC];
    __syncthreads();
    tab = tab_s;
    rs = NC;
  }
  const int i = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= B) return; // whole warps
  const float *tP = tab, *tD = tP + n_p * rs, *tA = tD + n_p * rs;
  float sv[3] = {0.f, 0.f, 0.f}, gv[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int a = 0; a < 3; ++a) if (a < dim) {
    sv[a] = (float)start[a];
    gv[a] = (float)(goal[a] - start[a]);
  }
  float L2 = 0.f;
#pragma unroll
  for (int a = 0; a < 3; ++a) if (a < dim) L2 = fmaf(gv[a], gv[a], L2);
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
        sp = fmaf(tP[t * rs + k], x[a][k], sp);
        sd = fmaf(tD[t * rs + k], x[a][k], sd);
        sa = fmaf(tA[t * rs + k], x[a][k], sa);
      }
      pos[a] = sp; vel[a] = sd * invT; acc[a] = sa * invT2;
    }
    float a2 = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) if (a < dim) a2 = fmaf(acc[a], acc[a], a2);
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
#pragma unroll
        for (int a = 0; a < 3; ++a) if (a < dim) u = fmaf(pos[a] - sv[a], gv[a], u);
        u = fminf(fmaxf(u / L2, 0.f), 1.f);
      }
      float d2 = 0.f;
#pragma unroll
      for (int a = 0; a < 3; ++a) if (a < dim) {
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

// Selection key: an order-preserving map of the float to 32 unsigned bits (-0 taken
// as +0, every NaN above +inf), with the sample index in the low word, so that the
// composites are distinct and their order is the float order with ties broken by the
// lower index.
__device__ __forceinline__ unsigned long long sel_key(float x, int id) {
  unsigned b = __float_as_uint(x);
  if (b == 0x80000000u) b = 0u;
  if ((b & 0x7fffffffu) > 0x7f800000u) b = 0x7fffffffu;
  b ^= (b & 0x80000000u) ? 0xffffffffu : 0x80000000u;
  return ((unsigned long long)b << 32) | (unsigned)id;
}

constexpr int RANK_THREADS = 256;
constexpr int RANK_SLICES = 8;                           // threads counting for one element
constexpr int RANK_ELEMS = RANK_THREADS / RANK_SLICES;  // elements per CTA

// Top-k by rank counting, one stage of ConstraintEliteSet / EliteSet. Group g =
// blockIdx.y has n candidates: candidate e is the sample id = ids[e] (e itself when
// ids is null) with key x[id]. Its rank is the number of candidates whose (key, id)
// comes first; every rank is distinct, and rank < n_out puts id at out[rank], so out
// holds the n_out first candidates in ascending order (the result of sorting the
// pairs). Each CTA stages all n composites of its group in shared memory and ranks
// RANK_ELEMS candidates, RANK_SLICES threads each counting over every
// RANK_SLICES-th composite.
__global__ void __launch_bounds__(RANK_THREADS) k_rank_select(const float *x, int x_stride,
                                                              const int *ids, int ids_stride,
                                                              int n, int n_out, int *out,
                                                              int out_stride) {
  extern __shared__ unsigned long long comp[];
  const int g = blockIdx.y;
  x += (size_t)g * x_stride;
  if (ids) ids += (size_t)g * ids_stride;
  out += (size_t)g * out_stride;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const int id = ids ? ids[e] : e;
    comp[e] = sel_key(x[id], id);
  }
  __syncthreads();
  const int e = blockIdx.x * RANK_ELEMS + threadIdx.x / RANK_SLICES;
  const int sl = threadIdx.x % RANK_SLICES;
  const unsigned long long mine = e < n ? comp[e] : 0ull;
  int c0 = 0, c1 = 0;
  int m = sl;
  for (; m + RANK_SLICES < n; m += 2 * RANK_SLICES) {
    c0 += comp[m] < mine;
    c1 += comp[m + RANK_SLICES] < mine;
  }
  if (m < n) c0 += comp[m] < mine;
  int cnt = c0 + c1;
#pragma unroll
  for (int o = RANK_SLICES / 2; o; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if (sl == 0 && e < n && cnt < n_out) out[cnt] = (int)(unsigned)(mine & 0xffffffffull);
}

// Weighted refit (eqs. update_mean, update_covariance) and the best elite, in two
// kernels. k_refit_mean, one CTA of 1024 threads per group g = blockIdx.x of Bg
// samples: the weights c_m, their sum S, the new mean (aux[g] = [mu_new, S]) and the
// best elite, and for the covariance the elites' centred coefficients xc[m][d] =
// x_m,d - mu_new,d and weighted ones wx[m][d] = c_m xc[m][d], stored contiguously.
// k_refit_cov, a row of CTAs per group: one covariance entry per thread, the sum of
// wx[m][i] xc[m][j] over the elites in order m = 0, 1, ...; the CTA with blockIdx.x
// == 0 then stores mu_new into mu (no other kernel of the step reads mu after
// k_refit_mean). stage: the elites' coefficients are first gathered into dynamic
// shared memory ([n_elite][D]). The operations and their order are those of the
// update equations written out entry by entry, whichever path runs.
constexpr int REFIT_THREADS = 1024;
constexpr int COV_THREADS = 256;
constexpr int GATHER_BATCH = 8;  // gathers in flight per thread

__global__ void __launch_bounds__(REFIT_THREADS) k_refit_mean(const float *xi, const float *caug,
                                                              const int *elite, int Bg,
                                                              int n_elite, int D, int ne_pad,
                                                              float gamma, float sig,
                                                              const float *mu,
                                                              float *best, float *aux,
                                                              float *wx, float *xc, int stage) {
  __shared__ float w_s[8192];
  __shared__ float red[32];
  __shared__ float mu_new[48];
  extern __shared__ float xs[];
  const size_t g = blockIdx.x;
  xi += g * Bg * D;
  caug += g * Bg;
  elite += g * n_elite;
  mu += g * D;
  best += g * (D + 1);
  aux += g * (D + 1);
  wx += g * ne_pad;
  xc += g * ne_pad;
  const int n = n_elite * D;
  if (stage) {  // the gathers of a batch are issued before any is stored
    for (int e0 = threadIdx.x; e0 < n; e0 += GATHER_BATCH * blockDim.x) {
      float v[GATHER_BATCH];
#pragma unroll
      for (int u = 0; u < GATHER_BATCH; ++u) {
        const int e = e0 + u * blockDim.x;
        v[u] = e < n ? __ldg(xi + (size_t)__ldg(elite + e / D) * D + e % D) : 0.f;
      }
#pragma unroll
      for (int u = 0; u < GATHER_BATCH; ++u) {
        const int e = e0 + u * blockDim.x;
        if (e < n) xs[e] = v[u];
      }
    }
  }
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
  for (int d = threadIdx.x; d < D; d += blockDim.x) {
    float s = 0.f;
#pragma unroll 8
    for (int m = 0; m < n_elite; ++m)
      s = fmaf(w_s[m], stage ? xs[m * D + d] : xi[(size_t)elite[m] * D + d], s);
    const float mn = (1.f - sig) * mu[d] + sig * (s / S);
    mu_new[d] = mn;
    aux[d] = mn;
    best[d] = xi[(size_t)elite[0] * D + d];
  }
  if (threadIdx.x == 0) {
    aux[D] = S;
    best[D] = delta;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const int m = e / D, d = e % D;
    const float c = (stage ? xs[e] : xi[(size_t)elite[m] * D + d]) - mu_new[d];
    xc[e] = c;
    wx[e] = w_s[m] * c;
  }
}

__global__ void __launch_bounds__(COV_THREADS) k_refit_cov(int n_elite, int D, int ne_pad,
                                                           float sig,
                                                           const float *__restrict__ wx,
                                                           const float *__restrict__ xc,
                                                           const float *aux, float *mu,
                                                           float *sigma, int stage) {
  extern __shared__ float4 cov_s[];  // [wx | xc], ne_pad floats each
  const size_t g = blockIdx.y;
  wx += g * ne_pad;
  xc += g * ne_pad;
  aux += g * (D + 1);
  mu += g * D;
  sigma += g * D * D;
  const float *w_src = wx, *x_src = xc;
  if (stage) {  // 16-byte loads, a batch of them issued before any is stored
    const int n4 = ne_pad / 4;
    const float4 *src0 = reinterpret_cast<const float4 *>(wx);
    const float4 *src1 = reinterpret_cast<const float4 *>(xc);
    for (int q0 = threadIdx.x; q0 < 2 * n4; q0 += GATHER_BATCH * blockDim.x) {
      float4 v[GATHER_BATCH];
#pragma unroll
      for (int u = 0; u < GATHER_BATCH; ++u) {
        const int q = q0 + u * blockDim.x;
        v[u] = q < n4 ? __ldg(src0 + q) : q < 2 * n4 ? __ldg(src1 + (q - n4)) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < GATHER_BATCH; ++u) {
        const int q = q0 + u * blockDim.x;
        if (q < 2 * n4) cov_s[q] = v[u];
      }
    }
    __syncthreads();
    w_src = reinterpret_cast<const float *>(cov_s);
    x_src = w_src + ne_pad;
  }
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < D * D) {
    const int i = e / D, j = e % D;
    float s = 0.f;
#pragma unroll 8
    for (int m = 0; m < n_elite; ++m) s = fmaf(w_src[m * D + i], x_src[m * D + j], s);
    sigma[e] = (1.f - sig) * sigma[e] + sig * (s / aux[D]);
  }
  if (blockIdx.x == 0)
    for (int d = threadIdx.x; d < D; d += blockDim.x) mu[d] = aux[d];
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
  if (D == 2 * NC) k_cholesky<2 * NC><<<n_dist, 64, 0, s>>>(sigma, eps, L_scratch, flag);
  else if (D == 3 * NC) k_cholesky<3 * NC><<<n_dist, 64, 0, s>>>(sigma, eps, L_scratch, flag);
  else return cudaErrorInvalidValue;
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
                                int *proj_idx, int *elite_idx, float *refit_scratch, float *mu,
                                float *sigma, float *best, cudaStream_t s) {
  const size_t tab_bytes = sizeof(float) * 3 * (size_t)n_p * NC;
  const int tab_stage = tab_bytes <= 160 * 1024 ? 1 : 0;
  cudaError_t e = cudaSuccess;
  if (tab_stage && (e = cudaFuncSetAttribute(k_cost, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)tab_bytes)) != cudaSuccess)
    return e;
  k_cost<<<(B + COST_WARPS - 1) / COST_WARPS, 32 * COST_WARPS, tab_stage ? tab_bytes : 0, s>>>(
      xi, res, tables, tbl_off, n_p, invT, invT2, dim, B, cost.w_res, cost.w_curv, cost.w_path,
      cost.start, cost.goal, r_out, caug_out, tab_stage);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int Bg = B / n_dist;
  // ConstraintEliteSet: the n_proj lowest r of each group; EliteSet: the n_elite
  // lowest c_aug among them
  e = cudaFuncSetAttribute(k_rank_select, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(sizeof(unsigned long long) * Bg));
  if (e != cudaSuccess) return e;
  k_rank_select<<<dim3((Bg + RANK_ELEMS - 1) / RANK_ELEMS, n_dist), RANK_THREADS,
                  sizeof(unsigned long long) * Bg, s>>>(r_out, Bg, nullptr, 0, Bg, n_proj,
                                                        proj_idx, n_proj);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_rank_select<<<dim3((n_proj + RANK_ELEMS - 1) / RANK_ELEMS, n_dist), RANK_THREADS,
                  sizeof(unsigned long long) * n_proj, s>>>(caug_out, Bg, proj_idx, n_proj,
                                                            n_proj, n_elite, elite_idx, n_elite);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // the elites' coefficients in shared memory when they fit beside the 32 KB of weights
  const int D = dim * NC;
  const size_t xs_bytes = sizeof(float) * (size_t)n_elite * D;
  const int stage = xs_bytes <= 160 * 1024 ? 1 : 0;
  if (stage && (e = cudaFuncSetAttribute(k_refit_mean, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)xs_bytes)) != cudaSuccess)
    return e;
  // per group, n_elite * D weighted and centred coefficients rounded up to a multiple of
  // 4 floats, so that every group's arrays start on a 16-byte boundary
  const int ne_pad = (n_elite * D + 3) & ~3;
  float *wx = refit_scratch, *xc = wx + (size_t)n_dist * ne_pad;
  float *aux = xc + (size_t)n_dist * ne_pad;
  k_refit_mean<<<n_dist, REFIT_THREADS, stage ? xs_bytes : 0, s>>>(
      xi, caug_out, elite_idx, Bg, n_elite, D, ne_pad, gamma, sig, mu, best, aux, wx, xc, stage);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const size_t cov_bytes = sizeof(float) * 2 * (size_t)ne_pad;
  const int cov_stage = cov_bytes <= 200 * 1024 ? 1 : 0;
  if (cov_stage && (e = cudaFuncSetAttribute(k_refit_cov, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)cov_bytes)) != cudaSuccess)
    return e;
  k_refit_cov<<<dim3((D * D + COV_THREADS - 1) / COV_THREADS, n_dist), COV_THREADS,
                cov_stage ? cov_bytes : 0, s>>>(n_elite, D, ne_pad, sig, wx, xc, aux, mu, sigma,
                                                cov_stage);
  return cudaGetLastError();
}

} // namespace tb

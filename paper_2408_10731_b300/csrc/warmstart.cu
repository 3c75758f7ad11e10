// warmstart.cu -- the learned warm start: an MLP from start, goal and the 64
// obstacles nearest to the start->goal segment to K = 8 proposal coefficient
// sets (offsets from the straight-line coefficients). The thesis lists
// learning-based methods as future work; the network, its features and its
// loss are this library's own design.
//
//   388 -> 256 -> 256 -> 256 -> 176, GELU (tanh form), BF16 weights and
//   activations on the tcgen05 tensor cores, FP32 accumulation, FP32 master
//   weights with AdamW. Loss (multiple choice / winner-takes-all): for every
//   solved label m of a scene, min_k ||y_k - t_m||^2 + 0.05 * mean_k ||y_k - t_m||^2,
//   averaged over the labels of the batch.
#include "trajbatch.h"
#include "internal.cuh"
#include "gelu.cuh"
#include "nvtx_range.h"

#include <cuda_bf16.h>
#include <math.h>
#include <string>
#include <vector>

namespace tb {
void set_thread_error(const std::string &msg);
}
using namespace tb;

namespace {

constexpr int IN = 388, IN_PAD = 400, HID = 256, OUT = 176, HEADS = 8, D22 = 22, NEAR = 64;
constexpr int MAX_OBS_PER_SCENE = 1024;
static_assert(IN == 4 + 6 * NEAR, "features: 4 start/goal inputs + 6 per nearest obstacle");

// padded flat parameter layout on the device (W1 padded to 400 columns)
constexpr int P_W1 = 0, P_B1 = P_W1 + HID * IN_PAD, P_W2 = P_B1 + HID, P_B2 = P_W2 + HID * HID,
              P_W3 = P_B2 + HID, P_B3 = P_W3 + HID * HID, P_W4 = P_B3 + HID,
              P_B4 = P_W4 + OUT * HID, P_TOTAL = P_B4 + OUT;
// public (unpadded) flat layout
constexpr int U_W1 = 0, U_B1 = U_W1 + HID * IN, U_W2 = U_B1 + HID, U_TOTAL = U_W2 + (P_TOTAL - P_W2);

// ---- features -----------------------------------------------------------------
// n_obs bounds the obstacle arrays: a scene whose offsets leave [0, n_obs] (or
// decrease) is treated as obstacle-free and raises bit 1 of *err.
__global__ void k_features(const double *start, const double *goal, const int *offsets,
                           int n_obs, const float *cen, const float *ax, const float *vel,
                           __nv_bfloat16 *X, float *line, int *err) {
  __shared__ float key[MAX_OBS_PER_SCENE];
  __shared__ int idx[MAX_OBS_PER_SCENE];
  const int s = blockIdx.x;
  int o0 = offsets[s], o1 = offsets[s + 1];
  if (o0 < 0 || o1 < o0 || o1 > n_obs) {
    if (threadIdx.x == 0) atomicOr(err, 2);
    o0 = o1 = 0;
  }
  const int n = min(o1 - o0, MAX_OBS_PER_SCENE);
  int np2 = NEAR; // the sort covers at least the NEAR slots of the features
  while (np2 < n) np2 <<= 1;
  const float sx = (float)start[2 * s], sy = (float)start[2 * s + 1];
  const float gx = (float)goal[2 * s] - sx, gy = (float)goal[2 * s + 1] - sy;
  const float L2 = gx * gx + gy * gy;
  for (int t = threadIdx.x; t < np2; t += blockDim.x) {
    float d = __int_as_float(0x7f800000);
    if (t < n) { // distance of the t = 0 centre to the start->goal segment
      const float px = cen[2 * (o0 + t)] - sx, py = cen[2 * (o0 + t) + 1] - sy;
      float u = L2 > 0.f ? (px * gx + py * gy) / L2 : 0.f;
      u = fminf(fmaxf(u, 0.f), 1.f);
      const float ex = px - u * gx, ey = py - u * gy;
      d = sqrtf(ex * ex + ey * ey);
    }
    key[t] = d;
    idx[t] = t;
  }
  __syncthreads();
  for (int k = 2; k <= np2; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < np2; t += blockDim.x) {
        const int p = t ^ j;
        if (p > t) {
          const bool up = (t & k) == 0;
          const float a = key[t], b = key[p];
          const int ia = idx[t], ib = idx[p];
          if (((a > b) || (a == b && ia > ib)) == up) { key[t] = b; key[p] = a; idx[t] = ib; idx[p] = ia; }
        }
      }
      __syncthreads();
    }
  __nv_bfloat16 *row = X + (size_t)s * IN_PAD;
  for (int f = threadIdx.x; f < IN_PAD; f += blockDim.x) {
    float v = 0.f;
    if (f == 2) v = 0.1f * gx;
    else if (f == 3) v = 0.1f * gy;
    else if (f >= 4 && f < IN) {
      const int slot = (f - 4) / 6, c = (f - 4) % 6;
      if (slot < n) {
        const int o = o0 + idx[slot];
        v = c == 0 ? 0.1f * (cen[2 * o] - sx) : c == 1 ? 0.1f * (cen[2 * o + 1] - sy)
          : c == 2 ? ax[2 * o] : c == 3 ? ax[2 * o + 1] : c == 4 ? vel[2 * o] : vel[2 * o + 1];
      }
    }
    row[f] = __float2bfloat16_rn(v);
  }
  for (int f = threadIdx.x; f < D22; f += blockDim.x) {
    const int a = f / NC, i = f % NC;
    const double s0 = start[2 * s + a], g0 = goal[2 * s + a];
    line[(size_t)s * D22 + f] = (float)(s0 + (g0 - s0) * (double)i / (double)(NC - 1));
  }
}

// ---- small helpers --------------------------------------------------------------
__global__ void k_transpose_bf16(const __nv_bfloat16 *in, __nv_bfloat16 *out, int R, int C) {
  __shared__ __nv_bfloat16 tile[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int r = r0 + j, c = c0 + threadIdx.x;
    tile[j][threadIdx.x] = (r < R && c < C) ? in[(size_t)r * C + c] : __float2bfloat16_rn(0.f);
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int c = c0 + j, r = r0 + threadIdx.x;
    if (c < C && r < R) out[(size_t)c * R + r] = tile[threadIdx.x][j];
  }
}

template <typename T>
__global__ void k_colsum(const T *in, int R, int C, float *out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  float s = 0.f;
  for (int r = 0; r < R; ++r) s += (float)in[(size_t)r * C + c];
  out[c] = s;
}

__global__ void k_count_labels(const int *n_labels, int R, float *total) {
  __shared__ float red[32];
  float s = 0.f;
  for (int r = threadIdx.x; r < R; r += blockDim.x) s += (float)n_labels[r];
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < (int)blockDim.x / 32; ++w) t += red[w];
    *total = t;
  }
}

// winner-takes-all loss and its gradient with respect to Y
__global__ void k_loss_wta(const float *Y, const float *targets, const int *n_labels, int R,
                           const float *total, float *dYf, __nv_bfloat16 *dYb, float *loss) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  float ls = 0.f;
  if (s < R) {
    const float inv = 1.f / fmaxf(*total, 1.f);
    float g[OUT];
    for (int q = 0; q < OUT; ++q) g[q] = 0.f;
    const float *y = Y + (size_t)s * OUT;
    const int nl = n_labels[s];
    for (int m = 0; m < nl; ++m) {
      const float *t = targets + ((size_t)s * HEADS + m) * D22;
      float d[HEADS];
      int kmin = 0;
      for (int k = 0; k < HEADS; ++k) {
        float acc = 0.f;
        for (int q = 0; q < D22; ++q) { const float e = y[k * D22 + q] - t[q]; acc = fmaf(e, e, acc); }
        d[k] = acc;
        if (acc < d[kmin]) kmin = k;
      }
      float mean = 0.f;
      for (int k = 0; k < HEADS; ++k) mean += d[k];
      ls += d[kmin] + 0.05f * mean / HEADS;
      for (int k = 0; k < HEADS; ++k) {
        const float coef = 2.f * ((k == kmin ? 1.f : 0.f) + 0.05f / HEADS) * inv;
        for (int q = 0; q < D22; ++q) g[k * D22 + q] += coef * (y[k * D22 + q] - t[q]);
      }
    }
    for (int q = 0; q < OUT; ++q) {
      dYf[(size_t)s * OUT + q] = g[q];
      dYb[(size_t)s * OUT + q] = __float2bfloat16_rn(g[q]);
    }
    ls *= inv;
  }
  for (int o = 16; o; o >>= 1) ls += __shfl_xor_sync(0xffffffffu, ls, o);
  if ((threadIdx.x & 31) == 0 && ls != 0.f) atomicAdd(loss, ls);
}

// AdamW (decoupled weight decay on the weight matrices, not on the biases), then
// the BF16 copies of every weight matrix and the transposes of layers 2-4.
__global__ void k_adamw(float *W, float *m, float *v, const float *g, int n, float lr, float b1,
                        float b2, float eps, float wd, float bc1, float bc2,
                        __nv_bfloat16 *W1b, __nv_bfloat16 *W2b, __nv_bfloat16 *W3b,
                        __nv_bfloat16 *W4b, __nv_bfloat16 *W2t, __nv_bfloat16 *W3t,
                        __nv_bfloat16 *W4t, int update) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const bool is_w = (i < P_B1) || (i >= P_W2 && i < P_B2) || (i >= P_W3 && i < P_B3) ||
                    (i >= P_W4 && i < P_B4);
  float w = W[i];
  if (update) {
    if (i < P_B1 && (i % IN_PAD) >= IN) { // padding columns of W1 stay zero
      w = 0.f;
    } else {
      const float gi = g[i];
      const float mi = b1 * m[i] + (1.f - b1) * gi;
      const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
      m[i] = mi; v[i] = vi;
      if (is_w) w -= lr * wd * w;
      w -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    }
    W[i] = w;
  }
  const __nv_bfloat16 wb = __float2bfloat16_rn(w);
  if (i < P_B1) W1b[i] = wb;
  else if (i >= P_W2 && i < P_B2) { const int k = i - P_W2; W2b[k] = wb; W2t[(k % HID) * HID + k / HID] = wb; }
  else if (i >= P_W3 && i < P_B3) { const int k = i - P_W3; W3b[k] = wb; W3t[(k % HID) * HID + k / HID] = wb; }
  else if (i >= P_W4 && i < P_B4) { const int k = i - P_W4; W4b[k] = wb; W4t[(k % HID) * OUT + k / HID] = wb; }
}

__global__ void k_proposals(const float *Y, const float *line, int R, float *out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= R * OUT) return;
  const int s = e / OUT, q = e % OUT;
  out[e] = Y[e] + line[(size_t)s * D22 + (q % D22)];
}

// ---- FP32-operand debug path ------------------------------------------------------
// C[m][n] = sum_k A(m, k) B(n, k) with every operand FP32 on the CUDA cores, the
// operands addressed through strides (A(m, k) = A[m sAm + k sAk], likewise B) so
// that the backward pass needs no transposed copies. Epilogues as the tensor-core
// GEMM's, in FP32: 0 store; 1 Z = C + bias and H = GELU(Z); 2 C + bias; 3
// C * GELU'(aux). 32 x 32 output tiles, K staged through shared memory in steps of 32.
struct F32Gemm {
  int M, N, K;
  const float *A; long long sAm, sAk;
  const float *B; long long sBn, sBk;
  float *C; int ldc;
  int epi;
  const float *bias, *aux; // aux [M][ldc]
  float *H;                // epilogue 1: GELU(Z) [M][ldc]
};

__global__ void k_gemm_f32(F32Gemm g) {
  __shared__ float As[32][33], Bs[32][33];
  const int tx = threadIdx.x, ty = threadIdx.y; // 32 x 8 threads, 4 rows each
  const int m0 = blockIdx.y * 32, n0 = blockIdx.x * 32;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int k0 = 0; k0 < g.K; k0 += 32) {
    for (int r = ty; r < 32; r += 8) {
      const int m = m0 + r, n = n0 + r, k = k0 + tx;
      As[r][tx] = (m < g.M && k < g.K) ? g.A[m * g.sAm + k * g.sAk] : 0.f;
      Bs[r][tx] = (n < g.N && k < g.K) ? g.B[n * g.sBn + k * g.sBk] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < 32; ++k) {
      const float b = Bs[tx][k];
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[i] = fmaf(As[ty + 8 * i][k], b, acc[i]);
    }
    __syncthreads();
  }
  const int n = n0 + tx;
  if (n >= g.N) return;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty + 8 * i;
    if (m >= g.M) continue;
    const size_t o = (size_t)m * g.ldc + n;
    float v = acc[i];
    if (g.epi == 1 || g.epi == 2) v += g.bias[n];
    if (g.epi == 3) v *= gelu_tanh_grad(g.aux[o]);
    g.C[o] = v;
    if (g.epi == 1) g.H[o] = gelu_tanh(v);
  }
}

__global__ void k_bf16_to_f32(const __nv_bfloat16 *in, float *out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = __bfloat162float(in[i]);
}

// padded <-> public parameter layouts (W1 rows 400 <-> 388)
__global__ void k_params_pad(const float *u, float *p, int to_padded) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P_TOTAL) return;
  if (i < P_B1) {
    const int r = i / IN_PAD, c = i % IN_PAD;
    if (to_padded) p[i] = c < IN ? u[r * IN + c] : 0.f;
    else if (c < IN) p[r * IN + c] = u[i]; // here u is the padded source, p the public one
  } else {
    const int k = i - P_B1 + U_B1;
    if (to_padded) p[i] = u[k];
    else p[k] = u[i];
  }
}

} // namespace

struct traj_warmstart {
  cudaStream_t stream = nullptr;
  int max_rows = 0;
  int step = 0;
  std::vector<void *> allocs;
  float *W = nullptr, *m = nullptr, *v = nullptr, *g = nullptr;
  __nv_bfloat16 *W1b, *W2b, *W3b, *W4b, *W2t, *W3t, *W4t;
  __nv_bfloat16 *Xt, *H1, *H2, *H3, *H1t, *H2t, *H3t, *dYb, *dYt, *dZ1, *dZ2, *dZ3, *dZ1t, *dZ2t, *dZ3t;
  float *Z1, *Z2, *Z3, *Y, *dYf, *total, *loss_tmp, *stage;
  // FP32-operand debug path (allocated on its first use): features, activations and
  // their gradients in FP32
  float *f_X = nullptr, *f_H1, *f_H2, *f_H3, *f_dZ1, *f_dZ2, *f_dZ3;
  double *d_start = nullptr, *d_goal = nullptr;
  int *d_offsets = nullptr, *err = nullptr;
  int feat_cap = 0;
};

namespace {

template <class T> bool ws_alloc(traj_warmstart *w, T **p, size_t n) {
  void *q = nullptr;
  if (cudaMalloc(&q, sizeof(T) * (n ? n : 1)) != cudaSuccess) return false;
  w->allocs.push_back(q);
  *p = static_cast<T *>(q);
  return true;
}

traj_status ws_fail(traj_status s, const std::string &m) {
  set_thread_error(m);
  return s;
}

#define WS_CK(expr)                                                                   \
  do {                                                                                \
    cudaError_t _e = (expr);                                                          \
    if (_e != cudaSuccess) return ws_fail(TRAJ_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
  } while (0)

cudaError_t transpose(const __nv_bfloat16 *in, __nv_bfloat16 *out, int R, int C, cudaStream_t s) {
  dim3 grid((C + 31) / 32, (R + 31) / 32), block(32, 8);
  k_transpose_bf16<<<grid, block, 0, s>>>(in, out, R, C);
  return cudaGetLastError();
}

cudaError_t refresh_bf16(traj_warmstart *w, int update, float lr, float wd) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const int t = w->step;
  const float bc1 = update ? 1.f - powf(b1, (float)t) : 1.f, bc2 = update ? 1.f - powf(b2, (float)t) : 1.f;
  k_adamw<<<(P_TOTAL + 255) / 256, 256, 0, w->stream>>>(w->W, w->m, w->v, w->g, P_TOTAL, lr, b1, b2, eps, wd,
                                                         bc1, bc2, w->W1b, w->W2b, w->W3b, w->W4b, w->W2t,
                                                         w->W3t, w->W4t, update);
  return cudaGetLastError();
}

// forward of `rows` feature rows (X bf16 [rows][400]) -> Y f32 [rows][176]
cudaError_t forward(traj_warmstart *w, int rows, const void *X) {
  cudaStream_t s = w->stream;
  cudaError_t e;
  if ((e = launch_gemm_bf16(1, X, w->W1b, rows, HID, IN_PAD, w->Z1, w->H1, HID, w->W + P_B1, nullptr, w->err, s))) return e;
  if ((e = launch_gemm_bf16(1, w->H1, w->W2b, rows, HID, HID, w->Z2, w->H2, HID, w->W + P_B2, nullptr, w->err, s))) return e;
  if ((e = launch_gemm_bf16(1, w->H2, w->W3b, rows, HID, HID, w->Z3, w->H3, HID, w->W + P_B3, nullptr, w->err, s))) return e;
  return launch_gemm_bf16(2, w->H3, w->W4b, rows, OUT, HID, w->Y, nullptr, OUT, w->W + P_B4, nullptr, w->err, s);
}

// loss and parameter gradients (padded layout) of one batch
cudaError_t backward(traj_warmstart *w, int R, const void *X, const float *targets,
                     const int *n_labels, float *loss) {
  cudaStream_t s = w->stream;
  cudaError_t e;
  if ((e = forward(w, R, X))) return e;
  if ((e = cudaMemsetAsync(loss, 0, sizeof(float), s))) return e;
  k_count_labels<<<1, 1024, 0, s>>>(n_labels, R, w->total);
  k_loss_wta<<<(R + 127) / 128, 128, 0, s>>>(w->Y, targets, n_labels, R, w->total, w->dYf, w->dYb, loss);
  if ((e = cudaGetLastError())) return e;
  float *g = w->g;
  // layer 4
  if ((e = transpose(w->dYb, w->dYt, R, OUT, s)) || (e = transpose(w->H3, w->H3t, R, HID, s))) return e;
  if ((e = launch_gemm_bf16(0, w->dYt, w->H3t, OUT, HID, R, g + P_W4, nullptr, HID, nullptr, nullptr, w->err, s))) return e;
  k_colsum<float><<<(OUT + 127) / 128, 128, 0, s>>>(w->dYf, R, OUT, g + P_B4);
  if ((e = launch_gemm_bf16(3, w->dYb, w->W4t, R, HID, OUT, nullptr, w->dZ3, HID, nullptr, w->Z3, w->err, s))) return e;
  // layer 3
  if ((e = transpose(w->dZ3, w->dZ3t, R, HID, s)) || (e = transpose(w->H2, w->H2t, R, HID, s))) return e;
  if ((e = launch_gemm_bf16(0, w->dZ3t, w->H2t, HID, HID, R, g + P_W3, nullptr, HID, nullptr, nullptr, w->err, s))) return e;
  k_colsum<__nv_bfloat16><<<(HID + 127) / 128, 128, 0, s>>>(w->dZ3, R, HID, g + P_B3);
  if ((e = launch_gemm_bf16(3, w->dZ3, w->W3t, R, HID, HID, nullptr, w->dZ2, HID, nullptr, w->Z2, w->err, s))) return e;
  // layer 2
  if ((e = transpose(w->dZ2, w->dZ2t, R, HID, s)) || (e = transpose(w->H1, w->H1t, R, HID, s))) return e;
  if ((e = launch_gemm_bf16(0, w->dZ2t, w->H1t, HID, HID, R, g + P_W2, nullptr, HID, nullptr, nullptr, w->err, s))) return e;
  k_colsum<__nv_bfloat16><<<(HID + 127) / 128, 128, 0, s>>>(w->dZ2, R, HID, g + P_B2);
  if ((e = launch_gemm_bf16(3, w->dZ2, w->W2t, R, HID, HID, nullptr, w->dZ1, HID, nullptr, w->Z1, w->err, s))) return e;
  // layer 1
  if ((e = transpose(w->dZ1, w->dZ1t, R, HID, s)) ||
      (e = transpose(reinterpret_cast<const __nv_bfloat16 *>(X), w->Xt, R, IN_PAD, s))) return e;
  if ((e = launch_gemm_bf16(0, w->dZ1t, w->Xt, HID, IN_PAD, R, g + P_W1, nullptr, IN_PAD, nullptr, nullptr, w->err, s))) return e;
  k_colsum<__nv_bfloat16><<<(HID + 127) / 128, 128, 0, s>>>(w->dZ1, R, HID, g + P_B1);
  return cudaGetLastError();
}

cudaError_t gemm_f32(cudaStream_t s, int M, int N, int K, const float *A, long long sAm,
                     long long sAk, const float *B, long long sBn, long long sBk, float *C, int ldc,
                     int epi, const float *bias = nullptr, const float *aux = nullptr,
                     float *H = nullptr) {
  F32Gemm g{M, N, K, A, sAm, sAk, B, sBn, sBk, C, ldc, epi, bias, aux, H};
  dim3 grid((N + 31) / 32, (M + 31) / 32), block(32, 8);
  k_gemm_f32<<<grid, block, 0, s>>>(g);
  return cudaGetLastError();
}

// The loss and parameter gradients of one batch with every GEMM operand in FP32 (the
// debug instantiation of backward(): same layers, loss and order, FP32 throughout).
cudaError_t backward_f32(traj_warmstart *w, int R, const void *X, const float *targets,
                         const int *n_labels, float *loss) {
  cudaStream_t s = w->stream;
  cudaError_t e;
  const float *W = w->W;
  float *g = w->g;
  k_bf16_to_f32<<<(R * IN_PAD + 255) / 256, 256, 0, s>>>(reinterpret_cast<const __nv_bfloat16 *>(X),
                                                         w->f_X, R * IN_PAD);
  // forward: Z = H W^T + b, H' = GELU(Z); Y = H3 W4^T + b4
  if ((e = gemm_f32(s, R, HID, IN_PAD, w->f_X, IN_PAD, 1, W + P_W1, IN_PAD, 1, w->Z1, HID, 1, W + P_B1,
                    nullptr, w->f_H1))) return e;
  if ((e = gemm_f32(s, R, HID, HID, w->f_H1, HID, 1, W + P_W2, HID, 1, w->Z2, HID, 1, W + P_B2,
                    nullptr, w->f_H2))) return e;
  if ((e = gemm_f32(s, R, HID, HID, w->f_H2, HID, 1, W + P_W3, HID, 1, w->Z3, HID, 1, W + P_B3,
                    nullptr, w->f_H3))) return e;
  if ((e = gemm_f32(s, R, OUT, HID, w->f_H3, HID, 1, W + P_W4, HID, 1, w->Y, OUT, 2, W + P_B4))) return e;
  if ((e = cudaMemsetAsync(loss, 0, sizeof(float), s))) return e;
  k_count_labels<<<1, 1024, 0, s>>>(n_labels, R, w->total);
  k_loss_wta<<<(R + 127) / 128, 128, 0, s>>>(w->Y, targets, n_labels, R, w->total, w->dYf, w->dYb, loss);
  if ((e = cudaGetLastError())) return e;
  // layer 4: dW4 = dY^T H3, db4 = colsum dY, dZ3 = (dY W4) GELU'(Z3)
  if ((e = gemm_f32(s, OUT, HID, R, w->dYf, 1, OUT, w->f_H3, 1, HID, g + P_W4, HID, 0))) return e;
  k_colsum<float><<<(OUT + 127) / 128, 128, 0, s>>>(w->dYf, R, OUT, g + P_B4);
  if ((e = gemm_f32(s, R, HID, OUT, w->dYf, OUT, 1, W + P_W4, 1, HID, w->f_dZ3, HID, 3, nullptr,
                    w->Z3))) return e;
  // layer 3
  if ((e = gemm_f32(s, HID, HID, R, w->f_dZ3, 1, HID, w->f_H2, 1, HID, g + P_W3, HID, 0))) return e;
  k_colsum<float><<<(HID + 127) / 128, 128, 0, s>>>(w->f_dZ3, R, HID, g + P_B3);
  if ((e = gemm_f32(s, R, HID, HID, w->f_dZ3, HID, 1, W + P_W3, 1, HID, w->f_dZ2, HID, 3, nullptr,
                    w->Z2))) return e;
  // layer 2
  if ((e = gemm_f32(s, HID, HID, R, w->f_dZ2, 1, HID, w->f_H1, 1, HID, g + P_W2, HID, 0))) return e;
  k_colsum<float><<<(HID + 127) / 128, 128, 0, s>>>(w->f_dZ2, R, HID, g + P_B2);
  if ((e = gemm_f32(s, R, HID, HID, w->f_dZ2, HID, 1, W + P_W2, 1, HID, w->f_dZ1, HID, 3, nullptr,
                    w->Z1))) return e;
  // layer 1 (the padding columns of W1 get the features' zero columns: zero gradient)
  if ((e = gemm_f32(s, HID, IN_PAD, R, w->f_dZ1, 1, HID, w->f_X, 1, IN_PAD, g + P_W1, IN_PAD, 0))) return e;
  k_colsum<float><<<(HID + 127) / 128, 128, 0, s>>>(w->f_dZ1, R, HID, g + P_B1);
  return cudaGetLastError();
}

traj_status check_rows(traj_warmstart *w, int rows) {
  if (rows < 8 || rows > w->max_rows || (rows % 8) != 0)
    return ws_fail(TRAJ_ESHAPE, "rows must be a multiple of 8 in [8, max_rows]");
  return TRAJ_OK;
}

} // namespace

extern "C" {

int traj_warmstart_num_params(void) { return U_TOTAL; }

traj_status traj_warmstart_create(int max_rows, void *cuda_stream, traj_warmstart **out) {
  set_thread_error("");
  if (!out || max_rows < 8 || (max_rows % 8) != 0) return ws_fail(TRAJ_EINVAL, "max_rows must be a positive multiple of 8");
  traj_warmstart *w = new (std::nothrow) traj_warmstart();
  if (!w) return TRAJ_ENOMEM;
  w->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  w->max_rows = max_rows;
  const size_t R = max_rows;
  bool ok = ws_alloc(w, &w->W, P_TOTAL) && ws_alloc(w, &w->m, P_TOTAL) && ws_alloc(w, &w->v, P_TOTAL) &&
            ws_alloc(w, &w->g, P_TOTAL) && ws_alloc(w, &w->W1b, HID * IN_PAD) &&
            ws_alloc(w, &w->W2b, HID * HID) && ws_alloc(w, &w->W3b, HID * HID) &&
            ws_alloc(w, &w->W4b, OUT * HID) && ws_alloc(w, &w->W2t, HID * HID) &&
            ws_alloc(w, &w->W3t, HID * HID) && ws_alloc(w, &w->W4t, HID * OUT) &&
            ws_alloc(w, &w->Xt, IN_PAD * R) && ws_alloc(w, &w->H1, R * HID) && ws_alloc(w, &w->H2, R * HID) &&
            ws_alloc(w, &w->H3, R * HID) && ws_alloc(w, &w->H1t, R * HID) && ws_alloc(w, &w->H2t, R * HID) &&
            ws_alloc(w, &w->H3t, R * HID) && ws_alloc(w, &w->dYb, R * OUT) && ws_alloc(w, &w->dYt, R * OUT) &&
            ws_alloc(w, &w->dZ1, R * HID) && ws_alloc(w, &w->dZ2, R * HID) && ws_alloc(w, &w->dZ3, R * HID) &&
            ws_alloc(w, &w->dZ1t, R * HID) && ws_alloc(w, &w->dZ2t, R * HID) && ws_alloc(w, &w->dZ3t, R * HID) &&
            ws_alloc(w, &w->Z1, R * HID) && ws_alloc(w, &w->Z2, R * HID) && ws_alloc(w, &w->Z3, R * HID) &&
            ws_alloc(w, &w->Y, R * OUT) && ws_alloc(w, &w->dYf, R * OUT) && ws_alloc(w, &w->total, 1) &&
            ws_alloc(w, &w->loss_tmp, 1) && ws_alloc(w, &w->err, 1) && ws_alloc(w, &w->stage, U_TOTAL);
  if (!ok) {
    for (void *p : w->allocs) cudaFree(p);
    delete w;
    return ws_fail(TRAJ_ENOMEM, "cudaMalloc failed");
  }
  cudaMemsetAsync(w->W, 0, sizeof(float) * P_TOTAL, w->stream);
  cudaMemsetAsync(w->m, 0, sizeof(float) * P_TOTAL, w->stream);
  cudaMemsetAsync(w->v, 0, sizeof(float) * P_TOTAL, w->stream);
  cudaMemsetAsync(w->g, 0, sizeof(float) * P_TOTAL, w->stream);
  cudaMemsetAsync(w->err, 0, sizeof(int), w->stream);
  *out = w;
  return TRAJ_OK;
}

traj_status traj_warmstart_destroy(traj_warmstart *w) {
  if (!w) return TRAJ_OK;
  cudaStreamSynchronize(w->stream);
  for (void *p : w->allocs) cudaFree(p);
  if (w->d_start) { cudaFree(w->d_start); cudaFree(w->d_goal); cudaFree(w->d_offsets); }
  delete w;
  return TRAJ_OK;
}

traj_status traj_warmstart_set_params(traj_warmstart *w, const float *params) {
  if (!w || !params) return TRAJ_EINVAL;
  WS_CK(cudaMemcpyAsync(w->stage, params, sizeof(float) * U_TOTAL, cudaMemcpyDefault, w->stream));
  k_params_pad<<<(P_TOTAL + 255) / 256, 256, 0, w->stream>>>(w->stage, w->W, 1);
  WS_CK(cudaGetLastError());
  WS_CK(cudaMemsetAsync(w->m, 0, sizeof(float) * P_TOTAL, w->stream));
  WS_CK(cudaMemsetAsync(w->v, 0, sizeof(float) * P_TOTAL, w->stream));
  w->step = 0;
  WS_CK(refresh_bf16(w, 0, 0.f, 0.f));
  WS_CK(cudaStreamSynchronize(w->stream)); // the caller may reuse a host source at once
  return TRAJ_OK;
}

traj_status traj_warmstart_get_params(traj_warmstart *w, float *params) {
  if (!w || !params) return TRAJ_EINVAL;
  k_params_pad<<<(P_TOTAL + 255) / 256, 256, 0, w->stream>>>(w->W, w->stage, 0);
  WS_CK(cudaGetLastError());
  WS_CK(cudaMemcpyAsync(params, w->stage, sizeof(float) * U_TOTAL, cudaMemcpyDefault, w->stream));
  WS_CK(cudaStreamSynchronize(w->stream));
  return TRAJ_OK;
}

traj_status traj_warmstart_get_state(traj_warmstart *w, float *params, float *m, float *v,
                                     int *step) {
  if (!w || !params || !m || !v || !step) return ws_fail(TRAJ_EINVAL, "NULL training-state argument");
  const float *src[3] = {w->W, w->m, w->v};
  float *dst[3] = {params, m, v};
  for (int i = 0; i < 3; ++i) { // stream order: each copy reads the staging buffer before it is reused
    k_params_pad<<<(P_TOTAL + 255) / 256, 256, 0, w->stream>>>(src[i], w->stage, 0);
    WS_CK(cudaGetLastError());
    WS_CK(cudaMemcpyAsync(dst[i], w->stage, sizeof(float) * U_TOTAL, cudaMemcpyDefault, w->stream));
  }
  WS_CK(cudaStreamSynchronize(w->stream));
  *step = w->step;
  return TRAJ_OK;
}

traj_status traj_warmstart_set_state(traj_warmstart *w, const float *params, const float *m,
                                     const float *v, int step) {
  if (!w || !params || !m || !v) return ws_fail(TRAJ_EINVAL, "NULL training-state argument");
  if (step < 0) return ws_fail(TRAJ_EINVAL, "step must be >= 0");
  const float *src[3] = {params, m, v};
  float *dst[3] = {w->W, w->m, w->v};
  for (int i = 0; i < 3; ++i) {
    WS_CK(cudaMemcpyAsync(w->stage, src[i], sizeof(float) * U_TOTAL, cudaMemcpyDefault, w->stream));
    k_params_pad<<<(P_TOTAL + 255) / 256, 256, 0, w->stream>>>(w->stage, dst[i], 1);
    WS_CK(cudaGetLastError());
  }
  w->step = step;
  WS_CK(refresh_bf16(w, 0, 0.f, 0.f)); // BF16 copies of the restored master weights
  WS_CK(cudaStreamSynchronize(w->stream));
  return TRAJ_OK;
}

traj_status traj_warmstart_features(traj_warmstart *w, int n_scenes, const double *start,
                                    const double *goal, const int *offsets, const float *centers,
                                    const float *semi_axes, const float *velocities,
                                    void *features, float *line) {
  if (!w || !start || !goal || !offsets || !features || !line || n_scenes < 1)
    return ws_fail(TRAJ_EINVAL, "NULL or empty feature arguments");
  if (offsets[0] != 0) return ws_fail(TRAJ_EINVAL, "offsets[0] must be 0");
  for (int p = 0; p < n_scenes; ++p)
    if (offsets[p + 1] < offsets[p]) return ws_fail(TRAJ_EINVAL, "offsets must be non-decreasing");
  if (offsets[n_scenes] > 0 && (!centers || !semi_axes || !velocities)) return ws_fail(TRAJ_EINVAL, "NULL obstacles");
  if (n_scenes > w->feat_cap) {
    if (w->d_start) { cudaFree(w->d_start); cudaFree(w->d_goal); cudaFree(w->d_offsets); }
    w->d_start = w->d_goal = nullptr; w->d_offsets = nullptr; w->feat_cap = 0;
    WS_CK(cudaMalloc(&w->d_start, sizeof(double) * 2 * n_scenes));
    WS_CK(cudaMalloc(&w->d_goal, sizeof(double) * 2 * n_scenes));
    WS_CK(cudaMalloc(&w->d_offsets, sizeof(int) * (n_scenes + 1)));
    w->feat_cap = n_scenes;
  }
  WS_CK(cudaMemcpyAsync(w->d_start, start, sizeof(double) * 2 * n_scenes, cudaMemcpyDefault, w->stream));
  WS_CK(cudaMemcpyAsync(w->d_goal, goal, sizeof(double) * 2 * n_scenes, cudaMemcpyDefault, w->stream));
  WS_CK(cudaMemcpyAsync(w->d_offsets, offsets, sizeof(int) * (n_scenes + 1), cudaMemcpyDefault, w->stream));
  k_features<<<n_scenes, 256, 0, w->stream>>>(w->d_start, w->d_goal, w->d_offsets, offsets[n_scenes],
                                               centers, semi_axes, velocities,
                                               reinterpret_cast<__nv_bfloat16 *>(features), line, w->err);
  WS_CK(cudaGetLastError());
  WS_CK(cudaStreamSynchronize(w->stream)); // host sources of start/goal/offsets
  return TRAJ_OK;
}

traj_status traj_warmstart_propose(traj_warmstart *w, int n_scenes, int n_obs, const double *start,
                                   const double *goal, const int *offsets, const float *centers,
                                   const float *semi_axes, const float *velocities, void *features,
                                   float *line, float *proposals) {
  tb::NvtxRange nvtx_range("traj_warmstart_propose");
  if (!w || !start || !goal || !offsets || !features || !line || !proposals || n_obs < 0)
    return ws_fail(TRAJ_EINVAL, "NULL argument or negative obstacle count");
  if (n_obs > 0 && (!centers || !semi_axes || !velocities)) return ws_fail(TRAJ_EINVAL, "NULL obstacles");
  traj_status rc = check_rows(w, n_scenes);
  if (rc != TRAJ_OK) return rc;
  k_features<<<n_scenes, 256, 0, w->stream>>>(start, goal, offsets, n_obs, centers, semi_axes,
                                               velocities, reinterpret_cast<__nv_bfloat16 *>(features),
                                               line, w->err);
  WS_CK(cudaGetLastError());
  WS_CK(forward(w, n_scenes, features));
  k_proposals<<<(n_scenes * OUT + 255) / 256, 256, 0, w->stream>>>(w->Y, line, n_scenes, proposals);
  WS_CK(cudaGetLastError());
  return TRAJ_OK;
}

traj_status traj_warmstart_forward(traj_warmstart *w, int rows, const void *features,
                                   const float *line, float *proposals) {
  tb::NvtxRange nvtx_range("traj_warmstart_forward");
  if (!w || !features || !line || !proposals) return TRAJ_EINVAL;
  traj_status rc = check_rows(w, rows);
  if (rc != TRAJ_OK) return rc;
  WS_CK(forward(w, rows, features));
  k_proposals<<<(rows * OUT + 255) / 256, 256, 0, w->stream>>>(w->Y, line, rows, proposals);
  WS_CK(cudaGetLastError());
  return TRAJ_OK;
}

traj_status traj_warmstart_gradients(traj_warmstart *w, int rows, const void *features,
                                     const float *targets, const int *n_labels, float *grads,
                                     float *loss) {
  if (!w || !features || !targets || !n_labels || !loss) return TRAJ_EINVAL;
  traj_status rc = check_rows(w, rows);
  if (rc != TRAJ_OK) return rc;
  WS_CK(backward(w, rows, features, targets, n_labels, loss));
  if (grads) {
    k_params_pad<<<(P_TOTAL + 255) / 256, 256, 0, w->stream>>>(w->g, w->stage, 0);
    WS_CK(cudaGetLastError());
    WS_CK(cudaMemcpyAsync(grads, w->stage, sizeof(float) * U_TOTAL, cudaMemcpyDefault, w->stream));
  }
  return TRAJ_OK;
}

traj_status traj_warmstart_gradients_fp32(traj_warmstart *w, int rows, const void *features,
                                          const float *targets, const int *n_labels, float *grads,
                                          float *loss) {
  if (!w || !features || !targets || !n_labels || !loss) return TRAJ_EINVAL;
  traj_status rc = check_rows(w, rows);
  if (rc != TRAJ_OK) return rc;
  if (!w->f_X) {
    const size_t R = w->max_rows;
    if (!ws_alloc(w, &w->f_X, R * IN_PAD) || !ws_alloc(w, &w->f_H1, R * HID) ||
        !ws_alloc(w, &w->f_H2, R * HID) || !ws_alloc(w, &w->f_H3, R * HID) ||
        !ws_alloc(w, &w->f_dZ1, R * HID) || !ws_alloc(w, &w->f_dZ2, R * HID) ||
        !ws_alloc(w, &w->f_dZ3, R * HID)) {
      w->f_X = nullptr; // the buffers allocated so far are released by destroy
      return ws_fail(TRAJ_ENOMEM, "cudaMalloc failed (FP32 debug buffers)");
    }
  }
  WS_CK(backward_f32(w, rows, features, targets, n_labels, loss));
  if (grads) {
    k_params_pad<<<(P_TOTAL + 255) / 256, 256, 0, w->stream>>>(w->g, w->stage, 0);
    WS_CK(cudaGetLastError());
    WS_CK(cudaMemcpyAsync(grads, w->stage, sizeof(float) * U_TOTAL, cudaMemcpyDefault, w->stream));
  }
  return TRAJ_OK;
}

traj_status traj_warmstart_train_step(traj_warmstart *w, int rows, const void *features,
                                      const float *targets, const int *n_labels, float lr,
                                      float weight_decay, float *loss) {
  tb::NvtxRange nvtx_range("traj_warmstart_train_step");
  if (!w || !features || !targets || !n_labels || !loss) return TRAJ_EINVAL;
  if (!(lr > 0) || !(weight_decay >= 0)) return ws_fail(TRAJ_EINVAL, "bad learning rate or decay");
  traj_status rc = check_rows(w, rows);
  if (rc != TRAJ_OK) return rc;
  WS_CK(backward(w, rows, features, targets, n_labels, loss));
  w->step += 1;
  WS_CK(refresh_bf16(w, 1, lr, weight_decay));
  return TRAJ_OK;
}

traj_status traj_warmstart_sync(traj_warmstart *w) {
  if (!w) return TRAJ_EINVAL;
  WS_CK(cudaStreamSynchronize(w->stream));
  int err = 0;
  WS_CK(cudaMemcpy(&err, w->err, sizeof(int), cudaMemcpyDeviceToHost));
  WS_CK(cudaMemsetAsync(w->err, 0, sizeof(int), w->stream));
  WS_CK(cudaStreamSynchronize(w->stream));
  if (err & 2) return ws_fail(TRAJ_EINVAL, "obstacle offsets outside [0, n_obs] in traj_warmstart_propose");
  if (err) return ws_fail(TRAJ_ECUDA, "a tensor-core GEMM pipeline wait expired");
  return TRAJ_OK;
}

} // extern "C"

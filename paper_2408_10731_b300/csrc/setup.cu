// setup.cu -- once-per-problem set-up on the GPU, in FP64.
//
//  * Bernstein tables per horizon (eq. parameter; degree 10 on tau = t/(n_p-1)):
//    P, dB/dtau, d2B/dtau2, FP64 evaluation stored as FP32 rows of 12.
//  * KKT formation and inversion per problem (eqs. over_2, zeta_1_sepration_3,
//    Q_matrix, matrix_vec): Q-bar = Q + rho F^T F with F^T F = n_o P^T P +
//    Pd^T Pd + Pdd^T Pdd (the stacked F of Paper II is never formed), boundary
//    rows A = [P_0; Pd_0; Pdd_0; P_{-1}] with b = (start, v0, a0, goal), v0 = a0 = 0
//    unless a start state is given, Gauss-Jordan with partial pivoting in
//    FP64, then the per-problem constants the FP32 loop needs, each split into
//    an FP32 (hi, lo) pair: K11, G = rho K11 F^T F, c = K12 b, hq = K11 (-q) + c.
//  * Obstacle packing: moving ellipses/ellipsoids into the float4 records the
//    solve kernel reads, with a per-problem flag for non-finite data.
#include "internal.cuh"
#include "basis.cuh"
#include <math.h>

namespace tb {

__global__ void k_tables(const int *horizons, const int *offsets, float *tables) {
  const int h = blockIdx.x;
  const int n_p = horizons[h];
  float *T0 = tables + offsets[h];
  for (int t = threadIdx.x; t < n_p; t += blockDim.x) {
    double P[NC], dB[NC], ddB[NC];
    basis_row(n_p, t, P, dB, ddB);
    for (int i = 0; i < ROW; ++i) {
      T0[(0 * n_p + t) * ROW + i] = i < NC ? (float)P[i] : 0.f;
      T0[(1 * n_p + t) * ROW + i] = i < NC ? (float)dB[i] : 0.f;
      T0[(2 * n_p + t) * ROW + i] = i < NC ? (float)ddB[i] : 0.f;
    }
  }
}

__device__ __forceinline__ void split_store(float *hi, float *lo, double x) {
  float h = (float)x;
  *hi = h;
  *lo = (float)(x - (double)h);
}

// One block of SETUP_THREADS per problem. The scaled basis rows are staged in
// shared memory SETUP_CHUNK grid points at a time (3 * min(max_np, SETUP_CHUNK) * NC
// doubles), so any horizon fits; each thread keeps its Gram / q sums over the
// chunks in a register, adding the grid points in ascending order.
constexpr int SETUP_THREADS = 256, SETUP_CHUNK = 256;
static_assert(NC * NC + 3 * NC <= SETUP_THREADS, "one Gram / q element per thread");

__global__ void __launch_bounds__(SETUP_THREADS)
k_setup_problems(ProblemDev *problems, const double *Tarr, const double *start,
                 const double *goal, const double *start_va, int dim, double rho, double w_s,
                 double w_t, int cost_mode, float *constants, double *kkt_out, size_t kkt_stride) {
  extern __shared__ double sm[];
  __shared__ double Q[NC * NC], M[NC * NC], qv[3 * NC];
  __shared__ double W[NK * 2 * NK];
  __shared__ double K11[NC * NC], K12[NC * NE], Gm[NC * NC];
  __shared__ double Bnd[NE][NC]; // boundary rows P_0, Pd_0, Pdd_0, P_{n_p - 1}
  __shared__ int piv_s;
  const int p = blockIdx.x;
  const ProblemDev pr = problems[p];
  const int n_p = pr.n_p, n_o = pr.n_o;
  const double T = Tarr[p];
  const int CH = n_p < SETUP_CHUNK ? n_p : SETUP_CHUNK;
  double *P = sm, *Pd = sm + CH * NC, *Pdd = sm + 2 * CH * NC;
  const double iT = 1.0 / T, iT2 = 1.0 / (T * T);

  // Q, M = F^T F (closed form of the stacked F), q per axis: element el of thread el
  const int el = threadIdx.x;
  const bool gram = el < NC * NC, qrow = el >= NC * NC && el < NC * NC + 3 * NC;
  const int ga = gram ? el / NC : 0, gb = gram ? el % NC : 0;
  const int qk = qrow ? el - NC * NC : 0, qax = qk / NC, qi = qk % NC;
  const double s0 = qrow && qax < dim ? start[p * dim + qax] : 0.0;
  const double g0 = qrow && qax < dim ? goal[p * dim + qax] : 0.0;
  double pp = 0, dd = 0, aa = 0, sq = 0, mo0 = 0, mo1 = 0; // mo0 / mo1: basis moments
  for (int c0 = 0; c0 < n_p; c0 += CH) {
    const int nc = n_p - c0 < CH ? n_p - c0 : CH;
    __syncthreads(); // the previous chunk has been read
    for (int t = threadIdx.x; t < nc; t += blockDim.x) {
      double a[NC], b[NC], c[NC];
      basis_row(n_p, c0 + t, a, b, c);
      for (int i = 0; i < NC; ++i) {
        P[t * NC + i] = a[i];
        Pd[t * NC + i] = b[i] * iT;
        Pdd[t * NC + i] = c[i] * iT2;
      }
    }
    __syncthreads();
    // boundary rows from the staged chunks: the first grid point and the last
    if (c0 == 0 && threadIdx.x < NC) {
      Bnd[0][threadIdx.x] = P[threadIdx.x];
      Bnd[1][threadIdx.x] = Pd[threadIdx.x];
      Bnd[2][threadIdx.x] = Pdd[threadIdx.x];
    }
    if (c0 + nc == n_p && threadIdx.x >= 32 && threadIdx.x < 32 + NC)
      Bnd[3][threadIdx.x - 32] = P[(nc - 1) * NC + threadIdx.x - 32];
    if (gram) {
      for (int t = 0; t < nc; ++t) {
        pp += P[t * NC + ga] * P[t * NC + gb];
        dd += Pd[t * NC + ga] * Pd[t * NC + gb];
        aa += Pdd[t * NC + ga] * Pdd[t * NC + gb];
      }
    } else if (qrow && qax < dim) {
      for (int t = 0; t < nc; ++t) {
        double tau = (double)(c0 + t) / (double)(n_p - 1);
        sq += P[t * NC + qi] * (s0 + (g0 - s0) * tau);
        mo0 += P[t * NC + qi] * (1.0 - tau);
        mo1 += P[t * NC + qi] * tau;
      }
    }
  }
  if (gram) {
    Q[el] = cost_mode == 0 ? (w_s * aa + w_t * pp) : (ga == gb ? 1.0 : 0.0);
    M[el] = (double)(n_o + 2 * pr.box) * pp + dd + aa; // G = [-P; P] per axis adds 2 P^T P
  } else if (qrow) {
    qv[qk] = -w_t * sq; // q = -w_t P^T x_des
  }
  __syncthreads();
  // augmented [K | I]
  for (int e = threadIdx.x; e < NK * 2 * NK; e += blockDim.x) {
    int r = e / (2 * NK), c = e % (2 * NK);
    double v;
    if (c >= NK) v = (c - NK == r) ? 1.0 : 0.0;
    else if (r < NC && c < NC) v = Q[r * NC + c] + rho * M[r * NC + c];
    else if (r < NC && c >= NC) { // A^T
      int er = c - NC;
      v = Bnd[er][r];
    } else if (r >= NC && c < NC) {
      int er = r - NC;
      v = Bnd[er][c];
    } else v = 0.0;
    W[e] = v;
  }
  __syncthreads();
  // Gauss-Jordan with partial pivoting
  for (int col = 0; col < NK; ++col) {
    if (threadIdx.x == 0) {
      int pv = col;
      for (int r = col + 1; r < NK; ++r)
        if (fabs(W[r * 2 * NK + col]) > fabs(W[pv * 2 * NK + col])) pv = r;
      piv_s = pv;
      const double pivot = W[pv * 2 * NK + col];
      if (pivot == 0.0 || !isfinite(pivot)) atomicOr(&problems[p].nan_flag, 2); // singular KKT
    }
    __syncthreads();
    const int pv = piv_s;
    if (pv != col)
      for (int c = threadIdx.x; c < 2 * NK; c += blockDim.x) {
        double tmp = W[col * 2 * NK + c];
        W[col * 2 * NK + c] = W[pv * 2 * NK + c];
        W[pv * 2 * NK + c] = tmp;
      }
    __syncthreads();
    const double inv = 1.0 / W[col * 2 * NK + col];
    __syncthreads();
    for (int c = threadIdx.x; c < 2 * NK; c += blockDim.x) W[col * 2 * NK + c] *= inv;
    __syncthreads();
    for (int e = threadIdx.x; e < NK * 2 * NK; e += blockDim.x) {
      int r = e / (2 * NK), c = e % (2 * NK);
      if (r == col) continue;
      double f = W[r * 2 * NK + col];
      if (c == col) continue; // column col is cleared after the loop
      W[e] -= f * W[col * 2 * NK + c];
    }
    __syncthreads();
    for (int r = threadIdx.x; r < NK; r += blockDim.x)
      if (r != col) W[r * 2 * NK + col] = 0.0;
    __syncthreads();
  }
  for (int e = threadIdx.x; e < NC * NC + NC * NE; e += blockDim.x) {
    if (e < NC * NC) K11[e] = W[(e / NC) * 2 * NK + NK + (e % NC)];
    else {
      int k = e - NC * NC, r = k / NE, c = k % NE;
      K12[k] = W[r * 2 * NK + NK + NC + c];
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < NC * NC; e += blockDim.x) {
    int a = e / NC, b = e % NC;
    double s = 0;
    for (int k = 0; k < NC; ++k) s += K11[a * NC + k] * M[k * NC + b];
    Gm[e] = rho * s;
  }
  __syncthreads();
  float *C = constants + pr.const_off;
  for (int e = threadIdx.x; e < NC * ROW; e += blockDim.x) {
    int r = e / ROW, c = e % ROW;
    double k11 = c < NC ? K11[r * NC + c] : 0.0, g = c < NC ? Gm[r * NC + c] : 0.0;
    split_store(&C[C_K11_HI + e], &C[C_K11_LO + e], k11);
    split_store(&C[C_G_HI + e], &C[C_G_LO + e], g);
  }
  for (int e = threadIdx.x; e < 3 * ROW; e += blockDim.x) {
    int ax = e / ROW, i = e % ROW;
    double cval = 0, hq = 0;
    if (ax < dim && i < NC) {
      // b = (start, v0, a0, goal): at rest unless a start state is given (the
      // receding-horizon step moves the start onto the executed plan)
      const double v0 = start_va ? start_va[(p * 2 + 0) * dim + ax] : 0.0;
      const double a0 = start_va ? start_va[(p * 2 + 1) * dim + ax] : 0.0;
      double bb[NE] = {start[p * dim + ax], v0, a0, goal[p * dim + ax]};
      for (int k = 0; k < NE; ++k) cval += K12[i * NE + k] * bb[k];
      hq = cval;
      for (int k = 0; k < NC; ++k) hq += K11[i * NC + k] * (-qv[ax * NC + k]);
    }
    split_store(&C[C_HQ_HI + e], &C[C_HQ_LO + e], hq);
    split_store(&C[C_C_HI + e], &C[C_C_LO + e], cval);
  }
  if (kkt_out) { // the blocks a boundary-only update needs (launch_setup_boundary)
    double *K = kkt_out + (size_t)p * kkt_stride;
    for (int e = threadIdx.x; e < NC * NC + NC * NE; e += blockDim.x)
      K[e] = e < NC * NC ? K11[e] : K12[e - NC * NC];
    if (qrow && qax == 0) {
      K[NC * NC + NC * NE + qi] = mo0;
      K[NC * NC + NC * NE + NC + qi] = mo1;
    }
  }
}

// One thread per (problem, level, constants entry of the hq / c blocks): hq and c from
// the stored FP64 blocks, in the full set-up's order of operations except q, which is
// formed from the basis moments (q_i = -w_t (s0 m0_i + g0 m1_i), the same sum
// regrouped).
__global__ void k_setup_boundary(int n_problems, int levels, const double *start,
                                 const double *goal, const double *start_va, int dim,
                                 double w_t, const double *kkt64, float *constants) {
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = (long long)n_problems * levels * 3 * ROW;
  if (id >= total) return;
  const int e = (int)(id % (3 * ROW));
  const long long pl = id / (3 * ROW);
  const int l = (int)(pl % levels), p = (int)(pl / levels);
  const double *K = kkt64 + (size_t)pl * KKT64_DOUBLES;
  const double *K11 = K, *K12 = K + NC * NC, *m0 = K12 + NC * NE, *m1 = m0 + NC;
  float *C = constants + (size_t)p * CONST_FLOATS * levels + (size_t)l * CONST_FLOATS;
  const int ax = e / ROW, i = e % ROW;
  double cval = 0, hq = 0;
  if (ax < dim && i < NC) {
    const double s0 = start[p * dim + ax], g0 = goal[p * dim + ax];
    const double v0 = start_va ? start_va[(p * 2 + 0) * dim + ax] : 0.0;
    const double a0 = start_va ? start_va[(p * 2 + 1) * dim + ax] : 0.0;
    const double bb[NE] = {s0, v0, a0, g0};
    for (int k = 0; k < NE; ++k) cval += K12[i * NE + k] * bb[k];
    hq = cval;
    for (int k = 0; k < NC; ++k) hq += K11[i * NC + k] * (w_t * (s0 * m0[k] + g0 * m1[k]));
  }
  split_store(&C[C_HQ_HI + e], &C[C_HQ_LO + e], hq);
  split_store(&C[C_C_HI + e], &C[C_C_LO + e], cval);
}

// One thread per half of a pair record (see the layout in internal.cuh): problem p
// owns records pair_off[p] .. pair_off[p + 1) - 1; the record's half h holds the
// problem's obstacle 2 (q - pair_off[p]) + h, or the sentinel past its last obstacle.
__global__ void k_pack_obstacles(int dim, int n_problems, int n_slots, const int *offsets,
                                 const int *pair_off, const float *cen, const float *ax,
                                 const float *vel, float4 *out, ProblemDev *problems) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_slots) return;
  const int q = s >> 1, h = s & 1;
  int lo = 0, hi = n_problems - 1;
  while (lo < hi) { // last problem whose first record is <= q
    const int mid = (lo + hi + 1) >> 1;
    if (pair_off[mid] <= q) lo = mid; else hi = mid - 1;
  }
  const int p = lo;
  const int l = 2 * (q - pair_off[p]) + h;
  const int n_o = offsets[p + 1] - offsets[p];
  float *rec = reinterpret_cast<float *>(out + (size_t)pair_vec(dim) * q);
  const int B = 4 * dim;
  if (l >= n_o) {
    for (int d = 0; d < dim; ++d) {
      rec[4 * d + h] = PAIR_SENTINEL;
      rec[4 * d + 2 + h] = 0.f;
      rec[B + 2 * d + h] = 1.f;
      rec[B + 2 * dim + 2 * d + h] = 1.f;
    }
    return;
  }
  const int j = offsets[p] + l;
  bool ok = true;
  for (int d = 0; d < dim; ++d) {
    const double c = cen[j * dim + d], a = ax[j * dim + d], v = vel[j * dim + d];
    ok = ok && isfinite(c) && isfinite(v) && isfinite(a) && a > 0.0;
    rec[4 * d + h] = (float)(-c / a);
    rec[4 * d + 2 + h] = (float)(-v / a);
    rec[B + 2 * d + h] = (float)(1.0 / a);
    rec[B + 2 * dim + 2 * d + h] = (float)a;
  }
  if (!ok) atomicOr(&problems[p].nan_flag, 1);
}

cudaError_t launch_setup_tables(const int *d_horizons, const int *d_offsets, int n_horizons,
                                float *d_tables, cudaStream_t s) {
  if (n_horizons <= 0) return cudaSuccess;
  k_tables<<<n_horizons, 128, 0, s>>>(d_horizons, d_offsets, d_tables);
  return cudaGetLastError();
}

cudaError_t launch_setup_problems(ProblemDev *d_problems, int n_problems, const double *d_T,
                                  const double *d_start, const double *d_goal,
                                  const double *d_start_va, int dim,
                                  double rho, double w_smooth, double w_track, int cost_mode,
                                  int max_np, float *d_constants, cudaStream_t s, double *kkt_out,
                                  size_t kkt_stride) {
  if (n_problems <= 0) return cudaSuccess;
  const int ch = max_np < SETUP_CHUNK ? max_np : SETUP_CHUNK;
  size_t smem = sizeof(double) * 3 * (size_t)ch * NC;
  cudaError_t e = cudaFuncSetAttribute(k_setup_problems,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_setup_problems<<<n_problems, SETUP_THREADS, smem, s>>>(d_problems, d_T, d_start, d_goal,
                                                           d_start_va, dim, rho, w_smooth, w_track,
                                                           cost_mode, d_constants, kkt_out,
                                                           kkt_stride);
  return cudaGetLastError();
}

cudaError_t launch_setup_boundary(int n_problems, int levels, const double *d_start,
                                  const double *d_goal, const double *d_start_va, int dim,
                                  double w_track, const double *kkt64, float *d_constants,
                                  cudaStream_t s) {
  if (n_problems <= 0 || levels <= 0) return cudaSuccess;
  // small blocks: the FP64 dot products spread over every SM instead of a few
  const long long total = (long long)n_problems * levels * 3 * ROW;
  k_setup_boundary<<<(unsigned)((total + 31) / 32), 32, 0, s>>>(
      n_problems, levels, d_start, d_goal, d_start_va, dim, w_track, kkt64, d_constants);
  return cudaGetLastError();
}

cudaError_t launch_pack_obstacles(int dim, int n_problems, int n_slots, const int *offsets,
                                  const int *pair_off, const float *centers, const float *axes,
                                  const float *vel, float4 *out, ProblemDev *problems,
                                  cudaStream_t s) {
  if (n_slots <= 0 || n_problems <= 0) return cudaSuccess;
  // small blocks: the FP64 divisions spread over every SM instead of a few
  k_pack_obstacles<<<(n_slots + 31) / 32, 32, 0, s>>>(dim, n_problems, n_slots, offsets,
                                                      pair_off, centers, axes, vel, out,
                                                      problems);
  return cudaGetLastError();
}

} // namespace tb

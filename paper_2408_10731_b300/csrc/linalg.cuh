// linalg.cuh -- small FP64 helpers of the once-per-problem set-up kernels.
#pragma once

namespace tb {

// In-place Gauss-Jordan with partial pivoting of the augmented [K | I] (n x 2n,
// row stride 2n) by the whole block; sets *bad if a pivot is zero or not finite.
// piv and bad point to shared memory.
__device__ inline void gj_invert(double *W, int n, int *piv, int *bad) {
  const int ld = 2 * n;
  for (int col = 0; col < n; ++col) {
    if (threadIdx.x == 0) {
      int pv = col;
      for (int r = col + 1; r < n; ++r)
        if (fabs(W[r * ld + col]) > fabs(W[pv * ld + col])) pv = r;
      *piv = pv;
      const double pvv = W[pv * ld + col];
      if (pvv == 0.0 || !isfinite(pvv)) *bad = 1;
    }
    __syncthreads();
    const int pv = *piv;
    if (pv != col)
      for (int c = threadIdx.x; c < ld; c += blockDim.x) {
        const double t = W[col * ld + c];
        W[col * ld + c] = W[pv * ld + c];
        W[pv * ld + c] = t;
      }
    __syncthreads();
    const double inv = 1.0 / W[col * ld + col];
    __syncthreads();
    for (int c = threadIdx.x; c < ld; c += blockDim.x) W[col * ld + c] *= inv;
    __syncthreads();
    for (int e = threadIdx.x; e < n * ld; e += blockDim.x) {
      const int r = e / ld, c = e % ld;
      if (r != col && c != col) W[e] -= W[r * ld + col] * W[col * ld + c];
    }
    __syncthreads();
    for (int r = threadIdx.x; r < n; r += blockDim.x)
      if (r != col) W[r * ld + col] = 0.0;
    __syncthreads();
  }
}

// x as an FP32 (hi, lo) pair
__device__ __forceinline__ void split2(float *hi, float *lo, double x) {
  const float h = (float)x;
  *hi = h;
  *lo = (float)(x - (double)h);
}

} // namespace tb

// basis.cuh -- the Bernstein basis in FP64 (eq. parameter; degree 10 on
// tau = t / (n_p - 1)), shared by the single-agent and multi-agent set-up kernels.
#pragma once

namespace tb {

__device__ inline double bern_d(int n, int i, double tau) {
  if (i < 0 || i > n) return 0.0;
  double c = 1.0;
  for (int k = 1; k <= i; ++k) c = c * (double)(n - i + k) / (double)k;
  double p = 1.0;
  for (int k = 0; k < i; ++k) p *= tau;
  for (int k = 0; k < n - i; ++k) p *= (1.0 - tau);
  return c * p;
}

// Unscaled basis values and tau-derivatives (11 each) at grid point t of an
// n_p-point horizon.
__device__ inline void basis_row(int n_p, int t, double *P, double *dB, double *ddB) {
  const int n = 10;
  double tau = (double)t / (double)(n_p - 1);
  for (int i = 0; i <= n; ++i) {
    P[i] = bern_d(n, i, tau);
    dB[i] = n * (bern_d(n - 1, i - 1, tau) - bern_d(n - 1, i, tau));
    ddB[i] = n * (n - 1) *
             (bern_d(n - 2, i - 2, tau) - 2.0 * bern_d(n - 2, i - 1, tau) + bern_d(n - 2, i, tau));
  }
}

} // namespace tb

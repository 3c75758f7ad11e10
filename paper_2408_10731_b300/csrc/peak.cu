// peak.cu -- FP32 FFMA throughput microbenchmark: the denominator of the ALU
// roofline that the solve kernel is measured against (no FP32 figure exists in
// the driver's measured peaks). Eight independent FMA chains per thread keep
// the FMA pipes busy without memory traffic.
#include "internal.cuh"

namespace tb {

__global__ void k_ffma_peak(float *out, int iters) {
  float a0 = threadIdx.x * 1e-7f, a1 = a0 + 1e-7f, a2 = a0 + 2e-7f, a3 = a0 + 3e-7f;
  float a4 = a0 + 4e-7f, a5 = a0 + 5e-7f, a6 = a0 + 6e-7f, a7 = a0 + 7e-7f;
  const float b = 0.999999f, c = 1e-7f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      a0 = fmaf(a0, b, c); a1 = fmaf(a1, b, c); a2 = fmaf(a2, b, c); a3 = fmaf(a3, b, c);
      a4 = fmaf(a4, b, c); a5 = fmaf(a5, b, c); a6 = fmaf(a6, b, c); a7 = fmaf(a7, b, c);
    }
  }
  const float s = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
  if (s == 123.456f) out[blockIdx.x] = s; // practically never true; keeps the chains live
}

cudaError_t launch_ffma_peak(float *out, int blocks, int iters, cudaStream_t s) {
  k_ffma_peak<<<blocks, 256, 0, s>>>(out, iters);
  return cudaGetLastError();
}

} // namespace tb

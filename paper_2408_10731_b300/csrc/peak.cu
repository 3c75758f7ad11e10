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

// Same with packed two-lane FMA (fma.rn.f32x2): 16 FP32 FMAs per inner step.
__global__ void k_ffma2_peak(float *out, int iters) {
  float2 a0 = make_float2(threadIdx.x * 1e-7f, 1e-7f), a1 = make_float2(2e-7f, 3e-7f);
  float2 a2 = make_float2(4e-7f, 5e-7f), a3 = make_float2(6e-7f, 7e-7f);
  float2 a4 = make_float2(8e-7f, 9e-7f), a5 = make_float2(1e-6f, 2e-6f);
  float2 a6 = make_float2(3e-6f, 4e-6f), a7 = make_float2(5e-6f, 6e-6f);
  const float2 b = make_float2(0.999999f, 0.999998f), c = make_float2(1e-7f, 2e-7f);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      a0 = __ffma2_rn(a0, b, c); a1 = __ffma2_rn(a1, b, c); a2 = __ffma2_rn(a2, b, c);
      a3 = __ffma2_rn(a3, b, c); a4 = __ffma2_rn(a4, b, c); a5 = __ffma2_rn(a5, b, c);
      a6 = __ffma2_rn(a6, b, c); a7 = __ffma2_rn(a7, b, c);
    }
  }
  const float s = a0.x + a1.x + a2.x + a3.x + a4.x + a5.x + a6.x + a7.x + a0.y + a1.y + a2.y +
                  a3.y + a4.y + a5.y + a6.y + a7.y;
  if (s == 123.456f) out[blockIdx.x] = s;
}

cudaError_t launch_ffma_peak(float *out, int blocks, int iters, cudaStream_t s) {
  k_ffma_peak<<<blocks, 256, 0, s>>>(out, iters);
  return cudaGetLastError();
}

cudaError_t launch_ffma2_peak(float *out, int blocks, int iters, cudaStream_t s) {
  k_ffma2_peak<<<blocks, 256, 0, s>>>(out, iters);
  return cudaGetLastError();
}

} // namespace tb

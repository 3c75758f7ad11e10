// peak.cu -- FP32 FFMA and MUFU reciprocal-square-root throughput
// microbenchmarks: the denominators of the ALU roofline that the solve kernels
// are measured against (no FP32 or MUFU figure exists in the measured peaks).
// Eight independent chains per thread keep the pipe busy without memory traffic.
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

// Eight independent rsqrtf chains (x <- 1/sqrt(x), which stays in (0, inf) and
// tends to 1): the same instruction the projections issue once per point inside an
// obstacle and once per velocity / acceleration bound test.
__global__ void k_rsqrt_peak(float *out, int iters) {
  float a0 = 1.0f + threadIdx.x * 1e-3f, a1 = a0 + 0.1f, a2 = a0 + 0.2f, a3 = a0 + 0.3f;
  float a4 = a0 + 0.4f, a5 = a0 + 0.5f, a6 = a0 + 0.6f, a7 = a0 + 0.7f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      a0 = rsqrtf(a0); a1 = rsqrtf(a1); a2 = rsqrtf(a2); a3 = rsqrtf(a3);
      a4 = rsqrtf(a4); a5 = rsqrtf(a5); a6 = rsqrtf(a6); a7 = rsqrtf(a7);
    }
  }
  const float s = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
  if (s == 123.456f) out[blockIdx.x] = s;
}

cudaError_t launch_rsqrt_peak(float *out, int blocks, int iters, cudaStream_t s) {
  k_rsqrt_peak<<<blocks, 256, 0, s>>>(out, iters);
  return cudaGetLastError();
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

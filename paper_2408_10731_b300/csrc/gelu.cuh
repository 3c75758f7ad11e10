// gelu.cuh -- the tanh form of GELU (Hendrycks & Gimpel, 2016) and its derivative,
// shared by the tensor-core GEMM's epilogues (gemm_tc.cu) and the FP32-operand
// debug path of the warm-start network (warmstart.cu).
#pragma once

namespace tb {

__device__ __forceinline__ float gelu_tanh(float z) {
  const float k0 = 0.7978845608028654f, k1 = 0.044715f;
  return 0.5f * z * (1.f + tanhf(k0 * (z + k1 * z * z * z)));
}

__device__ __forceinline__ float gelu_tanh_grad(float z) {
  const float k0 = 0.7978845608028654f, k1 = 0.044715f;
  const float t = tanhf(k0 * (z + k1 * z * z * z));
  return 0.5f * (1.f + t) + 0.5f * z * (1.f - t * t) * k0 * (1.f + 3.f * k1 * z * z);
}

} // namespace tb

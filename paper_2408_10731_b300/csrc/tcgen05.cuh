// tcgen05.cuh -- helpers for the 5th-generation tensor cores shared by the
// BF16 GEMM (gemm_tc.cu) and the tensor-core AM form (am_mixed.cu): shared
// addresses, bounded mbarrier waits, the shared-memory matrix descriptor of a
// K-major tile in the 128-byte swizzle layout, and the kind::f16 instruction
// descriptor.
#pragma once
#include <stdint.h>

namespace tb {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
               " selp.u32 %0, 1, 0, p;\n}"
               : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
  return ok != 0;
}

// Bounded wait: false if the phase did not complete within `limit` polls.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint32_t limit = 1u << 22) {
  for (uint32_t i = 0; i < limit; ++i)
    if (mbar_try(bar, parity)) return true;
  return false;
}

// K-major tile in the 128-byte swizzle layout (8-row atoms of 1024 B, the
// layout TMA writes with CU_TENSOR_MAP_SWIZZLE_128B): start address, LBO 16 B
// (unused for this layout), SBO 1024 B between 8-row groups, descriptor
// version 1, layout type 2. Element (r, k) of a 64-column tile sits at byte
// r * 128 + (((k / 8) ^ (r % 8)) * 16) + (k % 8) * 2 from a 1024-aligned base.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

__device__ __forceinline__ uint32_t sw128_offset(int r, int k) {
  return (uint32_t)(r * 128 + ((((k >> 3) ^ (r & 7)) & 7) << 4) + ((k & 7) << 1));
}

// kind::f16 instruction descriptor: FP32 D, BF16 A and B, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

} // namespace tb

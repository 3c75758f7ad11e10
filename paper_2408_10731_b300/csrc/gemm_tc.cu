// gemm_tc.cu -- BF16 GEMM on the 5th-generation tensor cores (tcgen05) with
// TMA-staged operands, for the warm-start network's training and inference.
//
//   C[M x N] = A[M x K] * B[N x K]^T,   A, B row-major BF16 (K contiguous),
//   FP32 accumulation in tensor memory, fused epilogues (bias, GELU, GELU').
//
// One CTA computes one 128 x BN tile (BN = 64, or 128 when N > 64) with 4 warps:
// warp 0 lane 0 streams 128 x 64 A and BN x 64 B tiles into shared memory with
// TMA (128-byte swizzle, a ring of 4 stages for BN = 64 and 3 for BN = 128, so
// that two CTAs share an SM), warp 1 lane 0 issues tcgen05.mma (kind::f16,
// M = 128, N = BN, K = 16 per instruction) into a BN-column FP32 accumulator in
// TMEM and commits each stage back to the producer. The wider tile halves the
// re-reads of A from L2. The
// epilogue: all four warps read the accumulator with tcgen05.ld (warp w owns
// rows 32w..32w+31) into a padded shared-memory tile (the operand ring, free
// once the MMAs are done), then write the outputs row by row with consecutive
// threads on consecutive columns (coalesced), applying bias / GELU / GELU'
// there. Every mbarrier wait is bounded: on expiry the CTA sets the error
// flag, skips the remaining work, still frees its TMEM and returns.
#include "internal.cuh"
#include "tcgen05.cuh"
#include "gelu.cuh"
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <math.h>
#include <mutex>

namespace tb {

constexpr int GM_BM = 128, GM_BK = 64;
constexpr int GM_TILE_A = GM_BM * GM_BK * 2;
template <int BN> struct GemmTile {
  static constexpr int STAGES = BN == 64 ? 4 : 3;
  static constexpr int LDS = BN + 1; // padded row of the epilogue staging tile (floats)
  static constexpr int TILE_B = BN * GM_BK * 2;
  static constexpr int SMEM = STAGES * (GM_TILE_A + TILE_B) + 1024 /*align*/ + 256 /*barriers*/;
  static_assert(GM_BM * LDS * 4 <= STAGES * (GM_TILE_A + TILE_B), "staging tile over the ring");
};

struct GemmArgs {
  int M, N, K;
  float *out_f32;           // EPI_F32 / EPI_BIAS_F32: C; EPI_BIAS_GELU: pre-activation Z
  __nv_bfloat16 *out_bf16;  // EPI_BIAS_GELU: GELU(Z); EPI_GELU_BWD: dZ = C * GELU'(Z)
  int ldo;                  // row stride of the outputs (elements)
  const float *bias;        // [N] (bias epilogues)
  const float *aux;         // EPI_GELU_BWD: Z [M][ldo]
  int *err;                 // bit 0 set if a wait expired
};

template <int EPI, int GM_BN>
__global__ void __launch_bounds__(128, 1)
k_gemm_bf16(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
            const __grid_constant__ GemmArgs g) {
  constexpr int GM_STAGES = GemmTile<GM_BN>::STAGES, GM_LDS = GemmTile<GM_BN>::LDS;
  constexpr int GM_TILE_B = GemmTile<GM_BN>::TILE_B;
  extern __shared__ uint8_t gm_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(gm_raw) + 1023) & ~uintptr_t(1023));
  uint8_t *sA = smem;
  uint8_t *sB = smem + GM_STAGES * GM_TILE_A;
  uint64_t *full = reinterpret_cast<uint64_t *>(sB + GM_STAGES * GM_TILE_B);
  uint64_t *empty = full + GM_STAGES;
  uint64_t *done = empty + GM_STAGES;
  uint32_t *taddr_s = reinterpret_cast<uint32_t *>(done + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * GM_BM, n0 = blockIdx.y * GM_BN;
  const int KT = (g.K + GM_BK - 1) / GM_BK;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(taddr_s)), "r"((uint32_t)GM_BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 32) {
    for (int s = 0; s < GM_STAGES; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&full[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&empty[s])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(done)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *taddr_s;

  if (warp == 0 && lane == 0) {
    // TMA producer
    for (int kt = 0; kt < KT; ++kt) {
      const int s = kt % GM_STAGES;
      if (kt >= GM_STAGES && !mbar_wait(smem_u32(&empty[s]), ((kt / GM_STAGES) - 1) & 1)) {
        atomicOr(g.err, 1);
        break;
      }
      const uint32_t fb = smem_u32(&full[s]);
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                   :: "r"(fb), "r"((uint32_t)(GM_TILE_A + GM_TILE_B)) : "memory");
      asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
                   " [%0], [%1, {%2, %3}], [%4];"
                   :: "r"(smem_u32(sA + s * GM_TILE_A)), "l"(reinterpret_cast<uint64_t>(&tmA)),
                      "r"(kt * GM_BK), "r"(m0), "r"(fb) : "memory");
      asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
                   " [%0], [%1, {%2, %3}], [%4];"
                   :: "r"(smem_u32(sB + s * GM_TILE_B)), "l"(reinterpret_cast<uint64_t>(&tmB)),
                      "r"(kt * GM_BK), "r"(n0), "r"(fb) : "memory");
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    constexpr uint32_t idesc = idesc_bf16(GM_BM, GM_BN);
    for (int kt = 0; kt < KT; ++kt) {
      const int s = kt % GM_STAGES;
      if (!mbar_wait(smem_u32(&full[s]), (kt / GM_STAGES) & 1)) { atomicOr(g.err, 1); break; }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint64_t da = sdesc_sw128(smem_u32(sA + s * GM_TILE_A));
      const uint64_t db = sdesc_sw128(smem_u32(sB + s * GM_TILE_B));
#pragma unroll
      for (int ks = 0; ks < GM_BK / 16; ++ks) {
        const uint32_t acc = (kt > 0 || ks > 0) ? 1u : 0u;
        asm volatile("{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                     " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                     :: "r"(tmem), "l"(da + 2 * ks), "l"(db + 2 * ks), "r"(idesc), "r"(acc));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                   :: "r"(smem_u32(&empty[s])) : "memory");
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(smem_u32(done)) : "memory");
  }
  __syncwarp();
  const bool ok = mbar_wait(smem_u32(done), 0);
  asm volatile("tcgen05.fence::after_thread_sync;");
  float *stage = reinterpret_cast<float *>(smem); // [GM_BM][GM_LDS], over the idle operand ring
  if (!ok) {
    if (lane == 0) atomicOr(g.err, 1);
  } else {
    const int r = warp * 32 + lane;
#pragma unroll
    for (int c = 0; c < GM_BN; c += 16) {
      uint32_t v[16];
      const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c;
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,"
                   "%11,%12,%13,%14,%15}, [%16];"
                   : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                     "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
                     "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                   : "r"(ta));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int j = 0; j < 16; ++j) stage[r * GM_LDS + c + j] = __uint_as_float(v[j]);
    }
  }
  const bool all_ok = __syncthreads_and(ok);
  if (all_ok) {
    // consecutive threads on consecutive columns: BN columns x 128 / BN rows per pass
    const int cl = threadIdx.x & (GM_BN - 1), r0 = threadIdx.x / GM_BN;
    const int col = n0 + cl;
    if (col < g.N) {
      const float bias = (EPI == 1 || EPI == 2) ? g.bias[col] : 0.f;
#pragma unroll 4
      for (int rr = r0; rr < GM_BM; rr += 128 / GM_BN) {
        const int row = m0 + rr;
        if (row >= g.M) break;
        const float v = stage[rr * GM_LDS + cl];
        const size_t o = (size_t)row * g.ldo + col;
        if constexpr (EPI == 0) {
          g.out_f32[o] = v;
        } else if constexpr (EPI == 1) {
          const float z = v + bias;
          if (g.out_f32) g.out_f32[o] = z;
          g.out_bf16[o] = __float2bfloat16_rn(gelu_tanh(z));
        } else if constexpr (EPI == 2) {
          g.out_f32[o] = v + bias;
        } else {
          g.out_bf16[o] = __float2bfloat16_rn(v * gelu_tanh_grad(g.aux[o]));
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                 :: "r"(tmem), "r"((uint32_t)GM_BN));
}

// ---- host ----------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess && q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// Row-major BF16 matrix [rows][cols] (cols contiguous, cols % 8 == 0, 16-byte aligned base)
// as a 2D tensor map with 64-column x box_rows boxes and the 128-byte swizzle; out-of-range
// elements of a box read as zero.
static cudaError_t make_map(CUtensorMap *m, const void *ptr, int rows, int cols, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  if ((cols % 8) != 0 || (reinterpret_cast<uintptr_t>(ptr) & 15) != 0) return cudaErrorInvalidValue;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
  cuuint32_t box[2] = {(cuuint32_t)GM_BK, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides,
                  box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_gemm_bf16(int epi, const void *A, const void *B, int M, int N, int K,
                             float *out_f32, void *out_bf16, int ldo, const float *bias,
                             const float *aux, int *err, cudaStream_t s) {
  if (M < 1 || N < 1 || K < 1) return cudaErrorInvalidValue;
  CUtensorMap ma, mb;
  cudaError_t e = make_map(&ma, A, M, K, GM_BM);
  if (e != cudaSuccess) return e;
  GemmArgs g{M, N, K, out_f32, reinterpret_cast<__nv_bfloat16 *>(out_bf16), ldo, bias, aux, err};
  if (epi < 0 || epi > 3) return cudaErrorInvalidValue;
  const int bn = N > 64 ? 128 : 64;
  if ((e = make_map(&mb, B, N, K, bn)) != cudaSuccess) return e;
  dim3 grid((M + GM_BM - 1) / GM_BM, (N + bn - 1) / bn);
  void (*kern)(CUtensorMap, CUtensorMap, GemmArgs) = nullptr;
  int smem = 0;
  if (bn == 64) {
    smem = GemmTile<64>::SMEM;
    kern = epi == 0 ? k_gemm_bf16<0, 64> : epi == 1 ? k_gemm_bf16<1, 64>
         : epi == 2 ? k_gemm_bf16<2, 64> : k_gemm_bf16<3, 64>;
  } else {
    smem = GemmTile<128>::SMEM;
    kern = epi == 0 ? k_gemm_bf16<0, 128> : epi == 1 ? k_gemm_bf16<1, 128>
         : epi == 2 ? k_gemm_bf16<2, 128> : k_gemm_bf16<3, 128>;
  }
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  kern<<<grid, 128, smem, s>>>(ma, mb, g);
  return cudaGetLastError();
}

} // namespace tb

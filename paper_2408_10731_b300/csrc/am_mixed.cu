// am_mixed.cu -- the tensor-core form of the AM iteration (TRAJ_PREC_MIXED).
//
// Same persistent warp-per-trajectory scheme and FP32 state as am_solve.cu, but
// the residual contraction u = F^T r = P^T sum_j r_j + Pd^T r_v + Pdd^T r_a of
// all eight warps of a CTA runs on the 5th-generation tensor cores:
//
//   D[128 x 16] (FP32, TMEM) = A[128 x K] * B[16 x K]^T,   K = 3 n_p padded to 64,
//   A row 32 (w % 4) + 16 (w / 4) + a = warp w's residuals of axis a, BF16:
//                     [sum_j r_j(t) | r_v(t)/T | r_a(t)/T^2]  (warp w can read TMEM lanes
//                     32 (w % 4) .. + 31 only, so each lane quarter holds two warps' rows)
//   B row i         = coefficient i's basis column, BF16: [P(t, i) | dB(t, i) | d2B(t, i)]
//
// Both operands live in shared memory in the K-major 128-byte swizzle layout; the
// CUDA cores write A directly (no TMA: it is produced on chip every iteration),
// fence it into the async proxy, and one elected thread issues K/16
// tcgen05.mma (M = 128, N = 16) and commits to an mbarrier. Warp w reads its
// rows with tcgen05.ld. The warps step their iterations in lock-step (one CTA
// barrier per iteration); a warp whose trajectory ends pulls the next one from
// the queue at once.
//
// Refinement: when an iteration's FP32 residuals meet the tolerance, the warp
// recomputes that iteration's contraction in FP32, redoes the multiplier update
// with it, and runs one more full FP32 iteration; the trajectory is reported
// converged if the refined iterate's FP32 residuals meet the tolerance too
// (otherwise it continues). The reported residuals are always FP32.
#include "internal.cuh"
#include "am_device.cuh"
#include "tcgen05.cuh"
#include <cuda_bf16.h>

namespace tb {

constexpr int MX_WARPS = 8;
constexpr int MX_TILE_A = 128 * 128; // bytes of one 128-row x 64-column BF16 tile
constexpr int MX_TILE_B = 16 * 128;  // bytes of one 16-row x 64-column BF16 tile

__host__ __device__ inline int mixed_kt(int n_p) { return (3 * n_p + 63) / 64; }
__host__ __device__ inline size_t mixed_smem(int n_p, int table_floats) {
  return 1024 + (size_t)mixed_kt(n_p) * (MX_TILE_A + MX_TILE_B) + sizeof(float) * table_floats + 64;
}

template <int DIM>
__device__ __forceinline__ void broadcast_xi(float xo, float xo2, float (&xa)[DIM][NC]) {
#pragma unroll
  for (int i = 0; i < NC; ++i) {
    xa[0][i] = __shfl_sync(FULL, xo, i);
    xa[1][i] = __shfl_sync(FULL, xo, 16 + i);
    if constexpr (DIM == 3) xa[2][i] = __shfl_sync(FULL, xo2, i);
  }
}

// xi^k = hq + G xi^{k-1} + K11 (lambda - rho u) at the owner lanes (compensated FP32)
template <int DIM>
__device__ __forceinline__ void xi_step(const float *C, int lane, float rho, float hq_hi,
                                        float hq_lo, float hq2_hi, float hq2_lo, float lam,
                                        float lam2, float uo, float uo2, float &xo, float &xo2) {
  const int oi = lane & 15;
  const int ri = oi < NC ? oi : NC - 1;
  const float vo = lam - rho * uo, vo2 = lam2 - rho * uo2;
  float hi = hq_hi, lo = hq_lo, hi2 = hq2_hi, lo2 = hq2_lo;
  const float x_own = xo, x_own2 = xo2;
#pragma unroll
  for (int q = 0; q < NC; ++q) {
    const float xk = __shfl_sync(FULL, x_own, (lane & 16) + q);
    const float vk = __shfl_sync(FULL, vo, (lane & 16) + q);
    const float g_hi = C[C_G_HI + ri * ROW + q], g_lo = C[C_G_LO + ri * ROW + q];
    const float k_hi = C[C_K11_HI + ri * ROW + q], k_lo = C[C_K11_LO + ri * ROW + q];
    df_fma(hi, lo, g_hi, g_lo, xk);
    df_fma(hi, lo, k_hi, k_lo, vk);
    if constexpr (DIM == 3) {
      const float xk2 = __shfl_sync(FULL, x_own2, q);
      const float vk2 = __shfl_sync(FULL, vo2, q);
      df_fma(hi2, lo2, g_hi, g_lo, xk2);
      df_fma(hi2, lo2, k_hi, k_lo, vk2);
    }
  }
  xo = hi + lo;
  if constexpr (DIM == 3) xo2 = hi2 + lo2;
}

template <int DIM>
__device__ __forceinline__ void scatter_u(float (&up)[DIM][NC], int lane, float &uo, float &uo2) {
  float v32[32];
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    v32[i] = i < NC ? up[0][i] : 0.f;
    v32[16 + i] = i < NC ? up[1][i] : 0.f;
  }
  uo = reduce_scatter32(v32, lane);
  if constexpr (DIM == 3) {
    float v16[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) v16[i] = i < NC ? up[2][i] : 0.f;
    uo2 = reduce_scatter16(v16, lane);
  }
}

template <int DIM, int NT>
__global__ void __launch_bounds__(MX_WARPS * 32) k_am_mixed(const __grid_constant__ SolveArgs A) {
  extern __shared__ uint8_t mx_raw[];
  uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(mx_raw) + 1023) & ~uintptr_t(1023));
  const int n_p = A.problems[0].n_p; // one horizon per batch in this form (checked on the host)
  const int KT = mixed_kt(n_p);
  uint8_t *sA = base;
  uint8_t *sB = sA + KT * MX_TILE_A;
  float *stab = reinterpret_cast<float *>(sB + KT * MX_TILE_B);
  uint64_t *mbar = reinterpret_cast<uint64_t *>(stab + A.table_floats_total);
  uint32_t *taddr_s = reinterpret_cast<uint32_t *>(mbar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  {
    const float4 *g4 = reinterpret_cast<const float4 *>(A.tables);
    float4 *s4 = reinterpret_cast<float4 *>(stab);
    for (int i = tid; i < A.table_floats_total / 4; i += blockDim.x) s4[i] = g4[i];
    uint4 *a4 = reinterpret_cast<uint4 *>(sA);
    for (int i = tid; i < KT * MX_TILE_A / 16; i += blockDim.x) a4[i] = make_uint4(0, 0, 0, 0);
  }
  __syncthreads();
  {
    const int tbl = A.problems[0].tbl_off;
    for (int e = tid; e < 16 * KT * 64; e += blockDim.x) {
      const int i = e / (KT * 64), k = e % (KT * 64);
      float v = 0.f;
      if (i < NC && k < 3 * n_p) v = stab[tbl + ((k / n_p) * n_p + (k % n_p)) * ROW + i];
      *reinterpret_cast<__nv_bfloat16 *>(sB + (k >> 6) * MX_TILE_B + sw128_offset(i, k & 63)) =
          __float2bfloat16_rn(v);
    }
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(taddr_s)), "r"(32u));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 32) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *taddr_s;

  unsigned long long deadline = 0;
  if (A.timeout_ns) {
    unsigned long long t0 = 0;
    if (lane == 0) {
      const unsigned long long now = globaltimer_ns();
      const unsigned long long prev = atomicCAS(A.t0, 0ull, now);
      t0 = prev ? prev : now;
    }
    deadline = __shfl_sync(FULL, t0, 0) + A.timeout_ns;
  }

  const int oi = lane & 15, oa = lane >> 4;
  const int ri = oi < NC ? oi : NC - 1;
  const float rho = A.rho;
  const int row0 = 32 * (warp & 3) + 16 * (warp >> 2); // this warp's first A row / TMEM lane
  // per-warp trajectory state
  int b = -1, k = 0;
  bool qdone = false, dirty = false;
  const float *C = nullptr;
  const float4 *obs = nullptr;
  int n_o = 0;
  float dt = 0.f, invT = 0.f, invT2 = 0.f;
  float xo = 0.f, xo2 = 0.f, lam = 0.f, lam2 = 0.f, uo = 0.f, uo2 = 0.f;
  float hq_hi = 0.f, hq_lo = 0.f, hq2_hi = 0.f, hq2_lo = 0.f;
  uint32_t phase = 0;
  const float *tP = stab + A.problems[0].tbl_off, *tD = tP + n_p * ROW, *tA = tD + n_p * ROW;
  const uint32_t idesc = idesc_bf16(128, 16);

  for (;;) {
    if (b < 0 && !qdone) {
      int item = 0;
      if (lane == 0) item = atomicAdd(A.queue, 1);
      item = __shfl_sync(FULL, item, 0);
      if (item >= A.n_traj) {
        qdone = true;
      } else {
        b = A.order[item];
        const ProblemDev pr = A.problems[A.traj_problem[b]];
        C = A.constants + pr.const_off;
        obs = A.obstacles + (size_t)pr.obs_off * obs_vec(DIM);
        n_o = pr.n_o; dt = pr.dt; invT = pr.invT; invT2 = pr.invT2;
        const float *x0 = A.xi0 + (size_t)b * DIM * NC;
        xo = x0[oa * NC + ri];
        xo2 = DIM == 3 ? x0[2 * NC + ri] : 0.f;
        bool finite = isfinite(xo) && isfinite(xo2);
        finite = __all_sync(FULL, finite) && pr.nan_flag == 0;
        if (!finite) {
          float *xout = A.xi + (size_t)b * DIM * NC;
          if (oi < NC) {
            xout[oa * NC + oi] = xo;
            if (DIM == 3 && oa == 0) xout[2 * NC + oi] = xo2;
          }
          if (lane < 3) A.res[b * 3 + lane] = __int_as_float(0x7fc00000);
          if (lane == 0) { A.iters[b] = 0; A.status[b] = 2; atomicOr(A.flags, 2); }
          b = -1;
        } else {
          if (A.cost_mode == 0) {
            hq_hi = C[C_HQ_HI + oa * ROW + ri]; hq_lo = C[C_HQ_LO + oa * ROW + ri];
            if (DIM == 3) { hq2_hi = C[C_HQ_HI + 2 * ROW + ri]; hq2_lo = C[C_HQ_LO + 2 * ROW + ri]; }
          } else {
            hq_hi = C[C_C_HI + oa * ROW + ri]; hq_lo = C[C_C_LO + oa * ROW + ri];
            if (DIM == 3) { hq2_hi = C[C_C_HI + 2 * ROW + ri]; hq2_lo = C[C_C_LO + 2 * ROW + ri]; }
#pragma unroll
            for (int q = 0; q < NC; ++q) {
              const float xk = __shfl_sync(FULL, xo, (lane & 16) + q);
              df_fma(hq_hi, hq_lo, C[C_K11_HI + ri * ROW + q], C[C_K11_LO + ri * ROW + q], xk);
              if (DIM == 3) {
                const float xk2 = __shfl_sync(FULL, xo2, q);
                df_fma(hq2_hi, hq2_lo, C[C_K11_HI + ri * ROW + q], C[C_K11_LO + ri * ROW + q], xk2);
              }
            }
            float s = hq_hi + hq_lo; hq_lo = hq_lo - (s - hq_hi); hq_hi = s;
            if (DIM == 3) { float s2 = hq2_hi + hq2_lo; hq2_lo = hq2_lo - (s2 - hq2_hi); hq2_hi = s2; }
          }
          lam = lam2 = uo = uo2 = 0.f;
          k = 0;
        }
      }
    }
    const bool active = b >= 0;
    float Ro[NT][DIM], Rv[NT][DIM], Ra[NT][DIM], xa[DIM][NC];
    float mo = 0.f, mv = 0.f, ma = 0.f;
    if (active) {
      if (k > 0) xi_step<DIM>(C, lane, rho, hq_hi, hq_lo, hq2_hi, hq2_lo, lam, lam2, uo, uo2, xo, xo2);
      broadcast_xi<DIM>(xo, xo2, xa);
      project_only<DIM, NT>(xa, tP, tD, tA, obs, n_o, n_p, dt, invT, invT2, A.vmax, A.amax, lane,
                            Ro, Rv, Ra, mo, mv, ma);
#pragma unroll
      for (int m = 0; m < NT; ++m) {
        const int t = lane + 32 * m;
        if (t < n_p) {
#pragma unroll
          for (int a = 0; a < DIM; ++a) {
            const int row = row0 + a;
            const float vals[3] = {Ro[m][a], Rv[m][a], Ra[m][a]};
#pragma unroll
            for (int g = 0; g < 3; ++g) {
              const int kk = g * n_p + t;
              *reinterpret_cast<__nv_bfloat16 *>(sA + (kk >> 6) * MX_TILE_A + sw128_offset(row, kk & 63)) =
                  __float2bfloat16_rn(vals[g]);
            }
          }
        }
      }
      dirty = true;
    } else if (dirty) { // an idle warp contributes zero rows
      for (int e = lane; e < DIM * KT * 64; e += 32) {
        const int a = e / (KT * 64), kk = e % (KT * 64);
        *reinterpret_cast<__nv_bfloat16 *>(sA + (kk >> 6) * MX_TILE_A + sw128_offset(row0 + a, kk & 63)) =
            __float2bfloat16_rn(0.f);
      }
      dirty = false;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      for (int j = 0; j < KT; ++j) {
        const uint64_t da = sdesc_sw128(smem_u32(sA + j * MX_TILE_A));
        const uint64_t db = sdesc_sw128(smem_u32(sB + j * MX_TILE_B));
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
          const uint32_t acc = (j > 0 || ks > 0) ? 1u : 0u;
          asm volatile("{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                       " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                       :: "r"(tmem), "l"(da + 2 * ks), "l"(db + 2 * ks), "r"(idesc), "r"(acc));
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                   :: "r"(smem_u32(mbar)) : "memory");
    }
    const bool waited = mbar_wait(smem_u32(mbar), phase);
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;");
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,"
                 "%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                   "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                   "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(tmem + ((uint32_t)(32 * (warp & 3)) << 16)));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    if (!__syncthreads_and(waited)) { // the MMA never completed: give up on this CTA's work
      if (tid == 0) atomicOr(A.flags, 8);
      break;
    }
    if (active) {
      // lane 16 a + i takes coefficient i of axis a from the lane of row row0 + a
      float un = 0.f, un2 = 0.f;
      const int src = 16 * (warp >> 2);
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const float v0 = __shfl_sync(FULL, __uint_as_float(r[c]), src + oa);
        if (oi == c) un = v0;
        if constexpr (DIM == 3) {
          const float v2 = __shfl_sync(FULL, __uint_as_float(r[c]), src + 2);
          if (oi == c) un2 = v2;
        }
      }
      mo = warp_max(mo); mv = warp_max(mv); ma = warp_max(ma);
      signed char st = -1;
      if (k == 0) {
        uo = un; uo2 = un2;
      } else {
        const bool under = A.tol >= 0.f && sqrtf(mo) <= A.tol && sqrtf(mv) <= A.tol && sqrtf(ma) <= A.tol;
        if (!under) {
          lam -= rho * un; lam2 -= rho * un2;
          uo = un; uo2 = un2;
        } else {
          // refinement pass: this iteration's contraction in FP32, then one FP32 iteration
          float up[DIM][NC];
          contract_fp32<DIM, NT>(Ro, Rv, Ra, tP, tD, tA, n_p, lane, up);
          scatter_u<DIM>(up, lane, uo, uo2);
          lam -= rho * uo; lam2 -= rho * uo2;
          xi_step<DIM>(C, lane, rho, hq_hi, hq_lo, hq2_hi, hq2_lo, lam, lam2, uo, uo2, xo, xo2);
          ++k;
          broadcast_xi<DIM>(xo, xo2, xa);
          project_contract<DIM, NT>(xa, tP, tD, tA, obs, n_o, n_p, NT, dt, invT, invT2, A.vmax,
                                    A.amax, lane, up, mo, mv, ma);
          scatter_u<DIM>(up, lane, uo, uo2);
          mo = warp_max(mo); mv = warp_max(mv); ma = warp_max(ma);
          lam -= rho * uo; lam2 -= rho * uo2;
          if (sqrtf(mo) <= A.tol && sqrtf(mv) <= A.tol && sqrtf(ma) <= A.tol) st = 0;
        }
      }
      if (st < 0 && k >= A.max_iters) st = 1;
      if (st < 0 && deadline) {
        unsigned long long now = 0;
        if (lane == 0) now = globaltimer_ns();
        now = __shfl_sync(FULL, now, 0);
        if (now > deadline) st = 3;
      }
      if (st >= 0) {
        float *xout = A.xi + (size_t)b * DIM * NC;
        if (oi < NC) {
          xout[oa * NC + oi] = xo;
          if (A.lam) A.lam[(size_t)b * DIM * NC + oa * NC + oi] = lam;
          if (A.u) A.u[(size_t)b * DIM * NC + oa * NC + oi] = uo;
          if (DIM == 3 && oa == 0) {
            xout[2 * NC + oi] = xo2;
            if (A.lam) A.lam[(size_t)b * DIM * NC + 2 * NC + oi] = lam2;
            if (A.u) A.u[(size_t)b * DIM * NC + 2 * NC + oi] = uo2;
          }
        }
        if (lane == 0) {
          A.res[b * 3 + 0] = sqrtf(mo);
          A.res[b * 3 + 1] = sqrtf(mv);
          A.res[b * 3 + 2] = sqrtf(ma);
          A.iters[b] = k;
          A.status[b] = st;
          if (st == 3) atomicOr(A.flags, 1);
        }
        b = -1;
      } else {
        ++k;
      }
    }
    if (!__syncthreads_or(b >= 0 || !qdone)) break;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(32u));
}

template <int DIM, int NT>
static cudaError_t launch_mx(const SolveArgs &a, int n_p, int n_sm, cudaStream_t s) {
  auto kern = k_am_mixed<DIM, NT>;
  const size_t smem = mixed_smem(n_p, a.table_floats_total);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, MX_WARPS * 32, smem);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  long long grid = (long long)n_sm * occ, want = ((long long)a.n_traj + MX_WARPS - 1) / MX_WARPS;
  if (want < grid) grid = want;
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, MX_WARPS * 32, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_am_mixed(int dim, int n_p, const SolveArgs &a, int n_sm, cudaStream_t s) {
  const int nt = (n_p + 31) / 32;
  if (mixed_smem(n_p, a.table_floats_total) > 227 * 1024) return cudaErrorInvalidValue;
  if (dim == 2) {
    if (nt <= 2) return launch_mx<2, 2>(a, n_p, n_sm, s);
    if (nt <= 4) return launch_mx<2, 4>(a, n_p, n_sm, s);
    if (nt <= 5) return launch_mx<2, 5>(a, n_p, n_sm, s);
    return launch_mx<2, 8>(a, n_p, n_sm, s);
  }
  if (nt <= 2) return launch_mx<3, 2>(a, n_p, n_sm, s);
  if (nt <= 4) return launch_mx<3, 4>(a, n_p, n_sm, s);
  if (nt <= 5) return launch_mx<3, 5>(a, n_p, n_sm, s);
  return launch_mx<3, 8>(a, n_p, n_sm, s);
}

} // namespace tb

// am_mixed.cu -- the tensor-core form of the AM iteration (TRAJ_PREC_MIXED and
// TRAJ_PREC_MIXED_SPLIT).
//
// Same persistent warp-per-trajectory scheme and FP32 state as am_solve.cu, but
// the residual contraction u_a = F^T r_a = P^T sum_j r_j + Pd^T r_v + Pdd^T r_a
// (Algorithm 2 line 6) of each warp's trajectory runs on the 5th-generation
// tensor cores, every warp on its own (no CTA barrier inside the iteration):
//
//   D_w[128 x N] (FP32, TMEM columns N w ..) = A_h[128 x K] * B_w[N x K]^T,
//   K = n_p padded to a multiple of 16 (contraction over the timesteps),
//   A_h rows 32 q + r of every quarter q (warp w may only read TMEM lanes
//                  32 (w % 4) .. + 31, so the 32 rows are repeated per quarter), BF16,
//                  one copy per distinct horizon h of the batch:
//                  r = i < 11: P(t, i); r = 11 + i: dB(t, i); r = 22 + i (i < 10): d2B(t, i),
//   B_w row g dim + a = warp w's residual group g of axis a, BF16:
//                  g = 0: sum_j r_j(t); 1: r_v(t) / T; 2: r_a(t) / T^2;
//                  3: r_a(n_p - 1 - t) / T^2 (time-reversed), other rows zero,
//   so that u_a[i] = D[i][a] + D[11 + i][dim + a] + D[22 + i][2 dim + a] (i < 10) and
//   u_a[10] = D[0][a] + ... : the last column of d2B is the time-reversed first one
//   (d2B_10(tau) = d2B_0(1 - tau) on the symmetric grid tau_t = t / (n_p - 1)),
//   whence its term D[22][3 dim + a]. Packing the three basis groups along M keeps
//   K at n_p: ceil(n_p / 16) MMAs per iteration (7 at n_p = 100).
//
// Split operands (TRAJ_PREC_MIXED_SPLIT): every BF16 operand x is stored as a pair
// hi = bf16(x), lo = bf16(x - hi), which together carry 16 significant bits. The
// residual's lo part rides in the rows of B_w past the hi rows (2D: rows 8-15 of the
// same N = 16; 3D: N = 32, lo rows from 16), and the basis's lo part is a second A
// tile set whose MMAs accumulate into the same D: D = A_hi B^T + A_lo B^T, twice the
// MMAs, and u = D[hi columns] + D[lo columns]. Only the product of the two lo parts
// is dropped (relative 2^-18).
//
// A_h is written once per CTA, for every distinct horizon of the batch (uneven
// batches run in this one launch; each trajectory's MMAs read its horizon's A and
// run its own K). Per iteration a warp writes its B_w rows (the columns between n_p
// and K are cleared once per trajectory), fences them into the async proxy, and its lane 0 issues the tcgen05.mma
// (kind::f16, M = 128, N = 16 or 32) and commits to the warp's own mbarrier; while
// the MMAs run the warp reduces its residual maxima, then reads its columns with
// tcgen05.ld and sums the three groups with shuffles. Both operands live in shared
// memory in the K-major 128-byte swizzle layout.
//
// Refinement: when an iteration's residuals meet the tolerance, the warp
// recomputes that iteration's contraction in FP32, redoes the multiplier update
// with it, and runs one more full FP32 iteration; the trajectory is reported
// converged if the refined iterate's FP32 residuals meet the tolerance too
// (otherwise it continues). The reported residuals are always FP32.
#include "internal.cuh"
#include "am_device.cuh"
#include "tcgen05.cuh"
#include <cuda_bf16.h>
#include <algorithm>

namespace tb {

constexpr int MX_MAX_WARPS = 8;  // registers unrestricted: one block of up to 8 warps
constexpr int MX_CAP_WARPS = 6;  // the occupancy build: 170 registers, two blocks of up to 6
constexpr int MX_TILE_A = 128 * 128; // bytes of one 128-row x 64-column BF16 tile

__host__ __device__ inline int mixed_kp(int n_p) { return (n_p + 15) & ~15; }       // K
__host__ __device__ inline int mixed_kt(int n_p) { return (mixed_kp(n_p) + 63) / 64; } // 64-wide tiles
// B_w rows (N of the MMA), the first lo row, and B_w's bytes per 64-wide K tile
__host__ __device__ constexpr int mixed_n(int dim, bool split) { return dim == 3 && split ? 32 : 16; }
__host__ __device__ constexpr int mixed_lo_row(int dim) { return dim == 2 ? 8 : 16; }
__host__ __device__ constexpr int mixed_tile_b(int dim, bool split) { return mixed_n(dim, split) * 128; }

// Bytes of the A tiles of every distinct horizon, and the largest K tile count.
__host__ __device__ inline size_t mixed_a_bytes(const SolveArgs &a, bool split, int *kt_max) {
  size_t s = 0;
  int m = 1;
  for (int h = 0; h < a.hz_n; ++h) {
    const int kt = mixed_kt(a.hz_np[h]);
    s += (size_t)kt * (split ? 2 : 1) * MX_TILE_A;
    m = kt > m ? kt : m;
  }
  if (kt_max) *kt_max = m;
  return s;
}
__host__ __device__ inline size_t mixed_smem(const SolveArgs &a, int dim, bool split, int warps) {
  int ktm = 1;
  const size_t sa = mixed_a_bytes(a, split, &ktm);
  return 1024 + sa + (size_t)warps * ktm * mixed_tile_b(dim, split) +
         sizeof(float) * a.table_floats_total + 8 * MX_MAX_WARPS + 16;
}
__host__ __device__ inline uint32_t mixed_tmem_cols(int warps, int ncol) {
  uint32_t c = 32;
  while (c < (uint32_t)(ncol * warps)) c <<= 1;
  return c;
}

// Per-warp constants of the MMA path.
struct MxWarp {
  uint8_t *sA;     // all A tiles (horizon h after those of the horizons before it)
  uint8_t *myB;    // this warp's B_w tiles
  uint32_t mbar;   // this warp's mbarrier
  uint32_t d_col;  // MMA destination column
  uint32_t d_read; // this warp's quarter, same columns
  uint32_t phase;  // mbarrier parity
};

// One trajectory of the tensor-core form. Returns false if an MMA wait expired (the
// warp then leaves its work: the launch is flagged).
template <int DIM, int NT, bool SPLIT>
__device__ __forceinline__ bool mixed_one(const SolveArgs &A, int b, const float *stab, int lane,
                                          unsigned long long deadline, MxWarp &W) {
  constexpr int N = mixed_n(DIM, SPLIT), LO = mixed_lo_row(DIM), TB = mixed_tile_b(DIM, SPLIT);
  const ProblemDev *prp = A.problems + A.traj_problem[b];
  const ProblemDev pr = *prp;
  const int n_p = pr.n_p, KP = mixed_kp(n_p), n_k16 = KP / 16, KT = mixed_kt(n_p);
  // this horizon's A tiles
  size_t a_off = 0;
  for (int h = 0; h < A.hz_n; ++h) {
    if (A.hz_tbl[h] == pr.tbl_off) break;
    a_off += (size_t)mixed_kt(A.hz_np[h]) * (SPLIT ? 2 : 1) * MX_TILE_A;
  }
  const uint8_t *sAh = W.sA + a_off, *sAl = sAh + (size_t)KT * MX_TILE_A;
  const float *tP = stab + pr.tbl_off, *tD = tP + n_p * ROW, *tA = tD + n_p * ROW;
  const float *Cb = A.constants + pr.const_off, *C = Cb;
  const float4 *obs = A.obstacles + (size_t)pr.pair_off * pair_vec(DIM);
  const int oi = lane & 15, oa = lane >> 4;
  const int ri = oi < NC ? oi : NC - 1;
  const float *x0 = A.xi0 + (size_t)b * DIM * NC;
  float xo = x0[oa * NC + ri];
  float xo2 = DIM == 3 ? x0[2 * NC + ri] : 0.f;
  bool finite = isfinite(xo) && isfinite(xo2);
  finite = __all_sync(FULL, finite) && pr.nan_flag == 0;
  float *xout = A.xi + (size_t)b * DIM * NC;
  if (!finite) {
    if (oi < NC) {
      xout[oa * NC + oi] = xo;
      if (DIM == 3 && oa == 0) xout[2 * NC + oi] = xo2;
    }
    if (lane < 3) A.res[b * 3 + lane] = __int_as_float(0x7fc00000);
    if (lane == 0) { A.iters[b] = 0; A.status[b] = 2; atomicOr(A.flags, 2); }
    return true;
  }
  const float xs = xo, xs2 = xo2;
  float hq_hi, hq_lo, hq2_hi, hq2_lo;
  load_hq<DIM>(C, A.cost_mode, lane, xs, xs2, hq_hi, hq_lo, hq2_hi, hq2_lo);
  int level = 0;
  float rho = A.rho;
  float lam = 0.f, lam2 = 0.f, uo = 0.f, uo2 = 0.f;
  float mo = 0.f, mv = 0.f, ma = 0.f;
  signed char st = -1;
  int k = 0;
  if (A.lam0) {
    resume_state<DIM>(A, b, oa, ri, lam, lam2, uo, uo2);
    k = A.u0 ? 1 : 0; // resume: the next step is a QP step; carry: project first
  }
  const uint32_t idesc = idesc_bf16(128, N);
  // B_w columns between n_p and K (read by the last MMA, against zero A columns) are
  // cleared once: earlier trajectories of this warp may have left values there
  for (int t = n_p + lane; t < KP; t += 32)
#pragma unroll
    for (int r = 0; r < N; ++r)
      *reinterpret_cast<__nv_bfloat16 *>(W.myB + (t >> 6) * TB + sw128_offset(r, t & 63)) =
          __float2bfloat16_rn(0.f);
  for (;; ++k) {
    if (k > 0) qp_step<DIM>(C, lane, rho, hq_hi, hq_lo, hq2_hi, hq2_lo, lam, lam2, uo, uo2, xo, xo2);
    {
      float2 xp[DIM][6];
      broadcast_pairs<DIM>(xo, xo2, xp);
      float Ro[NT][DIM], Rv[NT][DIM], Ra[NT][DIM];
      project_only<DIM, NT>(xp, tP, tD, tA, obs, prp, n_p, pr.dt, pr.invT, pr.invT2, A.vmax,
                            A.amax, lane, Ro, Rv, Ra, mo, mv, ma);
      // this warp's B rows g dim + a at k = t (group 3: k = n_p - 1 - t)
#pragma unroll
      for (int m = 0; m < NT; ++m) {
        const int t = lane + 32 * m;
        if (t < n_p) {
#pragma unroll
          for (int a = 0; a < DIM; ++a) {
            const float vals[4] = {Ro[m][a], Rv[m][a], Ra[m][a], Ra[m][a]};
#pragma unroll
            for (int g = 0; g < 4; ++g) {
              const int kk = g < 3 ? t : n_p - 1 - t;
              const float v = vals[g];
              const __nv_bfloat16 hi = __float2bfloat16_rn(v);
              uint8_t *tile = W.myB + (kk >> 6) * TB;
              *reinterpret_cast<__nv_bfloat16 *>(tile + sw128_offset(g * DIM + a, kk & 63)) = hi;
              if constexpr (SPLIT)
                *reinterpret_cast<__nv_bfloat16 *>(tile + sw128_offset(LO + g * DIM + a, kk & 63)) =
                    __float2bfloat16_rn(v - __bfloat162float(hi));
            }
          }
        }
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncwarp();
    if (lane == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      for (int s16 = 0; s16 < n_k16; ++s16) {
        const int j = s16 >> 2, ks = s16 & 3;
        const uint64_t db = sdesc_sw128(smem_u32(W.myB + j * TB)) + 2 * ks;
        const uint64_t da = sdesc_sw128(smem_u32(sAh + j * MX_TILE_A)) + 2 * ks;
        const uint32_t acc = s16 > 0 ? 1u : 0u;
        asm volatile("{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                     " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                     :: "r"(W.d_col), "l"(da), "l"(db), "r"(idesc), "r"(acc));
        if constexpr (SPLIT) {
          const uint64_t dl = sdesc_sw128(smem_u32(sAl + j * MX_TILE_A)) + 2 * ks;
          asm volatile("{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                       " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                       :: "r"(W.d_col), "l"(dl), "l"(db), "r"(idesc), "r"(1u));
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                   :: "r"(W.mbar) : "memory");
    }
    __syncwarp();
    mo = warp_max(mo); mv = warp_max(mv); ma = warp_max(ma); // while the MMAs run
    const bool waited = __all_sync(FULL, mbar_wait(W.mbar, W.phase));
    W.phase ^= 1u;
    if (!waited) { // the MMA never completed: give up on this warp's work
      if (lane == 0) { A.iters[b] = k; A.status[b] = 3; atomicOr(A.flags, 8); }
      return false;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // s[c] = D[lane][c] (+ D[lane][LO + c] in the split form), c < 4 dim
    float s[4 * DIM];
    {
      uint32_t r[8], r2[4] = {0u, 0u, 0u, 0u};
      uint32_t l[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u}, l2[4] = {0u, 0u, 0u, 0u};
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                   : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                     "=r"(r[6]), "=r"(r[7])
                   : "r"(W.d_read));
      if constexpr (DIM == 3)
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(r2[0]), "=r"(r2[1]), "=r"(r2[2]), "=r"(r2[3]) : "r"(W.d_read + 8u));
      if constexpr (SPLIT) {
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                     : "=r"(l[0]), "=r"(l[1]), "=r"(l[2]), "=r"(l[3]), "=r"(l[4]), "=r"(l[5]),
                       "=r"(l[6]), "=r"(l[7])
                     : "r"(W.d_read + (uint32_t)LO));
        if constexpr (DIM == 3)
          asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                       : "=r"(l2[0]), "=r"(l2[1]), "=r"(l2[2]), "=r"(l2[3])
                       : "r"(W.d_read + (uint32_t)LO + 8u));
      }
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
#pragma unroll
      for (int c = 0; c < 4 * DIM; ++c) {
        s[c] = __uint_as_float(c < 8 ? r[c] : r2[c - 8]);
        if constexpr (SPLIT) s[c] += __uint_as_float(c < 8 ? l[c] : l2[c - 8]);
      }
    }
    // lane l holds row l of the quarter: its basis group's column per axis (v), and
    // lane 22 also the time-reversed term of column 10; lane 16 a + i sums u_a[i]
    float uax[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      const float v = lane < NC ? s[a] : (lane < 2 * NC ? s[DIM + a] : s[2 * DIM + a]);
      const float s1 = __shfl_sync(FULL, v, ri);
      const float s2 = __shfl_sync(FULL, v, NC + ri);
      const float s3 = __shfl_sync(FULL, v, 2 * NC + (ri < NC - 1 ? ri : 0));
      const float s4 = __shfl_sync(FULL, s[3 * DIM + a], 2 * NC);
      uax[a] = (s1 + s2) + (ri < NC - 1 ? s3 : s4);
    }
    const float un = oa ? uax[1] : uax[0];
    const float un2 = DIM == 3 ? uax[2] : 0.f;
    if (k == 0) {
      uo = un; uo2 = un2;
    } else {
      const bool under = A.tol >= 0.f && sqrtf(mo) <= A.tol && sqrtf(mv) <= A.tol && sqrtf(ma) <= A.tol;
      if (!under) {
        lam -= rho * un; lam2 -= rho * un2;
        uo = un; uo2 = un2;
      } else {
        // refinement pass: this iteration's contraction in FP32 (its residuals formed
        // again from the same iterate), then one FP32 iteration
        float2 xp[DIM][6];
        broadcast_pairs<DIM>(xo, xo2, xp);
        float2 up[DIM][6];
        {
          float Ro[NT][DIM], Rv[NT][DIM], Ra[NT][DIM];
          float m0, m1, m2;
          project_only<DIM, NT>(xp, tP, tD, tA, obs, prp, n_p, pr.dt, pr.invT, pr.invT2, A.vmax,
                                A.amax, lane, Ro, Rv, Ra, m0, m1, m2);
          contract_fp32<DIM, NT>(Ro, Rv, Ra, tP, tD, tA, n_p, lane, up);
        }
        scatter_pairs<DIM>(up, lane, uo, uo2);
        lam -= rho * uo; lam2 -= rho * uo2;
        qp_step<DIM>(C, lane, rho, hq_hi, hq_lo, hq2_hi, hq2_lo, lam, lam2, uo, uo2, xo, xo2);
        ++k;
        broadcast_pairs<DIM>(xo, xo2, xp);
        project_contract<DIM, NT, true>(xp, tP, tD, tA, obs, prp, n_p, NT, pr.dt, pr.invT,
                                  pr.invT2, A.vmax, A.amax, lane, up, mo, mv, ma);
        scatter_pairs<DIM>(up, lane, uo, uo2);
        mo = warp_max(mo); mv = warp_max(mv); ma = warp_max(ma);
        lam -= rho * uo; lam2 -= rho * uo2;
        if (sqrtf(mo) <= A.tol && sqrtf(mv) <= A.tol && sqrtf(ma) <= A.tol) { st = 0; break; }
      }
    }
    if (k >= A.max_iters) { st = 1; break; }
    if (deadline) {
      unsigned long long now = 0;
      if (lane == 0) now = globaltimer_ns();
      now = __shfl_sync(FULL, now, 0);
      if (now > deadline) { st = 3; break; }
    }
    rho_step<DIM>(A, k, level, Cb, C, rho, lane, xs, xs2, hq_hi, hq_lo, hq2_hi, hq2_lo);
  }
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
  return true;
}

// Per-trajectory specialisation on the number of 32-step slots, in the steps 2, 4, 5
// and 8 (short horizons of an uneven batch do not pay for the longest one's).
template <int DIM, int MAXNT, bool SPLIT>
__device__ __forceinline__ bool mixed_nt(const SolveArgs &A, int b, const float *stab, int lane,
                                         unsigned long long deadline, MxWarp &W, int nt) {
  if constexpr (MAXNT > 2)
    if (nt <= 2) return mixed_one<DIM, 2, SPLIT>(A, b, stab, lane, deadline, W);
  if constexpr (MAXNT > 4)
    if (nt <= 4) return mixed_one<DIM, 4, SPLIT>(A, b, stab, lane, deadline, W);
  if constexpr (MAXNT > 5)
    if (nt <= 5) return mixed_one<DIM, 5, SPLIT>(A, b, stab, lane, deadline, W);
  return mixed_one<DIM, MAXNT, SPLIT>(A, b, stab, lane, deadline, W);
}

template <int DIM, int MAXNT, bool SPLIT, bool CAP = false>
__global__ void __launch_bounds__(CAP ? MX_CAP_WARPS * 32 : MX_MAX_WARPS * 32, CAP ? 2 : 1)
k_am_mixed(const __grid_constant__ SolveArgs A) {
  constexpr int N = mixed_n(DIM, SPLIT), TB = mixed_tile_b(DIM, SPLIT);
  extern __shared__ uint8_t mx_raw[];
  uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(mx_raw) + 1023) & ~uintptr_t(1023));
  const int nw = blockDim.x >> 5;
  int ktm = 1;
  const size_t a_bytes = mixed_a_bytes(A, SPLIT, &ktm);
  uint8_t *sA = base;
  uint8_t *sB = sA + a_bytes;
  float *stab = reinterpret_cast<float *>(sB + (size_t)nw * ktm * TB);
  uint64_t *mbar = reinterpret_cast<uint64_t *>(stab + A.table_floats_total);
  uint32_t *taddr_s = reinterpret_cast<uint32_t *>(mbar + MX_MAX_WARPS);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t tcols = mixed_tmem_cols(nw, N);

  {
    const float4 *g4 = reinterpret_cast<const float4 *>(A.tables);
    float4 *s4 = reinterpret_cast<float4 *>(stab);
    for (int i = tid; i < A.table_floats_total / 4; i += blockDim.x) s4[i] = g4[i];
    uint4 *z4 = reinterpret_cast<uint4 *>(sB);
    for (int i = tid; i < nw * ktm * TB / 16; i += blockDim.x) z4[i] = make_uint4(0, 0, 0, 0);
  }
  __syncthreads();
  // A of every distinct horizon (zero past its n_p), hi tiles then lo tiles
  {
    size_t off = 0;
    for (int h = 0; h < A.hz_n; ++h) {
      const int n_p = A.hz_np[h], KT = mixed_kt(n_p);
      const float *tb = stab + A.hz_tbl[h];
      uint8_t *Ah = sA + off, *Al = Ah + (size_t)KT * MX_TILE_A;
      for (int e = tid; e < 32 * KT * 64; e += blockDim.x) {
        const int r = e / (KT * 64), k = e % (KT * 64);
        const int g = r < NC ? 0 : (r < 2 * NC ? 1 : 2), i = r - g * NC; // basis group, column
        const float v = k < n_p ? tb[(g * n_p + k) * ROW + i] : 0.f;
        const __nv_bfloat16 hv = __float2bfloat16_rn(v);
        const __nv_bfloat16 lv = __float2bfloat16_rn(v - __bfloat162float(hv));
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const uint32_t o = (k >> 6) * MX_TILE_A + sw128_offset(32 * q + r, k & 63);
          *reinterpret_cast<__nv_bfloat16 *>(Ah + o) = hv;
          if (SPLIT) *reinterpret_cast<__nv_bfloat16 *>(Al + o) = lv;
        }
      }
      off += (size_t)KT * (SPLIT ? 2 : 1) * MX_TILE_A;
    }
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(taddr_s)), "r"(tcols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int w = 0; w < nw; ++w) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(mbar + w)));
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

  MxWarp W;
  W.sA = sA;
  W.myB = sB + (size_t)warp * ktm * TB;
  W.mbar = smem_u32(mbar + warp);
  W.d_col = tmem + (uint32_t)(N * warp);
  W.d_read = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(N * warp);
  W.phase = 0;
  for (;;) {
    int item = 0;
    if (lane == 0) item = atomicAdd(A.queue, 1);
    item = __shfl_sync(FULL, item, 0);
    if (item >= A.n_traj) break;
    const int b = A.order[item];
    const int nt = (A.problems[A.traj_problem[b]].n_p + 31) >> 5;
    if (!mixed_nt<DIM, MAXNT, SPLIT>(A, b, stab, lane, deadline, W, nt)) break;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(tcols));
}

template <int DIM, int MAXNT, bool SPLIT, bool CAP = false>
static cudaError_t launch_mx(const SolveArgs &a, const LaunchShape &shape, int n_sm,
                             cudaStream_t s, LaunchShape *used) {
  auto kern = k_am_mixed<DIM, MAXNT, SPLIT, CAP>;
  constexpr int MAXW = CAP ? MX_CAP_WARPS : MX_MAX_WARPS;
  // warps per CTA: as asked (default: the batch spread over all SMs), capped by
  // what the shared memory holds
  int warps = shape.warps_per_block > 0 ? shape.warps_per_block
                                        : (int)((a.n_traj + n_sm - 1) / (n_sm > 0 ? n_sm : 1));
  if (warps < 1) warps = 1;
  if (warps > MAXW) warps = MAXW;
  while (warps > 1 && mixed_smem(a, DIM, SPLIT, warps) > 227 * 1024) --warps;
  const size_t smem = mixed_smem(a, DIM, SPLIT, warps);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // the whole unified L1 / shared array as shared memory, so that several CTAs (each
  // with its own copy of the basis operands) fit on an SM
  e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                           (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, warps * 32, smem);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  // A count of blocks per SM asked for explicitly is honoured up to what the SM's
  // resources hold -- registers, shared memory (1 KB reserved per block), tensor memory
  // and warp slots -- even where the occupancy query answers fewer for this kernel.
  if (shape.blocks_per_sm > 0) {
    cudaFuncAttributes fa{};
    e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return e;
    const int regs_cta = ((fa.numRegs * 32 + 255) / 256) * 256 * warps;
    int fit = 65536 / (regs_cta > 0 ? regs_cta : 1);
    fit = std::min(fit, (int)((228 * 1024) / (smem + 1024)));
    fit = std::min(fit, (int)(512u / mixed_tmem_cols(warps, mixed_n(DIM, SPLIT))));
    fit = std::min(fit, 64 / warps);
    occ = std::max(1, std::min(shape.blocks_per_sm, fit));
  }
  // TMEM: every resident CTA holds mixed_tmem_cols of the SM's 512 columns
  while (occ > 1 && (uint32_t)occ * mixed_tmem_cols(warps, mixed_n(DIM, SPLIT)) > 512u) --occ;
  long long grid = (long long)n_sm * occ, want = ((long long)a.n_traj + warps - 1) / warps;
  if (want < grid) grid = want;
  if (grid < 1) grid = 1;
  if (used) {
    used->warps_per_block = warps; used->blocks_per_sm = occ; used->grid = (int)grid; used->team = 1;
    used->occupancy = CAP ? 1 : 0;
    cudaFuncAttributes fa{};
    used->regs = cudaFuncGetAttributes(&fa, kern) == cudaSuccess ? fa.numRegs : 0;
    used->smem = (int)smem;
  }
  kern<<<(unsigned)grid, warps * 32, smem, s>>>(a);
  return cudaGetLastError();
}

template <bool SPLIT>
static cudaError_t launch_mixed_t(int dim, int max_np, const SolveArgs &a, const LaunchShape &shape,
                                  int n_sm, cudaStream_t s, LaunchShape *used) {
  const int nt = (max_np + 31) / 32;
  if (shape.occupancy) { // the register-capped build: horizons up to 160 grid points
    if (nt > 5) return cudaErrorInvalidValue;
    if (dim == 2) return nt <= 4 ? launch_mx<2, 4, SPLIT, true>(a, shape, n_sm, s, used)
                                 : launch_mx<2, 5, SPLIT, true>(a, shape, n_sm, s, used);
    return nt <= 4 ? launch_mx<3, 4, SPLIT, true>(a, shape, n_sm, s, used)
                   : launch_mx<3, 5, SPLIT, true>(a, shape, n_sm, s, used);
  }
  if (dim == 2) {
    if (nt <= 2) return launch_mx<2, 2, SPLIT>(a, shape, n_sm, s, used);
    if (nt <= 4) return launch_mx<2, 4, SPLIT>(a, shape, n_sm, s, used);
    if (nt <= 5) return launch_mx<2, 5, SPLIT>(a, shape, n_sm, s, used);
    return launch_mx<2, 8, SPLIT>(a, shape, n_sm, s, used);
  }
  if (nt <= 2) return launch_mx<3, 2, SPLIT>(a, shape, n_sm, s, used);
  if (nt <= 4) return launch_mx<3, 4, SPLIT>(a, shape, n_sm, s, used);
  if (nt <= 5) return launch_mx<3, 5, SPLIT>(a, shape, n_sm, s, used);
  return launch_mx<3, 8, SPLIT>(a, shape, n_sm, s, used);
}

size_t mixed_smem_bytes(const SolveArgs &a, int dim, bool split, int warps) {
  return mixed_smem(a, dim, split, warps);
}

cudaError_t launch_am_mixed(int dim, int max_np, bool split, const SolveArgs &a,
                            const LaunchShape &shape, int n_sm, cudaStream_t s, LaunchShape *used) {
  const int nt = (max_np + 31) / 32;
  if (shape.team > 1 || nt > 8 || a.hz_n < 1 || a.hz_n > MAX_HZ) return cudaErrorInvalidValue;
  return split ? launch_mixed_t<true>(dim, max_np, a, shape, n_sm, s, used)
               : launch_mixed_t<false>(dim, max_np, a, shape, n_sm, s, used);
}

} // namespace tb

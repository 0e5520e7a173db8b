// tcgen05 complex GEMM in 3xTF32 split precision for the transformed states of the
// precision form (step (iii), Eqs. SCHnewstate / SCHtransmatrix):
//     W^T[m][n] = sum_q S^T[m][q] P^T[q][n],   complex, FP32 in / FP32 out.
//
// The complex product is written as two real K-major GEMMs over K' = 2 n_pw with
// interleaved real/imaginary parts:
//     A1[m][2q] = Re S,  A1[m][2q+1] = -Im S        (row m of S^T)
//     A2[m][2q] = Im S,  A2[m][2q+1] =  Re S
//     B [n][2q] = Re P,  B [n][2q+1] =  Im P        (P = conj(P^T)^T, P Hermitian)
//     Re W = A1 B^T,  Im W = A2 B^T.
// Each operand x is split as x_hi = tf32(x), x_lo = tf32(x - x_hi) (round to nearest),
// and every product is x_hi y_hi + x_hi y_lo + x_lo y_hi, accumulated in FP32 in tensor
// memory.  Operands arrive by TMA into a shared-memory ring; one thread issues the TMA
// copies and the MMAs; four warps read the accumulators.  Two layouts, both chosen
// between by the autotuner: k_tc_cgemm_drain (separate Re / Im operands, N = 64) and
// k_tc_cgemm_stacked (Re / Im rows stacked in one MMA tile; the default, and the only
// one for real orbitals).  Every wait is bounded: on expiry the kernel raises an error
// flag, waits (bounded) for the TMA copies it issued, writes no output, frees its
// tensor memory and returns, instead of hanging.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "tcgen05.cuh"

namespace ltmp2 {
namespace tc {

constexpr int BM = 128;             // rows of A per tile (complex rows of W^T)
constexpr int BK = 32;              // fp32 elements per k block = one 128-byte swizzle row
constexpr int A_TILE_BYTES = BM * 128;
constexpr int STAGES = 2;
// Tile of BN columns with NREG accumulator pairs (Re, Im) in tensor memory.  The tensor
// core's internal accumulation is not round-to-nearest: a single chain over K' ~ 6000
// drifted by ~1e-4 (relative) on the transformed states, so the kernels below drain every
// k block's partial into FP32 register sums.
template <int BN, int NREG> struct TcCfg {
  static constexpr int B_TILE_BYTES = BN * 128;
  static constexpr int STAGE_BYTES = 4 * A_TILE_BYTES + 2 * B_TILE_BYTES;
  static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024;   // + alignment slack
  static constexpr int TMEM_COLS = 2 * BN * NREG;
  static_assert(TMEM_COLS == 64 || TMEM_COLS == 128 || TMEM_COLS == 256 || TMEM_COLS == 512, "TMEM columns");
  // instruction descriptor: D fp32, A and B tf32, both K-major, M = 128, N = BN
  static constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) |
                                    ((uint32_t)(BM >> 4) << 24);
};
// Failure-path self-test: one thread waits, with the same bounded wait the GEMM kernels
// use, on an mbarrier that nothing ever arrives on; when the budget runs out it raises the
// same device error word, and the kernel returns.  Nothing hangs or faults.
__global__ void k_wait_selftest(int *err, unsigned long long limit_ns) {
  __shared__ uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  if (!mbar_wait(&bar, 0, limit_ns)) atomicExch(err, 1);
}
// ---------------------------------------------------------------- operand packing
// S^T complex [rows][npw] -> A1/A2 hi/lo, fp32 [rows][kpad]; zero past 2 npw
__global__ void k_pack_a(const float2 *__restrict__ st, int rows, int npw, int kpad, float *__restrict__ a1h,
                         float *__restrict__ a1l, float *__restrict__ a2h, float *__restrict__ a2l) {
  const int m = blockIdx.y;
  const int half = kpad / 2;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < half; q += gridDim.x * blockDim.x) {
    float re = 0.f, im = 0.f;
    if (q < npw && m < rows) {
      const float2 v = st[(size_t)m * npw + q];
      re = v.x;
      im = v.y;
    }
    const float h_re = tf32_rn(re), l_re = tf32_rn(re - h_re);
    const float h_im = tf32_rn(im), l_im = tf32_rn(im - h_im);
    const size_t o = (size_t)m * kpad + 2 * q;
    a1h[o] = h_re; a1h[o + 1] = -h_im;
    a1l[o] = l_re; a1l[o + 1] = -l_im;
    a2h[o] = h_im; a2h[o + 1] = h_re;
    a2l[o] = l_im; a2l[o + 1] = l_re;
  }
}
// P^T complex [npw][npw] (Hermitian P) -> B[n][2q] = Re P[n][q] = Re P^T[n][q],
// B[n][2q+1] = Im P[n][q] = -Im P^T[n][q]; hi/lo split, fp32 [npw][kpad]
__global__ void k_pack_b(const float2 *__restrict__ pt, int npw, int kpad, float *__restrict__ bh,
                         float *__restrict__ bl) {
  const int n = blockIdx.y;
  const int half = kpad / 2;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < half; q += gridDim.x * blockDim.x) {
    float re = 0.f, im = 0.f;
    if (q < npw) {
      const float2 v = pt[(size_t)n * npw + q];
      re = v.x;
      im = -v.y;
    }
    const float h_re = tf32_rn(re), l_re = tf32_rn(re - h_re);
    const float h_im = tf32_rn(im), l_im = tf32_rn(im - h_im);
    const size_t o = (size_t)n * kpad + 2 * q;
    bh[o] = h_re; bh[o + 1] = h_im;
    bl[o] = l_re; bl[o + 1] = l_im;
  }
}

struct TcMaps {
  CUtensorMap a1h, a1l, a2h, a2l, bh, bl;
};

// ---------------------------------------------------------------- drained variant
// Warp 4 (one elected thread) issues TMA copies and MMAs; warps 0-3 own tensor-memory
// lanes 0-127.  Each k block is accumulated into one of two tensor-memory accumulator
// pairs (Re, Im; BN columns each) starting from zero, and the four epilogue warps add
// that partial to FP32 register sums (round to nearest) and release the pair for the
// block after next.  The tensor core's own accumulation thus runs over 12 MMAs only.

template <int BN>
__global__ void __launch_bounds__(160, 1)
    k_tc_cgemm_drain(const __grid_constant__ CUtensorMap ta1h, const __grid_constant__ CUtensorMap ta1l,
                     const __grid_constant__ CUtensorMap ta2h, const __grid_constant__ CUtensorMap ta2l,
                     const __grid_constant__ CUtensorMap tbh, const __grid_constant__ CUtensorMap tbl, int M, int N,
                     int kblocks, float2 *__restrict__ C, int ldc, int *__restrict__ err) {
  using Cfg = TcCfg<BN, 2>;
  extern __shared__ unsigned char smem_raw[];
  __shared__ uint64_t full_bar[STAGES], empty_bar[STAGES], accf_bar[2], acce_bar[2], done_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_fail;   // any bounded wait of the CTA ran out: no output is written
  unsigned char *smem = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;

  if (warp == 0) tmem_alloc(&tmem_slot, Cfg::TMEM_COLS);
  if (threadIdx.x == 0) {
    s_fail = 0;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int r = 0; r < 2; ++r) {
      mbar_init(&accf_bar[r], 1);
      mbar_init(&acce_bar[r], 128);
    }
    mbar_init(&done_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_slot;
  bool ok = true;
  float sr[BN], si[BN];   // epilogue warps: the tile row's Re / Im sums
#pragma unroll
  for (int j = 0; j < BN; ++j) { sr[j] = 0.f; si[j] = 0.f; }

  if (warp == 4) {
    if (lane == 0) {
      auto issue = [&](int kb, int s) {
        unsigned char *st = smem + s * Cfg::STAGE_BYTES;
        mbar_expect_tx(&full_bar[s], Cfg::STAGE_BYTES);
        const int x = kb * BK;
        tma_load_2d(st + 0 * A_TILE_BYTES, &ta1h, &full_bar[s], x, m0);
        tma_load_2d(st + 1 * A_TILE_BYTES, &ta1l, &full_bar[s], x, m0);
        tma_load_2d(st + 2 * A_TILE_BYTES, &ta2h, &full_bar[s], x, m0);
        tma_load_2d(st + 3 * A_TILE_BYTES, &ta2l, &full_bar[s], x, m0);
        tma_load_2d(st + 4 * A_TILE_BYTES, &tbh, &full_bar[s], x, n0);
        tma_load_2d(st + 4 * A_TILE_BYTES + Cfg::B_TILE_BYTES, &tbl, &full_bar[s], x, n0);
      };
      int issued = 0, consumed = 0;
      for (int s = 0; s < STAGES && s < kblocks; ++s) issue(s, s), issued = s + 1;
      for (int kb = 0; kb < kblocks; ++kb) {
        const int s = kb % STAGES, r = kb & 1;
        if (!mbar_wait(&full_bar[s], (uint32_t)((kb / STAGES) & 1))) { ok = false; break; }
        consumed = kb + 1;
        if (kb >= 2 && !mbar_wait(&acce_bar[r], (uint32_t)(((kb - 2) >> 1) & 1))) { ok = false; break; }
        fence_after();
        const uint32_t base = smem_u32(smem + s * Cfg::STAGE_BYTES);
        const uint32_t dre = tmem + (uint32_t)r * (2 * BN), dim = dre + BN;
#pragma unroll
        for (int k = 0; k < BK / 8; ++k) {
          const uint32_t ko = k * 32;
          const uint64_t a1h = sdesc_sw128(base + 0 * A_TILE_BYTES + ko);
          const uint64_t a1l = sdesc_sw128(base + 1 * A_TILE_BYTES + ko);
          const uint64_t a2h = sdesc_sw128(base + 2 * A_TILE_BYTES + ko);
          const uint64_t a2l = sdesc_sw128(base + 3 * A_TILE_BYTES + ko);
          const uint64_t bh = sdesc_sw128(base + 4 * A_TILE_BYTES + ko);
          const uint64_t bl = sdesc_sw128(base + 4 * A_TILE_BYTES + Cfg::B_TILE_BYTES + ko);
          const uint32_t acc = k > 0 ? 1u : 0u;
          mma_tf32(dre, a1h, bh, Cfg::IDESC, acc);
          mma_tf32(dre, a1h, bl, Cfg::IDESC, 1u);
          mma_tf32(dre, a1l, bh, Cfg::IDESC, 1u);
          mma_tf32(dim, a2h, bh, Cfg::IDESC, acc);
          mma_tf32(dim, a2h, bl, Cfg::IDESC, 1u);
          mma_tf32(dim, a2l, bh, Cfg::IDESC, 1u);
        }
        mma_commit(&empty_bar[s]);
        mma_commit(&accf_bar[r]);
        if (kb >= 1 && kb + 1 < kblocks) {
          const int sp = (kb - 1) % STAGES;
          if (!mbar_wait(&empty_bar[sp], (uint32_t)(((kb - 1) / STAGES) & 1))) { ok = false; break; }
          issue(kb + 1, sp);
          issued = kb + 2;
        }
      }
      mma_commit(&done_bar);
      if (!ok) {
        s_fail = 1;
        atomicExch(err, 1);
        drain_issued<STAGES>(full_bar, consumed, issued);
      }
    }
  } else {
    // epilogue warps: drain every k block's partial into FP32 register sums
    const uint32_t t_lane = tmem + ((uint32_t)(warp * 32) << 16);
    for (int kb = 0; kb < kblocks; ++kb) {
      const int r = kb & 1;
      if (!mbar_wait(&accf_bar[r], (uint32_t)((kb >> 1) & 1))) { ok = false; break; }
      fence_after();
#pragma unroll
      for (int c = 0; c < BN / 32; ++c) {
        float v[32];
        tmem_ld32(t_lane + r * 2 * BN + c * 32, v);
#pragma unroll
        for (int j = 0; j < 32; ++j) sr[c * 32 + j] += v[j];
        tmem_ld32(t_lane + r * 2 * BN + BN + c * 32, v);
#pragma unroll
        for (int j = 0; j < 32; ++j) si[c * 32 + j] += v[j];
      }
      fence_before();
      mbar_arrive(&acce_bar[r]);
    }
    if (!ok) {
      s_fail = 1;
      if (lane == 0) atomicExch(err, 1);
    }
  }
  const bool done_ok = mbar_wait(&done_bar, 0);
  if (!done_ok) {
    s_fail = 1;
    if (lane == 0) atomicExch(err, 1);
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp < 4 && !s_fail) {
    const int gm = m0 + warp * 32 + lane;
    if (gm < M) {
      float2 *dst = C + (size_t)gm * ldc + n0;
#pragma unroll
      for (int j = 0; j < BN; ++j)
        if (n0 + j < N) dst[j] = make_float2(sr[j], si[j]);
    }
  }
  if (warp == 0) tmem_dealloc(tmem, Cfg::TMEM_COLS);
}

// ---------------------------------------------------------------- stacked, deep-ring variant
// One MMA row tile of 128 = 64 complex rows of A1 (rows 0-63) stacked over the same 64
// rows of A2 (rows 64-127), so a single accumulator holds Re (lanes 0-63) and Im
// (lanes 64-127) of a 64 x BN2 block of W^T.  K blocks of 16 fp32 (64-byte swizzle)
// make a stage 32 KB: A hi, A lo, B hi, B lo.  Three stages are in flight per CTA, and
// two CTAs share each SM (97 KB of shared memory and 256 tensor-memory columns each), so
// one CTA's MMAs fill the other's waits on TMA: 1.6x faster than one CTA with six stages
// on the 24^3 workload.  Accumulators
// alternate between two tensor-memory regions and are drained into FP32 register sums
// after every stage (6 MMAs per region).  Draining every second stage (12 MMAs, as in the
// drained variant above) left 30 % more relative error in the direct energy of the 24^3
// workload (the tensor core's accumulation is not round-to-nearest) for 6 % less time.
constexpr int S_BK = 16;                   // fp32 per k block (64 bytes)
constexpr int S_BN = 128;
constexpr int S_TILE = 128 * 64;           // 128 rows x 64 bytes
constexpr int S_STAGE = 4 * S_TILE;
constexpr int S_STAGES = 3;
constexpr int S_DRAIN = 1;                 // stages per accumulator region
constexpr int S_SMEM = S_STAGES * S_STAGE + 1024;
constexpr int S_TMEM_COLS = 2 * S_BN;
constexpr uint32_t S_IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(S_BN >> 3) << 17) |
                             ((uint32_t)(128 >> 4) << 24);


// S^T complex [rows][npw] -> stacked A hi/lo fp32 [2 * rows_pad64][kpad]:
// row 128 b + r = A1 row 64 b + r, row 128 b + 64 + r = A2 row 64 b + r
__global__ void k_pack_a_stacked(const float2 *__restrict__ st, int rows, int npw, int kpad,
                                 float *__restrict__ ah, float *__restrict__ al) {
  const int m = blockIdx.y;
  const int half = kpad / 2;
  const size_t r1 = (size_t)128 * (m / 64) + (m % 64), r2 = r1 + 64;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < half; q += gridDim.x * blockDim.x) {
    float re = 0.f, im = 0.f;
    if (q < npw && m < rows) {
      const float2 v = st[(size_t)m * npw + q];
      re = v.x;
      im = v.y;
    }
    const float h_re = tf32_rn(re), l_re = tf32_rn(re - h_re);
    const float h_im = tf32_rn(im), l_im = tf32_rn(im - h_im);
    const size_t o1 = r1 * kpad + 2 * q, o2 = r2 * kpad + 2 * q;
    ah[o1] = h_re; ah[o1 + 1] = -h_im;
    al[o1] = l_re; al[o1 + 1] = -l_im;
    ah[o2] = h_im; ah[o2 + 1] = h_re;
    al[o2] = l_im; al[o2 + 1] = l_re;
  }
}

// Real-basis Green's function (real orbitals): W^T = S_r^T P_r with S_r^T complex and P_r
// real symmetric, so Re W^T = (Re S_r^T) P_r and Im W^T = (Im S_r^T) P_r over K = n_pw.
// Stacked rows: row 128 b + r = Re of row 64 b + r, row 128 b + 64 + r = its Im;
// B[n][q] = P_r[n][q].  The same stacked kernel then yields Re (lanes 0-63) and Im
// (lanes 64-127) with half the k blocks of the complex form.
__global__ void k_pack_a_stacked_real(const float2 *__restrict__ st, int rows, int npw, int kpad,
                                      float *__restrict__ ah, float *__restrict__ al) {
  const int m = blockIdx.y;
  const size_t r1 = (size_t)128 * (m / 64) + (m % 64), r2 = r1 + 64;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < kpad; q += gridDim.x * blockDim.x) {
    float re = 0.f, im = 0.f;
    if (q < npw && m < rows) {
      const float2 v = st[(size_t)m * npw + q];
      re = v.x;
      im = v.y;
    }
    const float h_re = tf32_rn(re), h_im = tf32_rn(im);
    ah[r1 * kpad + q] = h_re;
    al[r1 * kpad + q] = tf32_rn(re - h_re);
    ah[r2 * kpad + q] = h_im;
    al[r2 * kpad + q] = tf32_rn(im - h_im);
  }
}
__global__ void k_pack_b_real(const float *__restrict__ pr, int npw, int kpad, float *__restrict__ bh,
                              float *__restrict__ bl) {
  const int n = blockIdx.y;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < kpad; q += gridDim.x * blockDim.x) {
    const float v = q < npw ? pr[(size_t)n * npw + q] : 0.f;
    const float h = tf32_rn(v);
    bh[(size_t)n * kpad + q] = h;
    bl[(size_t)n * kpad + q] = tf32_rn(v - h);
  }
}

// ---------------------------------------------------------------- Green's function operands
// Real basis: P_r = R_v^T D R_v (Eq. SCHtransmatrix summed over the virtuals), K = n_v.
// Two real rows of A = R_v^T D form one complex row of the stacked kernel (row 2m as Re,
// row 2m + 1 as Im), so its float2 output is P_r with rows 2m and 2m + 1 interleaved per
// column; B = R_v^T (row n = column n of R_v), split once per context.
__global__ void k_transpose_f(int rows, int cols, const float *__restrict__ in, float *__restrict__ out) {
  __shared__ float tile[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int r = r0 + k, c = c0 + threadIdx.x;
    if (r < rows && c < cols) tile[k][threadIdx.x] = in[(size_t)r * cols + c];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int c = c0 + k, r = r0 + threadIdx.x;
    if (r < rows && c < cols) out[(size_t)c * rows + r] = tile[threadIdx.x][k];
  }
}
// A hi/lo, stacked rows: row 128 b + r <- A row 2 (64 b + r), row 128 b + 64 + r <- A row 2 (64 b + r) + 1
__global__ void k_pack_green_a(const float *__restrict__ rvt, const float *__restrict__ dv, int npw, int nv, int kpad,
                               float *__restrict__ ah, float *__restrict__ al) {
  const int m = blockIdx.y;
  const size_t r1 = (size_t)128 * (m / 64) + (m % 64), r2 = r1 + 64;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < kpad; a += gridDim.x * blockDim.x) {
    const float d = a < nv ? dv[a] : 0.f;
    const float re = (2 * m < npw && a < nv) ? rvt[(size_t)(2 * m) * nv + a] * d : 0.f;
    const float im = (2 * m + 1 < npw && a < nv) ? rvt[(size_t)(2 * m + 1) * nv + a] * d : 0.f;
    const float hr = tf32_rn(re), hi = tf32_rn(im);
    ah[r1 * kpad + a] = hr;
    al[r1 * kpad + a] = tf32_rn(re - hr);
    ah[r2 * kpad + a] = hi;
    al[r2 * kpad + a] = tf32_rn(im - hi);
  }
}
// B hi/lo [rows][kpad] from a row-major real matrix with row length ld (zero past ld)
__global__ void k_pack_rows(const float *__restrict__ x, int ld, int kpad, float *__restrict__ bh, float *__restrict__ bl) {
  const int n = blockIdx.y;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < kpad; q += gridDim.x * blockDim.x) {
    const float v = q < ld ? x[(size_t)n * ld + q] : 0.f;
    const float h = tf32_rn(v);
    bh[(size_t)n * kpad + q] = h;
    bl[(size_t)n * kpad + q] = tf32_rn(v - h);
  }
}
// the transformed-state GEMM's B from the pair-interleaved Green's function
__global__ void k_pack_b_pairs(const float2 *__restrict__ c, int npw, int kpad, float *__restrict__ bh,
                               float *__restrict__ bl) {
  const int n = blockIdx.y;
  const float2 *row = c + (size_t)(n / 2) * npw;
  const bool odd = n & 1;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < kpad; q += gridDim.x * blockDim.x) {
    const float v = q < npw ? (odd ? row[q].y : row[q].x) : 0.f;
    const float h = tf32_rn(v);
    bh[(size_t)n * kpad + q] = h;
    bl[(size_t)n * kpad + q] = tf32_rn(v - h);
  }
}

// blockIdx.z runs over independent products of one launch: product z reads stacked A rows
// from z * a_zrows and B rows from z * b_zrows (tensor-map coordinates) and writes C + z * c_zstride.
// ---------------------------------------------------------------- direct-term operands
// Per primary G' z of the slab, Y_ij = sum_G v(G) M_ii(G) conj(M_jj(G)) (real orbitals) is
// the stacked product of A (complex rows i: M_ii over K = G) with the real rows B_n = v Re M_n
// (n < n_o) and B_{n_o + n} = v Im M_n.  mdiag is [slot][G][i]: 32 x 32 tiles through shared
// memory turn it K-major.  A rows of product z start at z * 2 r64 (r64: n_o rounded to 64).
__global__ void k_pack_direct(const float2 *__restrict__ mdiag, const float *__restrict__ v, int naux, int no,
                              int kpad, int r64, float *__restrict__ ah, float *__restrict__ al,
                              float *__restrict__ bh, float *__restrict__ bl) {
  __shared__ float2 tile[32][33];
  const int z = blockIdx.z, g0 = blockIdx.x * 32, i0 = blockIdx.y * 32;
  const float2 *mz = mdiag + (size_t)z * naux * no;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int g = g0 + k, i = i0 + threadIdx.x;
    tile[k][threadIdx.x] = (g < naux && i < no) ? mz[(size_t)g * no + i] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int i = i0 + k, g = g0 + threadIdx.x;
    if (i >= r64 || g >= kpad) continue;
    const float2 m = tile[threadIdx.x][k];
    const float vg = g < naux ? v[g] : 0.f;
    const size_t ra = (size_t)z * 2 * r64 + 128 * (i / 64) + (i % 64);
    float h = tf32_rn(m.x);
    ah[ra * kpad + g] = h;
    al[ra * kpad + g] = tf32_rn(m.x - h);
    h = tf32_rn(m.y);
    ah[(ra + 64) * kpad + g] = h;
    al[(ra + 64) * kpad + g] = tf32_rn(m.y - h);
    if (i < no) {
      const size_t rb = (size_t)z * 2 * no + i;
      const float re = vg * m.x, im = vg * m.y;
      h = tf32_rn(re);
      bh[rb * kpad + g] = h;
      bl[rb * kpad + g] = tf32_rn(re - h);
      h = tf32_rn(im);
      bh[(rb + no) * kpad + g] = h;
      bl[(rb + no) * kpad + g] = tf32_rn(im - h);
    }
  }
}
// Y_ij from the four blocks of product z: C [n_o][2 n_o] per z
__global__ void k_direct_combine(const float2 *__restrict__ C, int no, double2 *__restrict__ yd) {
  const int z = blockIdx.y;
  const float2 *c = C + (size_t)z * no * 2 * no;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < no * no; e += gridDim.x * blockDim.x) {
    const int i = e / no, j = e % no;
    const float2 a = c[(size_t)i * 2 * no + j], b = c[(size_t)i * 2 * no + no + j];
    yd[(size_t)z * no * no + e] = make_double2((double)a.x + (double)b.y, (double)a.y - (double)b.x);
  }
}

__global__ void __launch_bounds__(160, 2)
    k_tc_cgemm_stacked(const __grid_constant__ CUtensorMap tah, const __grid_constant__ CUtensorMap tal,
                       const __grid_constant__ CUtensorMap tbh, const __grid_constant__ CUtensorMap tbl, int M,
                       int N, int kblocks, float2 *__restrict__ C, int ldc, int *__restrict__ err, int a_zrows = 0,
                       int b_zrows = 0, long long c_zstride = 0) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ uint64_t full_bar[S_STAGES], empty_bar[S_STAGES], accf_bar[2], acce_bar[2], done_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_fail;   // any bounded wait of the CTA ran out: no output is written
  unsigned char *smem = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int arow0 = blockIdx.z * a_zrows + blockIdx.y * 128;   // stacked operand rows
  const int m0 = blockIdx.y * 64;         // complex rows of W^T
  const int n0 = blockIdx.x * S_BN;
  const int brow0 = blockIdx.z * b_zrows + n0;
  C += blockIdx.z * c_zstride;
  const int ndrain = (kblocks + S_DRAIN - 1) / S_DRAIN;

  if (warp == 0) tmem_alloc(&tmem_slot, S_TMEM_COLS);
  if (threadIdx.x == 0) {
    s_fail = 0;
    for (int s = 0; s < S_STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int r = 0; r < 2; ++r) {
      mbar_init(&accf_bar[r], 1);
      mbar_init(&acce_bar[r], 128);
    }
    mbar_init(&done_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_slot;
  bool ok = true;
  float sum[S_BN];   // epilogue warps: the lane's row of the tile
#pragma unroll
  for (int j = 0; j < S_BN; ++j) sum[j] = 0.f;

  if (warp == 4) {
    if (lane == 0) {
      auto issue = [&](int kb, int s) {
        unsigned char *st = smem + s * S_STAGE;
        mbar_expect_tx(&full_bar[s], S_STAGE);
        const int x = kb * S_BK;
        tma_load_2d(st + 0 * S_TILE, &tah, &full_bar[s], x, arow0);
        tma_load_2d(st + 1 * S_TILE, &tal, &full_bar[s], x, arow0);
        tma_load_2d(st + 2 * S_TILE, &tbh, &full_bar[s], x, brow0);
        tma_load_2d(st + 3 * S_TILE, &tbl, &full_bar[s], x, brow0);
      };
      int issued = 0, consumed = 0;
      for (int s = 0; s < S_STAGES && s < kblocks; ++s) issue(s, s), issued = s + 1;
      for (int kb = 0; kb < kblocks; ++kb) {
        const int s = kb % S_STAGES;
        const int db = kb / S_DRAIN, r = db & 1;
        if (!mbar_wait(&full_bar[s], (uint32_t)((kb / S_STAGES) & 1))) { ok = false; break; }
        consumed = kb + 1;
        if (kb % S_DRAIN == 0 && db >= 2 && !mbar_wait(&acce_bar[r], (uint32_t)(((db - 2) >> 1) & 1))) {
          ok = false;
          break;
        }
        fence_after();
        const uint32_t base = smem_u32(smem + s * S_STAGE);
        const uint32_t d = tmem + (uint32_t)r * S_BN;
#pragma unroll
        for (int k = 0; k < S_BK / 8; ++k) {
          const uint32_t ko = k * 32;
          const uint64_t ah = sdesc_sw64(base + 0 * S_TILE + ko), al = sdesc_sw64(base + 1 * S_TILE + ko);
          const uint64_t bh = sdesc_sw64(base + 2 * S_TILE + ko), bl = sdesc_sw64(base + 3 * S_TILE + ko);
          const uint32_t acc = (kb % S_DRAIN == 0 && k == 0) ? 0u : 1u;
          mma_tf32(d, ah, bh, S_IDESC, acc);
          mma_tf32(d, ah, bl, S_IDESC, 1u);
          mma_tf32(d, al, bh, S_IDESC, 1u);
        }
        mma_commit(&empty_bar[s]);
        if (kb % S_DRAIN == S_DRAIN - 1 || kb == kblocks - 1) mma_commit(&accf_bar[r]);
        // refill the stage of k block kb - 1 once its MMAs are done (those of kb are queued)
        if (kb >= 1 && kb - 1 + S_STAGES < kblocks) {
          const int sp = (kb - 1) % S_STAGES;
          if (!mbar_wait(&empty_bar[sp], (uint32_t)(((kb - 1) / S_STAGES) & 1))) { ok = false; break; }
          issue(kb - 1 + S_STAGES, sp);
          issued = kb - 1 + S_STAGES + 1;
        }
      }
      mma_commit(&done_bar);
      if (!ok) {
        s_fail = 1;
        atomicExch(err, 1);
        drain_issued<S_STAGES>(full_bar, consumed, issued);
      }
    }
  } else {
    const uint32_t t_lane = tmem + ((uint32_t)(warp * 32) << 16);
    for (int db = 0; db < ndrain; ++db) {
      const int r = db & 1;
      if (!mbar_wait(&accf_bar[r], (uint32_t)((db >> 1) & 1))) { ok = false; break; }
      fence_after();
#pragma unroll
      for (int c = 0; c < S_BN / 16; ++c) {
        uint32_t rr[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
            "%15}, [%16];"
            : "=r"(rr[0]), "=r"(rr[1]), "=r"(rr[2]), "=r"(rr[3]), "=r"(rr[4]), "=r"(rr[5]), "=r"(rr[6]), "=r"(rr[7]),
              "=r"(rr[8]), "=r"(rr[9]), "=r"(rr[10]), "=r"(rr[11]), "=r"(rr[12]), "=r"(rr[13]), "=r"(rr[14]), "=r"(rr[15])
            : "r"(t_lane + r * S_BN + c * 16));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int j = 0; j < 16; ++j) sum[c * 16 + j] += __uint_as_float(rr[j]);
      }
      fence_before();
      mbar_arrive(&acce_bar[r]);
    }
    if (!ok) {
      s_fail = 1;
      if (lane == 0) atomicExch(err, 1);
    }
    if (!mbar_wait(&done_bar, 0)) {
      s_fail = 1;
      if (lane == 0) atomicExch(err, 1);
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  // every MMA has completed and every TMA copy has landed unless s_fail is set; only then
  // is the ring reused as staging: Re (warps 0, 1) paired with Im (warps 2, 3)
  if (warp < 4 && !s_fail) {
    float *stage = reinterpret_cast<float *>(smem);   // [128][S_BN + 1]
    const int row = warp * 32 + lane;
#pragma unroll
    for (int j = 0; j < S_BN; ++j) stage[row * (S_BN + 1) + j] = sum[j];
    asm volatile("bar.sync 1, 128;" ::: "memory");
    for (int e = threadIdx.x; e < 64 * S_BN; e += 128) {
      const int rr = e / S_BN, cc = e % S_BN;
      const int gm = m0 + rr, gn = n0 + cc;
      if (gm < M && gn < N)
        C[(size_t)gm * ldc + gn] = make_float2(stage[rr * (S_BN + 1) + cc], stage[(rr + 64) * (S_BN + 1) + cc]);
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0) tmem_dealloc(tmem, S_TMEM_COLS);
}

}  // namespace tc
}  // namespace ltmp2

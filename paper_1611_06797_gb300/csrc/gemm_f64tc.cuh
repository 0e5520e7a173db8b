// FP64-accurate products on the tcgen05 tensor cores (the FP64 path's transformed-state GEMM,
// W^T = (U S)^T P_r of step (iii), Sec. III A), by exact integer slices (Ozaki's scheme):
//
//   each row of A and of B (C = A B^T, both K-major) is scaled by a power of two 2^e with
//   |x| < 2^e over the row and cut into S = 8 slices of 7 bits,
//       a = 2^e_a sum_s d_s 2^{-7(s+1)},  d_s integers, |d_0| <= 128, |d_s| <= 64 (s >= 1),
//   every slice exactly representable in TF32.  Then
//       (A B^T)_ij = 2^{e_i + f_j} sum_{d=0}^{S-1} 2^{-7(d+2)} sum_{s+t=d} sum_k a_{s,ik} b_{t,jk}
//   with the pairs s + t >= S left out (per term at most 7 x 2^12 x 2^-70 x 2^{e_a + e_b}
//   <= 7 x 2^-56 max|a| max|b|, at the rounding of an FP64 product).  Each inner sum is a
//   sum of integer products; over 400 k (25 k blocks) it stays below 2^24 in magnitude (at
//   most 2 x 128 x 64 + 6 x 64 x 64 = 2.5 x 2^14 per k for one order d), so every partial
//   sum is an integer that FP32 holds exactly and the tensor core's accumulation is exact,
//   whatever its rounding.  The accumulators of the 8 orders d live in tensor memory
//   (8 x 64 columns = all 512) and are drained every 25 k blocks into FP64 register sums,
//   scaled by 2^{-7(d+2)}.  The result carries the FP64 rounding of those
//   sums and of the slicing, about the error of an FP64 dot product.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "tcgen05.cuh"

namespace ltmp2 {
namespace oz {

constexpr int S = 8;                         // slices per operand
constexpr int BITS = 7;                      // bits per slice
constexpr int BM = 128;                      // rows of A per tile (tensor-memory lanes)
constexpr int BN = 64;                       // rows of B per tile (accumulator columns)
constexpr int BK = 16;                       // fp32 per k block (one 64-byte swizzle row)
constexpr int A_TILE = BM * 64;              // bytes of one A slice tile
constexpr int B_TILE = BN * 64;
constexpr int STAGE = S * (A_TILE + B_TILE); // 96 KB
constexpr int STAGES = 2;
constexpr int SMEM = STAGES * STAGE + 1024;  // + alignment slack
constexpr int TMEM_COLS = S * BN;            // one accumulator per slice order d = s + t
constexpr int DRAIN_KB = 25;                 // k blocks between drains (400 k: sums below 2^24)
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);

// the smallest e with |x| < 2^e for every |x| <= m (0 for m = 0)
__device__ __forceinline__ int row_exponent(double m) { return m > 0.0 ? ilogb(m) + 1 : 0; }

// x in (-1, 1) -> S slices (integers as floats) x = sum_s d_s 2^{-7(s+1)} + r, |r| <= 2^{-57}
__device__ __forceinline__ void slice(double x, float (&d)[S]) {
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const double t = x * 128.0;   // exact (power of two)
    const double r = rint(t);     // |r| <= 128 for s = 0, <= 64 after
    d[s] = (float)r;
    x = t - r;                    // exact: |x| <= 1/2
  }
}

// block-wide max of v over blockDim.x threads (blockDim.x a multiple of 32, <= 1024)
__device__ __forceinline__ double block_max(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x / 32, nw = blockDim.x / 32;
  __syncthreads();
  if (threadIdx.x % 32 == 0) red[w] = v;
  __syncthreads();
  double m = 0.0;
  for (int i = 0; i < nw; ++i) m = fmax(m, red[i]);
  return m;
}

// Slices of the rows of a real matrix X [nrows][ld], columns q < k, each times cscale[q]
// when cscale is not null: plane s row r at planes[(s * prows + r) * pitch + q] for
// q < kfill (zero past k); scale[r] = 2^e_r.  One block per row r < prows.
__global__ void k_oz_split_rows(const double *__restrict__ x, int nrows, int k, int ld, const double *__restrict__ cscale,
                                int kfill, int pitch, int prows, float *__restrict__ planes, double *__restrict__ scale) {
  __shared__ double red[32];
  const int r = blockIdx.x;
  double m = 0.0;
  if (r < nrows)
    for (int q = threadIdx.x; q < k; q += blockDim.x)
      m = fmax(m, fabs(x[(size_t)r * ld + q] * (cscale ? cscale[q] : 1.0)));
  const int e = row_exponent(block_max(m, red));
  if (threadIdx.x == 0) scale[r] = ldexp(1.0, e);
  for (int q = threadIdx.x; q < kfill; q += blockDim.x) {
    const double v = (r < nrows && q < k) ? ldexp(x[(size_t)r * ld + q] * (cscale ? cscale[q] : 1.0), -e) : 0.0;
    float d[S];
    slice(v, d);
#pragma unroll
    for (int s = 0; s < S; ++s) planes[((size_t)s * prows + r) * pitch + q] = d[s];
  }
}

// Slices of the stacked rows of a complex matrix X [rows][ld] (columns q < k): complex row
// m gives stacked row 128 (m / 64) + m % 64 (its real part) and that + 64 (its imaginary
// part), each with its own scale; plane s row r at planes[(s * prows + r) * pitch + q] for
// q < kfill.  One block per complex row m < prows / 2 (rows past `rows` are zero).
__global__ void k_oz_split_stacked(const double2 *__restrict__ x, int rows, int k, int ld, int kfill, int pitch,
                                   int prows, float *__restrict__ planes, double *__restrict__ scale) {
  __shared__ double red[32];
  const int m = blockIdx.x;
  const size_t r1 = (size_t)128 * (m / 64) + (m % 64), r2 = r1 + 64;
  double mr = 0.0, mi = 0.0;
  if (m < rows)
    for (int q = threadIdx.x; q < k; q += blockDim.x) {
      const double2 v = x[(size_t)m * ld + q];
      mr = fmax(mr, fabs(v.x));
      mi = fmax(mi, fabs(v.y));
    }
  const int er = row_exponent(block_max(mr, red));
  const int ei = row_exponent(block_max(mi, red));
  if (threadIdx.x == 0) {
    scale[r1] = ldexp(1.0, er);
    scale[r2] = ldexp(1.0, ei);
  }
  for (int q = threadIdx.x; q < kfill; q += blockDim.x) {
    double2 v = make_double2(0.0, 0.0);
    if (m < rows && q < k) v = x[(size_t)m * ld + q];
    float dr[S], di[S];
    slice(ldexp(v.x, -er), dr);
    slice(ldexp(v.y, -ei), di);
#pragma unroll
    for (int s = 0; s < S; ++s) {
      planes[((size_t)s * prows + r1) * pitch + q] = dr[s];
      planes[((size_t)s * prows + r2) * pitch + q] = di[s];
    }
  }
}

// C = A B^T from the slices.  Grid (ceil(N / 64), A rows / 128), 160 threads: warp 4 (one
// elected thread) issues the TMA copies and the MMAs, warps 0-3 own tensor-memory lanes
// 0-127 and drain the 8 accumulators every DRAIN_KB k blocks into FP64 register sums.
// STACKED: A rows are the stacked real / imaginary rows of k_oz_split_stacked and C is
// complex [M][ldc] (M complex rows); else C is real [M][ldc].  Every wait is bounded: on
// expiry the CTA raises *err, waits (bounded) for its own copies, writes nothing, frees its
// tensor memory and returns.
template <bool STACKED>
__global__ void __launch_bounds__(160, 1)
    k_dgemm_oz(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, int M, int N,
               int kblocks, int arows, int brows, const double *__restrict__ sa, const double *__restrict__ sb,
               double *__restrict__ C, int ldc, int *__restrict__ err) {
  using namespace tc;
  extern __shared__ unsigned char smem_raw[];
  __shared__ uint64_t full_bar[STAGES], empty_bar[STAGES], accf_bar, acce_bar, done_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_fail;
  unsigned char *smem = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int arow0 = blockIdx.y * BM, brow0 = blockIdx.x * BN;
  const int nwin = (kblocks + DRAIN_KB - 1) / DRAIN_KB;

  if (warp == 0) tmem_alloc(&tmem_slot, TMEM_COLS);
  if (threadIdx.x == 0) {
    s_fail = 0;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&accf_bar, 1);
    mbar_init(&acce_bar, 128);
    mbar_init(&done_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_slot;
  bool ok = true;
  double sum[BN];   // epilogue warps: the lane's row of the tile
#pragma unroll
  for (int j = 0; j < BN; ++j) sum[j] = 0.0;

  if (warp == 4) {
    if (lane == 0) {
      auto issue = [&](int kb, int st) {
        unsigned char *p = smem + st * STAGE;
        mbar_expect_tx(&full_bar[st], STAGE);
        const int x = kb * BK;
        for (int s = 0; s < S; ++s) tma_load_2d(p + s * A_TILE, &ta, &full_bar[st], x, s * arows + arow0);
        for (int t = 0; t < S; ++t)
          tma_load_2d(p + S * A_TILE + t * B_TILE, &tb, &full_bar[st], x, t * brows + brow0);
      };
      int issued = 0, consumed = 0;
      for (int st = 0; st < STAGES && st < kblocks; ++st) issue(st, st), issued = st + 1;
      for (int kb = 0; kb < kblocks; ++kb) {
        const int st = kb % STAGES;
        const int win = kb / DRAIN_KB;
        const bool first = kb % DRAIN_KB == 0;
        if (!mbar_wait(&full_bar[st], (uint32_t)((kb / STAGES) & 1))) { ok = false; break; }
        consumed = kb + 1;
        // the accumulators are free once the previous window has been drained
        if (first && win >= 1 && !mbar_wait(&acce_bar, (uint32_t)((win - 1) & 1))) { ok = false; break; }
        fence_after();
        // one descriptor per stage; a tile's descriptor adds its byte offset / 16 (the stage
        // lies below 256 KB of shared memory, so the 14-bit address field cannot overflow)
        const uint64_t d0 = sdesc_sw64(smem_u32(smem + st * STAGE));
#pragma unroll
        for (int s = 0; s < S; ++s)
#pragma unroll
          for (int t = 0; t < S - s; ++t)
#pragma unroll
            for (int k8 = 0; k8 < BK / 8; ++k8)
              mma_tf32(tmem + (uint32_t)((s + t) * BN), d0 + (uint64_t)((s * A_TILE + k8 * 32) >> 4),
                       d0 + (uint64_t)((S * A_TILE + t * B_TILE + k8 * 32) >> 4), IDESC,
                       (first && s == 0 && k8 == 0) ? 0u : 1u);
        mma_commit(&empty_bar[st]);
        if (kb % DRAIN_KB == DRAIN_KB - 1 || kb == kblocks - 1) mma_commit(&accf_bar);
        // refill the stage of k block kb - 1 once its MMAs are done (those of kb are queued)
        if (kb >= 1 && kb - 1 + STAGES < kblocks) {
          const int sp = (kb - 1) % STAGES;
          if (!mbar_wait(&empty_bar[sp], (uint32_t)(((kb - 1) / STAGES) & 1))) { ok = false; break; }
          issue(kb - 1 + STAGES, sp);
          issued = kb - 1 + STAGES + 1;
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
    const uint32_t t_lane = tmem + ((uint32_t)(warp * 32) << 16);
    for (int w = 0; w < nwin; ++w) {
      if (!mbar_wait(&accf_bar, (uint32_t)(w & 1))) { ok = false; break; }
      fence_after();
#pragma unroll
      for (int d = 0; d < S; ++d) {
        const double scale = ldexp(1.0, -BITS * (d + 2));
        // the order's 64 columns in flight together, one wait
        uint32_t rr[BN];
#pragma unroll
        for (int c = 0; c < BN / 16; ++c)
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
              "%14, %15}, [%16];"
              : "=r"(rr[c * 16 + 0]), "=r"(rr[c * 16 + 1]), "=r"(rr[c * 16 + 2]), "=r"(rr[c * 16 + 3]),
                "=r"(rr[c * 16 + 4]), "=r"(rr[c * 16 + 5]), "=r"(rr[c * 16 + 6]), "=r"(rr[c * 16 + 7]),
                "=r"(rr[c * 16 + 8]), "=r"(rr[c * 16 + 9]), "=r"(rr[c * 16 + 10]), "=r"(rr[c * 16 + 11]),
                "=r"(rr[c * 16 + 12]), "=r"(rr[c * 16 + 13]), "=r"(rr[c * 16 + 14]), "=r"(rr[c * 16 + 15])
              : "r"(t_lane + (uint32_t)(d * BN + c * 16)));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int j = 0; j < BN; ++j) sum[j] = fma((double)__uint_as_float(rr[j]), scale, sum[j]);
      }
      fence_before();
      mbar_arrive(&acce_bar);
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
  // every MMA has completed and every copy has landed unless s_fail is set; only then is
  // the ring reused as staging
  if (warp < 4 && !s_fail) {
    const int row = warp * 32 + lane;           // stacked row within the tile
    const double fa = sa[arow0 + row];
    if (STACKED) {
      double *stage = reinterpret_cast<double *>(smem);   // [128][BN + 1]
#pragma unroll
      for (int j = 0; j < BN; ++j) stage[row * (BN + 1) + j] = sum[j] * fa;
      asm volatile("bar.sync 1, 128;" ::: "memory");
      // complex rows m0 .. m0 + 63: real parts in rows 0-63, imaginary parts in 64-127
      const int m0 = blockIdx.y * 64;
      for (int e = threadIdx.x; e < 64 * BN; e += 128) {
        const int rr = e / BN, cc = e % BN;
        const int gm = m0 + rr, gn = brow0 + cc;
        if (gm < M && gn < N) {
          const double fb = sb[gn];
          reinterpret_cast<double2 *>(C)[(size_t)gm * ldc + gn] =
              make_double2(stage[rr * (BN + 1) + cc] * fb, stage[(rr + 64) * (BN + 1) + cc] * fb);
        }
      }
    } else {
      const int gm = arow0 + row;
      if (gm < M)
        for (int j = 0; j < BN; ++j) {
          const int gn = brow0 + j;
          if (gn < N) C[(size_t)gm * ldc + gn] = sum[j] * fa * sb[gn];
        }
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0) tmem_dealloc(tmem, TMEM_COLS);
}

}  // namespace oz
}  // namespace ltmp2

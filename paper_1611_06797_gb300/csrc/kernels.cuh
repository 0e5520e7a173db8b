// Kernel templates of the LTMP2 hot path, templated on the real type T
// (double for the plain path, float for the precision form) and on the grid
// size N.  Step names follow Sec. III A of arXiv:1611.06797:
//   (iii) transformed states w_j^{(G' tau)} (Eqs. SCHnewstate, SCHtransmatrix),
//         built as e^{(e_j-mu)tau} P_v(tau) e^{-iG'r}|j>;
//   (iv)  Fock-like (Eq. SCHfocklike) and Hartree-like (Eq. dLTMP2Compact)
//         contractions of the co-densities <i|e^{-iGr}|w_j^{(G' tau)}>.
#pragma once
#include <type_traits>

#include "fft.cuh"
#include "plan.h"

namespace ltmp2 {

template <typename T> __device__ __forceinline__ const T *vtab(const Plan &p);
template <typename T> __device__ __forceinline__ const T *vtab_k(const Plan &p);
template <> __device__ __forceinline__ const double *vtab_k<double>(const Plan &p) { return p.vcls64; }
template <> __device__ __forceinline__ const float *vtab_k<float>(const Plan &p) { return p.vcls32; }
template <> __device__ __forceinline__ const double *vtab<double>(const Plan &p) { return p.v_aux64; }
template <> __device__ __forceinline__ const float *vtab<float>(const Plan &p) { return p.v_aux32; }

__device__ __forceinline__ int wrapn(int m, int n) {
  int r = m % n;
  return r < 0 ? r + n : r;
}
// frequency of storage slot k on an N-point axis (|m| < N/2 for every used slot)
template <int N> __device__ __forceinline__ constexpr int freq_of(int k) { return k > N / 2 ? k - N : k; }
// Elements between the occupied planes of the compact [ib][n][nxa] intermediate of the
// plane kernels: the smallest Q >= n nxa with Q = nxa (mod 16).  Then element
// (i, k, xa) sits at i Q + k nxa + xa = (i nxa + xa) + k nxa (mod 16), so the y-pass threads
// (consecutive i nxa + xa) hit distinct banks even where a warp spans two planes.
__host__ __device__ __forceinline__ int plane_stride(int n, int nxa) {
  const int base = n * nxa;
  return base + ((nxa - base) % 16 + 16) % 16;
}

// position in A of the G' carried by a slot of the current slab
__device__ __forceinline__ int slot_aux(const Plan &p, int gp0, int np, int slot) {
  return slot < np ? p.prim[gp0 + slot] : p.aux_neg[p.prim[gp0 + slot - np]];
}

// ---------------------------------------------------------------- scale factors
// virtual a: e^{-(e_a - mu) tau} (Green's function weights); occupied j: e^{(e_j - mu) tau}
template <typename T>
__global__ void k_dscale(int n_orb, int n_occ, const double *__restrict__ eps, double mu, double tau,
                         T *__restrict__ d) {
  int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n_orb) return;
  double x = (eps[a] - mu) * tau;
  d[a] = (T)exp(a < n_occ ? x : -x);
}

// ---------------------------------------------------------------- SIMT complex GEMM
// C[m][n] = sum_k opA(m,k) * B[k][n] * s_k,  opA(m,k) = A[m*lda+k] (A_KM) or A[k*lda+m],
// conjugated if A_CONJ; s_k = kscale[k] or 1.  64x64 tile, 256 threads, 4x4 per thread.
// Two-level summation (FP32 only): each 8-wide k tile is summed into a fresh partial that
// is then added to the accumulator with compensated (Kahan) summation.  A single FP32
// chain over K ~ 3000 terms biased the MP2 energy by ~2e-5 (relative) on the 24^3
// workload; the two-level sum brings it to ~1e-6, the compensation further down.
template <typename T, bool A_KM, bool A_CONJ>
__global__ void __launch_bounds__(256) k_cgemm(int M, int N, int K, const cpx<T> *__restrict__ A, int lda,
                                               const cpx<T> *__restrict__ B, int ldb,
                                               const T *__restrict__ kscale, cpx<T> *__restrict__ C,
                                               int ldc) {
  constexpr int BM = 64, BN = 64, BK = 8;
  __shared__ cpx<T> As[BK][BM];
  __shared__ cpx<T> Bs[BK][BN];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  cpx<T> acc[4][4], cmp[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = cmp[i][j] = {T(0), T(0)};
  for (int k0 = 0; k0 < K; k0 += BK) {
    for (int e = threadIdx.x; e < BM * BK; e += 256) {
      int mm, kk;
      if (A_KM) { kk = e % BK; mm = e / BK; } else { mm = e % BM; kk = e / BM; }
      const int gm = m0 + mm, gk = k0 + kk;
      cpx<T> v = {T(0), T(0)};
      if (gm < M && gk < K) v = A_KM ? A[(size_t)gm * lda + gk] : A[(size_t)gk * lda + gm];
      if (A_CONJ) v.y = -v.y;
      As[kk][mm] = v;
    }
    for (int e = threadIdx.x; e < BN * BK; e += 256) {
      const int nn = e % BN, kk = e / BN;
      const int gn = n0 + nn, gk = k0 + kk;
      cpx<T> v = {T(0), T(0)};
      if (gn < N && gk < K) {
        v = B[(size_t)gk * ldb + gn];
        if (kscale) v = cscale(v, kscale[gk]);
      }
      Bs[kk][nn] = v;
    }
    __syncthreads();
    // FP32: fresh partial per k tile (two-level sum); FP64 accumulates directly
    constexpr bool kTwoLevel = std::is_same<T, float>::value;
    cpx<T> part[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) part[i][j] = kTwoLevel ? cpx<T>{T(0), T(0)} : acc[i][j];
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      cpx<T> a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          part[i][j].x = fma(a[i].x, b[j].x, fma(-a[i].y, b[j].y, part[i][j].x));
          part[i][j].y = fma(a[i].x, b[j].y, fma(a[i].y, b[j].x, part[i][j].y));
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (kTwoLevel) kadd(acc[i][j], cmp[i][j], part[i][j]);
        else acc[i][j] = part[i][j];
      }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gm = m0 + ty + 16 * i, gn = n0 + tx + 16 * j;
      if (gm < M && gn < N) C[(size_t)gm * ldc + gn] = acc[i][j];
    }
}

// ---------------------------------------------------------------- real-basis GEMM
// C[m][n] = sum_k opA(m,k) * B[k][n] * s_k with B real and A (hence C) either real
// (TA = T) or complex (TA = cpx<T>): the Green's function in the real basis (real x real)
// and the transformed states (complex x real, two multiply-adds per term).  Same tiling
// as k_cgemm.  FP32: each 8-wide k tile is summed into a fresh partial, and the partials
// are added with compensated (Kahan) summation; with a plain FP32 outer sum the FP32
// Green's function alone left a relative error of 1.2e-6 in the direct energy of the
// 24^3 workload (most of the precision form's 2e-6).
template <typename T> __device__ __forceinline__ void rmac(T &c, T a, T b) { c = fma(a, b, c); }
template <typename T> __device__ __forceinline__ void rmac(cpx<T> &c, cpx<T> a, T b) {
  c.x = fma(a.x, b, c.x);
  c.y = fma(a.y, b, c.y);
}
template <typename T> __device__ __forceinline__ void radd(T &c, T a) { c += a; }
template <typename T> __device__ __forceinline__ void radd(cpx<T> &c, cpx<T> a) { c.x += a.x; c.y += a.y; }
// compensated (Kahan) addition c += a with running compensation e
template <typename T> __device__ __forceinline__ void kadd(T &c, T &e, T a) {
  const T y = a - e;
  const T t = c + y;
  e = (t - c) - y;
  c = t;
}
template <typename T> __device__ __forceinline__ void kadd(cpx<T> &c, cpx<T> &e, cpx<T> a) {
  kadd(c.x, e.x, a.x);
  kadd(c.y, e.y, a.y);
}
template <typename X> __device__ __forceinline__ X rzero() { return X{}; }

template <typename T, typename TA, bool A_KM>
__global__ void __launch_bounds__(256) k_rgemm(int M, int N, int K, const TA *__restrict__ A, int lda,
                                               const T *__restrict__ B, int ldb, const T *__restrict__ kscale,
                                               TA *__restrict__ C, int ldc) {
  constexpr int BM = 64, BN = 64, BK = 8;
  __shared__ TA As[BK][BM];
  __shared__ T Bs[BK][BN];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  constexpr bool kTwoLevel = std::is_same<T, float>::value;
  TA acc[4][4], cmp[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = cmp[i][j] = rzero<TA>();
  for (int k0 = 0; k0 < K; k0 += BK) {
    for (int e = threadIdx.x; e < BM * BK; e += 256) {
      int mm, kk;
      if (A_KM) { kk = e % BK; mm = e / BK; } else { mm = e % BM; kk = e / BM; }
      const int gm = m0 + mm, gk = k0 + kk;
      TA v = rzero<TA>();
      if (gm < M && gk < K) v = A_KM ? A[(size_t)gm * lda + gk] : A[(size_t)gk * lda + gm];
      As[kk][mm] = v;
    }
    for (int e = threadIdx.x; e < BN * BK; e += 256) {
      const int nn = e % BN, kk = e / BN;
      const int gn = n0 + nn, gk = k0 + kk;
      T v = T(0);
      if (gn < N && gk < K) {
        v = B[(size_t)gk * ldb + gn];
        if (kscale) v *= kscale[gk];
      }
      Bs[kk][nn] = v;
    }
    __syncthreads();
    TA part[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) part[i][j] = kTwoLevel ? rzero<TA>() : acc[i][j];
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      TA a[4];
      T b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) rmac(part[i][j], a[i], b[j]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (kTwoLevel) kadd(acc[i][j], cmp[i][j], part[i][j]);
        else acc[i][j] = part[i][j];
      }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gm = m0 + ty + 16 * i, gn = n0 + tx + 16 * j;
      if (gm < M && gn < N) C[(size_t)gm * ldc + gn] = acc[i][j];
    }
}

// Real cos/sin basis of the orbital sphere (real orbitals).  For G_q in the primary half
// (first non-zero Miller index > 0) slot q holds the cos coordinate and slot qbar (-G_q)
// the sin coordinate of the pair; slot G = 0 is its own.  The map U (plane-wave
// coefficients -> real-basis coordinates) is unitary:
//     (U x)[q]    = (x(q) + x(qbar)) / sqrt2,   (U x)[qbar] = i (x(q) - x(qbar)) / sqrt2,
// and real functions have real coordinates, so P_v(tau) = U^+ P_r U with P_r real
// symmetric and W = P_v S = U^+ (P_r (U S)).
__device__ __forceinline__ bool pw_primary(const int *m) {
  return m[0] != 0 ? m[0] > 0 : (m[1] != 0 ? m[1] > 0 : m[2] > 0);
}
template <typename T> __device__ __forceinline__ cpx<T> to_real_basis(const int *m, cpx<T> xq, cpx<T> xb) {
  constexpr T r2 = T(0.70710678118654752440084436210485);
  if (m[0] == 0 && m[1] == 0 && m[2] == 0) return xq;
  if (pw_primary(m)) return {(xq.x + xb.x) * r2, (xq.y + xb.y) * r2};
  // slot q carries the sin coordinate of the pair (qbar, q): i (x(qbar) - x(q)) / sqrt2
  return {-(xb.y - xq.y) * r2, (xb.x - xq.x) * r2};
}
template <typename T> __device__ __forceinline__ cpx<T> from_real_basis(const int *m, cpx<T> wq, cpx<T> wb) {
  constexpr T r2 = T(0.70710678118654752440084436210485);
  if (m[0] == 0 && m[1] == 0 && m[2] == 0) return wq;
  // primary q: x(q) = (w[q] - i w[qbar]) / sqrt2;  otherwise x(q) = (w[qbar] + i w[q]) / sqrt2
  if (pw_primary(m)) return {(wq.x + wb.y) * r2, (wq.y - wb.x) * r2};
  return {(wb.x - wq.y) * r2, (wb.y + wq.x) * r2};
}

// S^T in the real basis: row (slot, j) = U (e^{(e_j-mu)tau} e^{-iG'r} phi_j); unscaled
// (factor 1) for the overlap densities of the paper's route
template <typename T>
__global__ void k_gather_s_real(Plan p, int gp0, int np, cpx<T> *__restrict__ st, bool unscaled = false) {
  const int col = blockIdx.y;
  const int slot = col / p.n_occ, j = col % p.n_occ;
  const int g = slot_aux(p, gp0, np, slot);
  const int gx = p.aux_m[3 * g], gy = p.aux_m[3 * g + 1], gz = p.aux_m[3 * g + 2];
  const T dj = unscaled ? T(1) : ((const T *)p.dscale)[j];
  const int n = p.n;
  const cpx<T> *cg = (const cpx<T> *)p.cgrid + (size_t)j * n * n * n;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < p.n_pw; q += gridDim.x * blockDim.x) {
    const int *m = p.pw_m + 3 * q;
    const cpx<T> xq = cg[((size_t)wrapn(m[2] + gz, n) * n + wrapn(m[1] + gy, n)) * n + wrapn(m[0] + gx, n)];
    const cpx<T> xb = cg[((size_t)wrapn(gz - m[2], n) * n + wrapn(gy - m[1], n)) * n + wrapn(gx - m[0], n)];
    st[(size_t)col * p.n_pw + q] = cscale(to_real_basis<T>(m, xq, xb), dj);
  }
}

// W^T rows back from real-basis coordinates to plane-wave coefficients; with rowscale
// (the paper's route) row (slot, j) is also multiplied by e^{(e_j-mu)tau}
template <typename T>
__global__ void k_from_real_basis(Plan p, const cpx<T> *__restrict__ w, cpx<T> *__restrict__ out,
                                  const T *__restrict__ rowscale = nullptr) {
  const size_t row = (size_t)blockIdx.y * p.n_pw;
  const T f = rowscale ? rowscale[blockIdx.y % p.n_occ] : T(1);
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < p.n_pw; q += gridDim.x * blockDim.x)
    out[row + q] = cscale(from_real_basis<T>(p.pw_m + 3 * q, w[row + q], w[row + p.pw_pair[q]]), f);
}

// out[c][r] = in[r][c] for a rows x cols matrix of T (32 x 32 tiles through shared memory)
template <typename T>
__global__ void k_transpose(int rows, int cols, const T *__restrict__ in, T *__restrict__ out) {
  __shared__ T tile[32][33];
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

// ---------------------------------------------------------------- gather S^T
// S^T[(slot, j)][q] = e^{(e_j - mu) tau} c_j((G_q + G'_slot) mod grid): the plane-wave
// coefficients of e^{-iG'r} phi_j restricted to the orbital sphere, scaled.
template <typename T>
__global__ void k_gather_s(Plan p, int gp0, int np, cpx<T> *__restrict__ st) {
  const int col = blockIdx.y;
  const int slot = col / p.n_occ, j = col % p.n_occ;
  const int g = slot_aux(p, gp0, np, slot);
  const int gx = p.aux_m[3 * g], gy = p.aux_m[3 * g + 1], gz = p.aux_m[3 * g + 2];
  const T dj = ((const T *)p.dscale)[j];
  const int n = p.n;
  const cpx<T> *cg = (const cpx<T> *)p.cgrid + (size_t)j * n * n * n;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < p.n_pw; q += gridDim.x * blockDim.x) {
    const int wx = wrapn(p.pw_m[3 * q] + gx, n), wy = wrapn(p.pw_m[3 * q + 1] + gy, n),
              wz = wrapn(p.pw_m[3 * q + 2] + gz, n);
    st[(size_t)col * p.n_pw + q] = cscale(cg[((size_t)wz * n + wy) * n + wx], dj);
  }
}

// scatter rows of coefficients (internal order) onto the full grid, layout [row][z][y][x]
template <typename T>
__global__ void k_scatter_grid(Plan p, int rows, const cpx<T> *__restrict__ c, cpx<T> *__restrict__ grid) {
  const int r = blockIdx.y;
  const int n = p.n;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < p.n_pw; q += gridDim.x * blockDim.x) {
    const int wx = wrapn(p.pw_m[3 * q], n), wy = wrapn(p.pw_m[3 * q + 1], n), wz = wrapn(p.pw_m[3 * q + 2], n);
    grid[(size_t)r * n * n * n + ((size_t)wz * n + wy) * n + wx] = c[(size_t)r * p.n_pw + q];
  }
}

// ---------------------------------------------------------------- inverse z transform
// For column vector col of W^T (plane-wave coefficients of one w_j^{G'}, internal order)
// and orbital-disk column d: place the m3 range on the z axis and inverse-transform.
// Output z1[col][t3][d].
template <typename T, int N>
__global__ void k_w_zinv(Plan p, int ld_in, const cpx<T> *__restrict__ wt, cpx<T> *__restrict__ z1) {
  const int col = blockIdx.y;
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= p.n_dorb) return;
  const int4 c = p.dorb[d];
  const cpx<T> *w = wt + (size_t)col * ld_in + p.dorb_off[d];
  cpx<T> a[N];
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const int m = freq_of<N>(k);
    a[k] = (m >= c.z && m <= c.w) ? w[m - c.z] : cpx<T>{T(0), T(0)};
  }
  LineFFT<T, N, +1>::run(a);
  cpx<T> *z = z1 + (size_t)col * N * p.n_dorb + d;
#pragma unroll
  for (int k = 0; k < N; ++k) z[(size_t)k * p.n_dorb] = a[k];
}

// ---------------------------------------------------------------- plane kernel
// Block (z, col).  Phase 1: the orbital-disk values of plane z -> inverse y then x
// transform = w_j^{G'}(x, y, z) in shared memory.  Phase 2, for each occupied i:
// conj(phi_i) * w_j^{G'} -> forward x then y transform, keep the aux disk, write
// tbuf[(col, i)][z][d_aux].  IB occupied planes are transformed together.
template <typename T, int N>
__device__ __forceinline__ void plane_inverse(const Plan &p, const cpx<T> *__restrict__ zrow, cpx<T> *xp) {
  constexpr int P = N + 1;
  const int tid = threadIdx.x, nth = blockDim.x;
  for (int e = tid; e < N * P; e += nth) xp[e] = {T(0), T(0)};
  __syncthreads();
  for (int d = tid; d < p.n_dorb; d += nth) {
    const int4 c = p.dorb[d];
    xp[wrapn(c.y, N) * P + wrapn(c.x, N)] = zrow[d];
  }
  __syncthreads();
  const int nxo = p.mxhi_orb - p.mxlo_orb + 1;
  for (int t = tid; t < nxo; t += nth) {
    const int x = wrapn(p.mxlo_orb + t, N);
    cpx<T> a[N];
#pragma unroll
    for (int k = 0; k < N; ++k) a[k] = xp[k * P + x];
    LineFFT<T, N, +1>::run(a);
#pragma unroll
    for (int k = 0; k < N; ++k) xp[k * P + x] = a[k];
  }
  __syncthreads();
  for (int t = tid; t < N; t += nth) {
    cpx<T> a[N];
#pragma unroll
    for (int k = 0; k < N; ++k) a[k] = xp[t * P + k];
    LineFFT<T, N, +1>::run(a);
#pragma unroll
    for (int k = 0; k < N; ++k) xp[t * P + k] = a[k];
  }
  __syncthreads();
}

template <typename T, int N>
__global__ void k_planes(Plan p, int ib, const cpx<T> *__restrict__ z1, cpx<T> *__restrict__ tbuf) {
  constexpr int P = N + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T> *xp = reinterpret_cast<cpx<T> *>(smem_raw);
  cpx<T> *wk = xp + N * P;
  const int z = blockIdx.x, col = blockIdx.y;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int no = p.n_occ;
  plane_inverse<T, N>(p, z1 + ((size_t)col * N + z) * p.n_dorb, xp);
  const cpx<T> *u = (const cpx<T> *)p.u;
  const int nxa = p.mxhi_aux - p.mxlo_aux + 1;
  // occupied i of this column: all, or the kept list when exchange pairs are screened
  const int jcol = col % no;
  const int ni = p.keep_count ? p.keep_count[jcol] : no;
  const int *ilist = p.keep_count ? p.keep_list + (size_t)jcol * no : nullptr;
  for (int i0 = 0; i0 < ni; i0 += ib) {
    const int nb = min(ib, ni - i0);
    for (int e = tid; e < nb * N * N; e += nth) {
      const int il = e / (N * N), r = e % (N * N), y = r / N, x = r % N;
      const int iocc = ilist ? ilist[i0 + il] : i0 + il;
      const cpx<T> uu = u[((size_t)iocc * N + z) * N * N + r];
      wk[(il * N + y) * P + x] = cmul(cconj(uu), xp[y * P + x]);
    }
    __syncthreads();
    for (int t = tid; t < nb * N; t += nth) {
      cpx<T> *row = wk + t * P;  // (il * N + y) * P
      cpx<T> a[N];
#pragma unroll
      for (int k = 0; k < N; ++k) a[k] = row[k];
      LineFFT<T, N, -1>::run(a);
#pragma unroll
      for (int k = 0; k < N; ++k) row[k] = a[k];
    }
    __syncthreads();
    for (int t = tid; t < nb * nxa; t += nth) {
      const int il = t / nxa, x = wrapn(p.mxlo_aux + t % nxa, N);
      cpx<T> *base = wk + il * N * P;
      cpx<T> a[N];
#pragma unroll
      for (int k = 0; k < N; ++k) a[k] = base[k * P + x];
      LineFFT<T, N, -1>::run(a);
#pragma unroll
      for (int k = 0; k < N; ++k) base[k * P + x] = a[k];
    }
    __syncthreads();
    for (int e = tid; e < nb * p.n_daux; e += nth) {
      const int il = e / p.n_daux, d = e % p.n_daux;
      const int4 c = p.daux[d];
      const size_t item = (size_t)col * no + (ilist ? ilist[i0 + il] : i0 + il);
      tbuf[(item * N + z) * p.n_daux + d] = wk[(il * N + wrapn(c.y, N)) * P + wrapn(c.x, N)];
    }
    __syncthreads();
  }
}

// Same result as k_planes, fewer shared-memory passes.  Per block of ib occupied i:
//  product: conj(phi_i) w_j^{G'} for the block's planes, loaded coalesced into shared
//           memory (pitch P = N + 1);
//  x pass : thread (i, y) transforms its row in registers and writes back, in place,
//           only the m1 of the aux range (columns 0 .. nxa-1 of the row);
//  y pass : thread (i, m1) transforms its column and writes only the aux-disk entries,
//           compactly in disk order;
//  copy   : coalesced copy of the compact plane to tbuf[(col, i)][z][d_aux].
template <typename T, int N>
__global__ void k_planes2(Plan p, int ib, const cpx<T> *__restrict__ z1, cpx<T> *__restrict__ tbuf) {
  constexpr int P = N + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T> *xp = reinterpret_cast<cpx<T> *>(smem_raw);
  const int nxa = p.mxhi_aux - p.mxlo_aux + 1;
  const int nd = p.n_daux;
  cpx<T> *wk = xp + N * P;                    // [ib][N][P]
  cpx<T> *ob = wk + (size_t)ib * N * P;       // [ib][nd]
  int *xs = reinterpret_cast<int *>(ob + (size_t)ib * nd);   // per m1: first disk column, m2 lo, m2 hi
  const int z = blockIdx.x, col = blockIdx.y;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int no = p.n_occ;
  for (int t = tid; t < nxa; t += nth) { xs[3 * t] = 0; xs[3 * t + 1] = 1; xs[3 * t + 2] = 0; }
  __syncthreads();
  for (int d = tid; d < nd; d += nth) {
    const int4 c = p.daux[d];
    const int xa = c.x - p.mxlo_aux;
    if (d == 0 || p.daux[d - 1].x != c.x) { xs[3 * xa] = d; xs[3 * xa + 1] = c.y; }
    if (d == nd - 1 || p.daux[d + 1].x != c.x) xs[3 * xa + 2] = c.y;
  }
  plane_inverse<T, N>(p, z1 + ((size_t)col * N + z) * p.n_dorb, xp);   // ends with a barrier
  const cpx<T> *u = (const cpx<T> *)p.u;
  // occupied i of this column: all, or the kept list when exchange pairs are screened
  const int jcol = col % no;
  const int ni = p.keep_count ? p.keep_count[jcol] : no;
  const int *ilist = p.keep_count ? p.keep_list + (size_t)jcol * no : nullptr;
  for (int i0 = 0; i0 < ni; i0 += ib) {
    const int nb = min(ib, ni - i0);
    for (int e = tid; e < nb * N * N; e += nth) {
      const int il = e / (N * N), r = e % (N * N), y = r / N, x = r % N;
      const int iocc = ilist ? ilist[i0 + il] : i0 + il;
      const cpx<T> uu = u[((size_t)iocc * N + z) * N * N + r];
      wk[(il * N + y) * P + x] = cmul(cconj(uu), xp[y * P + x]);
    }
    __syncthreads();
    for (int t = tid; t < nb * N; t += nth) {
      cpx<T> *row = wk + (size_t)t * P;    // (il * N + y) * P
      cpx<T> a[N];
#pragma unroll
      for (int k = 0; k < N; ++k) a[k] = row[k];
      LineFFT<T, N, -1>::run(a);
#pragma unroll
      for (int k = 0; k < N; ++k) {
        const int m = freq_of<N>(k);
        if (m >= p.mxlo_aux && m <= p.mxhi_aux) row[m - p.mxlo_aux] = a[k];
      }
    }
    __syncthreads();
    for (int t = tid; t < nb * nxa; t += nth) {
      const int il = t / nxa, xa = t % nxa;
      const cpx<T> *src = wk + (size_t)il * N * P + xa;
      cpx<T> b[N];
#pragma unroll
      for (int k = 0; k < N; ++k) b[k] = src[k * P];
      LineFFT<T, N, -1>::run(b);
      const int d0 = xs[3 * xa], lo = xs[3 * xa + 1], hi = xs[3 * xa + 2];
      cpx<T> *o = ob + (size_t)il * nd + d0 - lo;
#pragma unroll
      for (int k = 0; k < N; ++k) {
        const int m = freq_of<N>(k);
        if (m >= lo && m <= hi) o[m] = b[k];
      }
    }
    __syncthreads();
    for (int e = tid; e < nb * nd; e += nth) {
      const int il = e / nd, d = e % nd;
      const size_t item = (size_t)col * no + (ilist ? ilist[i0 + il] : i0 + il);
      tbuf[(item * N + z) * nd + d] = ob[(size_t)il * nd + d];
    }
  }
}

// Same result as k_planes, with the product formed in registers.  Per block of ib
// occupied i:
//  x pass : thread (i, y) loads row y of phi_i (from the plane-transposed copy, coalesced
//           across the warp, L2 resident) and of w_j^{G'} (shared), multiplies conj(phi_i) w
//           in registers, transforms, and keeps only the m1 of the aux range: a compact
//           [ib][N][nxa] intermediate (nxa is odd, so the row pitch spreads the banks);
//  y pass : thread (i, m1) transforms its column and writes it back in place (consecutive
//           threads, consecutive addresses);
//  copy   : the aux-disk entries gathered through a per-block table (consecutive disk
//           columns of one m1 are nxa apart: no bank conflicts) and written coalesced to
//           tbuf[(col, i)][z][d_aux].
template <typename T, int N>
__device__ __forceinline__ void planes3_body(const Plan &p, int ib, int z, int col, const cpx<T> *__restrict__ z1,
                                             cpx<T> *__restrict__ tbuf, unsigned char *smem_raw) {
  constexpr int P = N + 1;
  cpx<T> *xp = reinterpret_cast<cpx<T> *>(smem_raw);
  const int nxa = p.mxhi_aux - p.mxlo_aux + 1;   // odd: the aux sphere is symmetric
  const int nd = p.n_daux;
  const int Q = plane_stride(N, nxa);
  cpx<T> *wk = xp + N * P;                    // [ib] planes of [N][nxa], Q elements apart
  int *ytab = reinterpret_cast<int *>(wk + (size_t)ib * Q);   // [nd] position of disk column d in a plane of wk
  const int tid = threadIdx.x, nth = blockDim.x;
  const int no = p.n_occ;
  const int mlo = p.mxlo_aux, mhi = p.mxhi_aux;
  const unsigned inv_nxa = ((1u << 20) + nxa - 1) / nxa;   // ceil(2^20 / nxa)
  for (int d = tid; d < nd; d += nth) {
    const int4 c = p.daux[d];
    ytab[d] = wrapn(c.y, N) * nxa + (c.x - mlo);
  }
  plane_inverse<T, N>(p, z1 + ((size_t)col * N + z) * p.n_dorb, xp);   // ends with a barrier
  const cpx<T> *ut = (const cpx<T> *)p.ut;
  const T *utr = (const T *)p.utr;
  const int jcol = col % no;
  const int ni = p.keep_count ? p.keep_count[jcol] : no;
  const int *ilist = p.keep_count ? p.keep_list + (size_t)jcol * no : nullptr;
  for (int i0 = 0; i0 < ni; i0 += ib) {
    const int nb = min(ib, ni - i0);
    for (int t = tid; t < nb * N; t += nth) {
      const int il = t / N, y = t - il * N;
      const int iocc = ilist ? ilist[i0 + il] : i0 + il;
      cpx<T> a[N];
      // row y of phi_i from the transposed plane: element x at x N + y, so the threads of
      // a warp (consecutive y) read consecutive addresses.  Real orbitals: phi_i is real,
      // so conj(phi_i) w is two real products per point and half the bytes are read.
      const size_t urow = ((size_t)iocc * N + z) * N * N + y;
      const cpx<T> *wr = xp + y * P;
      if (utr) {
#pragma unroll
        for (int k = 0; k < N; ++k) a[k] = cscale(wr[k], utr[urow + k * N]);
      } else {
#pragma unroll
        for (int k = 0; k < N; ++k) a[k] = cmul(cconj(ut[urow + k * N]), wr[k]);
      }
      LineFFT<T, N, -1>::run(a);
      cpx<T> *row = wk + (size_t)il * Q + y * nxa - mlo;   // row[m] for m in [mlo, mhi]
#pragma unroll
      for (int k = 0; k < N; ++k) {
        const int m = freq_of<N>(k);
        if (m >= mlo && m <= mhi) row[m] = a[k];
      }
    }
    __syncthreads();
    for (int t = tid; t < nb * nxa; t += nth) {
      // t / nxa by an exact multiply-shift: t < 2^12 and nxa < 2^7 keep the rounding of the
      // reciprocal below one part in nxa
      const int il = (int)(((unsigned)t * inv_nxa) >> 20), xa = t - il * nxa;
      cpx<T> *src = wk + (size_t)il * Q + xa;
      cpx<T> b[N];
#pragma unroll
      for (int k = 0; k < N; ++k) b[k] = src[k * nxa];
      LineFFT<T, N, -1>::run(b);
#pragma unroll
      for (int k = 0; k < N; ++k) src[k * nxa] = b[k];
    }
    __syncthreads();
    for (int il = 0; il < nb; ++il) {
      const size_t item = (size_t)col * no + (ilist ? ilist[i0 + il] : i0 + il);
      cpx<T> *dst = tbuf + (item * N + z) * nd;
      const cpx<T> *src = wk + (size_t)il * Q;
      for (int d = tid; d < nd; d += nth) dst[d] = src[ytab[d]];
    }
    __syncthreads();
  }
}

template <typename T, int N>
__global__ void k_planes3(Plan p, int ib, const cpx<T> *__restrict__ z1, cpx<T> *__restrict__ tbuf) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  planes3_body<T, N>(p, ib, blockIdx.x, blockIdx.y, z1, tbuf, smem_raw);
}

// Same result as k_planes3 with no block barrier after the w plane is transformed: each of
// the block's kPlaneWarps warps takes its own occupied i (ib at a time, in its own slice of
// shared memory) through the x pass, the y pass and the disk gather, synchronising only
// within the warp.  Warps run out of step, so one warp's FFT arithmetic hides another's
// shared-memory and L2 latency; ib items per step keep the lanes busy for N < 32.
constexpr int kPlaneWarps = 4;
template <typename T, int N>
__global__ void __launch_bounds__(32 * kPlaneWarps) k_planes4(Plan p, int ib, const cpx<T> *__restrict__ z1,
                                                              cpx<T> *__restrict__ tbuf) {
  constexpr int P = N + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T> *xp = reinterpret_cast<cpx<T> *>(smem_raw);
  const int nxa = p.mxhi_aux - p.mxlo_aux + 1;
  const int nd = p.n_daux;
  const int Q = plane_stride(N, nxa);
  cpx<T> *wk_all = xp + N * P;                                          // [warps][ib] planes, Q apart
  int *ytab = reinterpret_cast<int *>(wk_all + (size_t)kPlaneWarps * ib * Q);   // [nd]
  const int z = blockIdx.x, col = blockIdx.y;
  const int no = p.n_occ;
  const int mlo = p.mxlo_aux, mhi = p.mxhi_aux;
  const unsigned inv_nxa = ((1u << 20) + nxa - 1) / nxa;   // ceil(2^20 / nxa)
  for (int d = threadIdx.x; d < nd; d += blockDim.x) {
    const int4 c = p.daux[d];
    ytab[d] = wrapn(c.y, N) * nxa + (c.x - mlo);
  }
  plane_inverse<T, N>(p, z1 + ((size_t)col * N + z) * p.n_dorb, xp);   // ends with a barrier
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  cpx<T> *wk = wk_all + (size_t)warp * ib * Q;
  const cpx<T> *ut = (const cpx<T> *)p.ut;
  const T *utr = (const T *)p.utr;
  const int jcol = col % no;
  const int ni = p.keep_count ? p.keep_count[jcol] : no;
  const int *ilist = p.keep_count ? p.keep_list + (size_t)jcol * no : nullptr;
  for (int i0 = warp * ib; i0 < ni; i0 += kPlaneWarps * ib) {
    const int nb = min(ib, ni - i0);
    for (int t = lane; t < nb * N; t += 32) {
      const int il = t / N, y = t - il * N;
      const int iocc = ilist ? ilist[i0 + il] : i0 + il;
      cpx<T> a[N];
      const size_t urow = ((size_t)iocc * N + z) * N * N + y;
      const cpx<T> *wr = xp + y * P;
      if (utr) {
#pragma unroll
        for (int k = 0; k < N; ++k) a[k] = cscale(wr[k], utr[urow + k * N]);
      } else {
#pragma unroll
        for (int k = 0; k < N; ++k) a[k] = cmul(cconj(ut[urow + k * N]), wr[k]);
      }
      LineFFT<T, N, -1>::run(a);
      cpx<T> *row = wk + (size_t)il * Q + y * nxa - mlo;
#pragma unroll
      for (int k = 0; k < N; ++k) {
        const int m = freq_of<N>(k);
        if (m >= mlo && m <= mhi) row[m] = a[k];
      }
    }
    __syncwarp();
    for (int t = lane; t < nb * nxa; t += 32) {
      const int il = (int)(((unsigned)t * inv_nxa) >> 20), xa = t - il * nxa;   // t / nxa, exact for t < 2^12
      cpx<T> *src = wk + (size_t)il * Q + xa;
      cpx<T> b[N];
#pragma unroll
      for (int k = 0; k < N; ++k) b[k] = src[k * nxa];
      LineFFT<T, N, -1>::run(b);
#pragma unroll
      for (int k = 0; k < N; ++k) src[k * nxa] = b[k];
    }
    __syncwarp();
    for (int il = 0; il < nb; ++il) {
      const size_t item = (size_t)col * no + (ilist ? ilist[i0 + il] : i0 + il);
      cpx<T> *dst = tbuf + (item * N + z) * nd;
      const cpx<T> *src = wk + (size_t)il * Q;
      for (int d = lane; d < nd; d += 32) dst[d] = src[ytab[d]];
    }
    __syncwarp();
  }
}

// setup: real-space occupied orbitals u[j][z][y][x] from z1 (cols = occupied orbitals)
// (and the plane-transposed copy outt[j][z][x][y] that the plane kernel reads row-wise)
template <typename T, int N>
__global__ void k_planes_store(Plan p, const cpx<T> *__restrict__ z1, cpx<T> *__restrict__ out,
                               cpx<T> *__restrict__ outt, T *__restrict__ outr) {
  constexpr int P = N + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T> *xp = reinterpret_cast<cpx<T> *>(smem_raw);
  const int z = blockIdx.x, col = blockIdx.y;
  plane_inverse<T, N>(p, z1 + ((size_t)col * N + z) * p.n_dorb, xp);
  for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
    const int y = e / N, x = e % N;
    out[((size_t)col * N + z) * N * N + e] = xp[y * P + x];
    const cpx<T> v = xp[x * P + y];   // e = x' N + y' with x' = y, y' = x
    outt[((size_t)col * N + z) * N * N + e] = v;
    if (outr) outr[((size_t)col * N + z) * N * N + e] = v.x;
  }
}

// ---------------------------------------------------------------- column kernel
// Block = one pair of co-density items.  Forward z transform of every aux-disk column
// of item A (kept in shared memory, indexed like A) and of the partner item B, then
//   general: X = sum_G v(G) M_A(-G) M_B(G)   (A = (i,j,G'), B = (j,i,-G'))
//   real   : X = sum_G v(G) M_A(G) conj(M_B(G))   (A = (i,j,G'), B = (j,i,G'))
// M values are unnormalised (N^3 times the co-density).  Diagonal items also store
// M_ii(G;G') in mdiag[slot][G][i] for the direct term.
template <typename T>
__device__ __forceinline__ void block_reduce_store(double ax, double ay, double2 *dst, double2 *dst_t) {
  __shared__ double red[2][32];
  for (int o = 16; o > 0; o >>= 1) {
    ax += __shfl_xor_sync(0xffffffffu, ax, o);
    ay += __shfl_xor_sync(0xffffffffu, ay, o);
  }
  const int w = threadIdx.x / 32, l = threadIdx.x % 32, nw = (blockDim.x + 31) / 32;
  if (l == 0) { red[0][w] = ax; red[1][w] = ay; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sx = 0, sy = 0;
    for (int k = 0; k < nw; ++k) { sx += red[0][k]; sy += red[1][k]; }
    *dst = make_double2(sx, sy);
    if (dst_t) *dst_t = make_double2(sx, -sy);
  }
}

// Level-resolved sums (internal cutoff extrapolation): terms staged per G in PR[]; warp w
// sums the groups n = w, w + nw, ... of lev_order (G with L(G) = n + 1), so each level
// costs one warp reduction.  Thread 0 then runs from the innermost level outwards: the
// running sum is the sum over A_n, stored for n = 1 in dst1 and for n >= 2 in lev.
template <typename T>
__device__ __forceinline__ void level_reduce_store(const Plan &p, const cpx<T> *PR, size_t elem, size_t elem_t,
                                                   bool transpose, double2 *dst1, double2 *lev) {
  __shared__ double lred[kMaxLevels][2];
  const int tid = threadIdx.x, nth = blockDim.x;
  const int w = tid / 32, l = tid % 32, nw = nth / 32;   // blockDim.x is a multiple of 32
  for (int n = w; n < p.n_lev; n += nw) {
    T bx = T(0), by = T(0);
    for (int k = p.lev_start[n] + l; k < p.lev_start[n + 1]; k += 32) {
      const cpx<T> t = PR[p.lev_order[k]];
      bx += t.x;
      by += t.y;
    }
    double dx = (double)bx, dy = (double)by;
    for (int o = 16; o > 0; o >>= 1) {
      dx += __shfl_xor_sync(0xffffffffu, dx, o);
      dy += __shfl_xor_sync(0xffffffffu, dy, o);
    }
    if (l == 0) { lred[n][0] = dx; lred[n][1] = dy; }
  }
  __syncthreads();
  if (tid == 0) {
    double rx = 0.0, ry = 0.0;
    for (int n = p.n_lev - 1; n >= 0; --n) {
      rx += lred[n][0];
      ry += lred[n][1];
      double2 *base = n == 0 ? dst1 : lev + (size_t)n * p.lev_stride;
      base[elem] = make_double2(rx, ry);
      if (transpose) base[elem_t] = make_double2(rx, -ry);
    }
  }
}

template <typename T, int N, bool LEV>
__device__ __forceinline__ void zcol_body(const Plan &p, int gp0, int np, int pair, const cpx<T> *__restrict__ tbuf,
                                          cpx<T> *__restrict__ mdiag, double2 *__restrict__ sx,
                                          unsigned char *smem_raw) {
  cpx<T> *MA = reinterpret_cast<cpx<T> *>(smem_raw);
  cpx<T> *PR = MA + p.n_aux;   // LEV only: v(G) times the product, per G
  const int no = p.n_occ;
  const int tid = threadIdx.x, nth = blockDim.x;
  int i, j, gpl, slotA, slotB;
  bool self = false;
  if (!p.real_orb) {
    gpl = pair / (no * no);
    const int r = pair % (no * no);
    i = r / no; j = r % no;
    slotA = gpl; slotB = gpl + np;
  } else {
    const int npairs = no * (no + 1) / 2;
    gpl = pair / npairs;
    int t = pair % npairs;
    i = 0;
    while (t >= no - i) { t -= no - i; ++i; }
    j = i + t;
    slotA = slotB = gpl;
    self = (i == j);
  }
  const bool diag = (i == j);
  if (p.pair_keep && !diag && !p.pair_keep[i * no + j]) {   // screened: exchange estimated elsewhere
    if (threadIdx.x == 0) {
      for (int n = 0; n < (LEV ? p.n_lev : 1); ++n) {
        double2 *base = n == 0 ? sx : p.sxl + (size_t)n * p.lev_stride;
        base[((size_t)gpl * no + i) * no + j] = make_double2(0.0, 0.0);
        if (p.real_orb) base[((size_t)gpl * no + j) * no + i] = make_double2(0.0, 0.0);
      }
    }
    return;
  }
  const size_t itemA = ((size_t)slotA * no + j) * no + i;   // (i, j, slotA)
  const size_t itemB = ((size_t)slotB * no + i) * no + j;   // (j, i, slotB)
  const T *v = vtab<T>(p);
  const int nd = p.n_daux;
  T accx = T(0), accy = T(0);
  for (int d = tid; d < nd; d += nth) {
    const int4 c = p.daux[d];
    const int off = p.daux_off[d];
    const cpx<T> *src = tbuf + itemA * N * nd + d;
    cpx<T> a[N];
#pragma unroll
    for (int k = 0; k < N; ++k) a[k] = src[(size_t)k * nd];
    LineFFT<T, N, -1>::run(a);
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const int m = freq_of<N>(k);
      if (m >= c.z && m <= c.w) {
        const int g = off + m - c.z;
        MA[g] = a[k];
        if (diag) mdiag[((size_t)slotA * p.n_aux + g) * no + i] = a[k];
        if (self) {
          const T t = v[g] * (a[k].x * a[k].x + a[k].y * a[k].y);
          if (LEV) PR[g] = {t, T(0)};
          else accx += t;
        }
      }
    }
  }
  __syncthreads();
  if (!self) {
    for (int d = tid; d < nd; d += nth) {
      const int4 c = p.daux[d];
      const int off = p.daux_off[d];
      const cpx<T> *src = tbuf + itemB * N * nd + d;
      cpx<T> a[N];
#pragma unroll
      for (int k = 0; k < N; ++k) a[k] = src[(size_t)k * nd];
      LineFFT<T, N, -1>::run(a);
#pragma unroll
      for (int k = 0; k < N; ++k) {
        const int m = freq_of<N>(k);
        if (m >= c.z && m <= c.w) {
          const int g = off + m - c.z;
          cpx<T> prod;
          if (!p.real_orb) {
            prod = cmul(MA[p.aux_neg[g]], a[k]);
            if (diag) mdiag[((size_t)slotB * p.n_aux + g) * no + i] = a[k];
          } else {
            prod = cmulconj(MA[g], a[k]);
          }
          if (LEV) {
            PR[g] = {v[g] * prod.x, v[g] * prod.y};
          } else {
            accx += v[g] * prod.x;
            accy += v[g] * prod.y;
          }
        }
      }
    }
  }
  const size_t elem = ((size_t)gpl * no + i) * no + j, elem_t = ((size_t)gpl * no + j) * no + i;
  const bool transpose = p.real_orb && i != j;
  if constexpr (LEV) {
    __syncthreads();
    level_reduce_store<T>(p, PR, elem, elem_t, transpose, sx, p.sxl);
  } else {
    block_reduce_store<T>((double)accx, (double)accy, sx + elem, transpose ? sx + elem_t : nullptr);
  }
}

template <typename T, int N, bool LEV>
__global__ void __launch_bounds__(256) k_zcol(Plan p, int gp0, int np, const cpx<T> *__restrict__ tbuf,
                                              cpx<T> *__restrict__ mdiag, double2 *__restrict__ sx) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  zcol_body<T, N, LEV>(p, gp0, np, blockIdx.x, tbuf, mdiag, sx, smem_raw);
}

// ---------------------------------------------------------------- direct term
// Y_ij(G') = sum_G v(G) M_ii(G;G') M_jj(-G;-G')  (general)  or  M_ii(G;G') conj(M_jj(G;G')) (real)
template <typename T, bool LEV>
__global__ void k_direct(Plan p, int np, const cpx<T> *__restrict__ mdiag, double2 *__restrict__ yd) {
  const int gpl = blockIdx.x, i = blockIdx.y;
  const int no = p.n_occ;
  const int slotA = gpl, slotB = p.real_orb ? gpl : gpl + np;
  const T *v = vtab<T>(p);
  const cpx<T> *MA = mdiag + (size_t)slotA * p.n_aux * no;
  const cpx<T> *MB = mdiag + (size_t)slotB * p.n_aux * no;
  for (int j = threadIdx.x; j < no; j += blockDim.x) {
    if constexpr (LEV) {
      // groups from the innermost level outwards; the running sum is the sum over A_n
      double ax = 0, ay = 0;
      for (int n = p.n_lev - 1; n >= 0; --n) {
        T cx = T(0), cy = T(0);
        int cnt = 0;
        for (int k = p.lev_start[n]; k < p.lev_start[n + 1]; ++k) {
          const int g = p.lev_order[k];
          const cpx<T> x = MA[(size_t)g * no + i];
          cpx<T> prod;
          if (!p.real_orb) prod = cmul(x, MB[(size_t)p.aux_neg[g] * no + j]);
          else prod = cmulconj(x, MB[(size_t)g * no + j]);
          cx += v[g] * prod.x;
          cy += v[g] * prod.y;
          if ((++cnt & 31) == 0) { ax += (double)cx; ay += (double)cy; cx = cy = T(0); }
        }
        ax += (double)cx; ay += (double)cy;
        double2 *base = n == 0 ? yd : p.ydl + (size_t)n * p.lev_stride;
        base[((size_t)gpl * no + i) * no + j] = make_double2(ax, ay);
      }
      continue;
    }
    double ax = 0, ay = 0;
    T cx = T(0), cy = T(0);
    for (int g = 0; g < p.n_aux; ++g) {
      const cpx<T> x = MA[(size_t)g * no + i];
      cpx<T> prod;
      if (!p.real_orb) prod = cmul(x, MB[(size_t)p.aux_neg[g] * no + j]);
      else prod = cmulconj(x, MB[(size_t)g * no + j]);
      cx += v[g] * prod.x;
      cy += v[g] * prod.y;
      if ((g & 31) == 31) { ax += (double)cx; ay += (double)cy; cx = cy = T(0); }
    }
    ax += (double)cx; ay += (double)cy;
    yd[((size_t)gpl * no + i) * no + j] = make_double2(ax, ay);
  }
}

// ---------------------------------------------------------------- pair descriptors
// Per occupied orbital: z_k = (1/N) sum_t |u(t)|^2 exp(2 pi i t_k / n), k = x, y, z
// (periodic centroid from arg z_k, spread from |z_k|).  out[i][6] = (Re, Im) x 3.
// Direct term, tiled: block (G' of the slab, 32 x 32 tile of (i, j)); the G sum runs in
// chunks of 32 staged in shared memory (M_ii for the tile's i, M_jj at -G or conjugated for
// its j, v(G)).  Each thread owns one j and four i; every 32-term chunk is summed in T and
// added to a double accumulator, as in k_direct.
template <typename T>
__global__ void __launch_bounds__(256) k_direct_tiled(Plan p, int np, const cpx<T> *__restrict__ mdiag,
                                                      double2 *__restrict__ yd) {
  constexpr int TC = 32;
  __shared__ cpx<T> As[TC][TC + 1], Bs[TC][TC + 1];
  __shared__ T vs[TC];
  const int gpl = blockIdx.x, i0 = blockIdx.y * TC, j0 = blockIdx.z * TC;
  const int no = p.n_occ, naux = p.n_aux;
  const int tx = threadIdx.x % TC, ty = threadIdx.x / TC;   // 32 x 8 threads
  const int slotA = gpl, slotB = p.real_orb ? gpl : gpl + np;
  const T *v = vtab<T>(p);
  const cpx<T> *MA = mdiag + (size_t)slotA * naux * no;
  const cpx<T> *MB = mdiag + (size_t)slotB * naux * no;
  double ax[4] = {0, 0, 0, 0}, ay[4] = {0, 0, 0, 0};
  for (int g0 = 0; g0 < naux; g0 += TC) {
    for (int e = threadIdx.x; e < TC * TC; e += blockDim.x) {
      const int gg = e / TC, c = e % TC, g = g0 + gg;
      cpx<T> a = {T(0), T(0)}, b = {T(0), T(0)};
      if (g < naux) {
        if (i0 + c < no) a = MA[(size_t)g * no + i0 + c];
        if (j0 + c < no) b = p.real_orb ? MB[(size_t)g * no + j0 + c] : MB[(size_t)p.aux_neg[g] * no + j0 + c];
      }
      As[gg][c] = a;
      Bs[gg][c] = b;
    }
    if (threadIdx.x < TC) vs[threadIdx.x] = g0 + threadIdx.x < naux ? v[g0 + threadIdx.x] : T(0);
    __syncthreads();
    T cx[4] = {T(0), T(0), T(0), T(0)}, cy[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll 8
    for (int gg = 0; gg < TC; ++gg) {
      const cpx<T> b = Bs[gg][tx];
      const T vg = vs[gg];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const cpx<T> a = As[gg][ty + 8 * k];
        const cpx<T> prod = p.real_orb ? cmulconj(a, b) : cmul(a, b);
        cx[k] += vg * prod.x;
        cy[k] += vg * prod.y;
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) { ax[k] += (double)cx[k]; ay[k] += (double)cy[k]; }
    __syncthreads();
  }
  const int j = j0 + tx;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int i = i0 + ty + 8 * k;
    if (i < no && j < no) yd[((size_t)gpl * no + i) * no + j] = make_double2(ax[k], ay[k]);
  }
}

template <typename T> __global__ void k_orb_moments(Plan p, double *__restrict__ out) {
  const int i = blockIdx.x, n = p.n;
  const size_t n3 = (size_t)n * n * n;
  const cpx<T> *u = (const cpx<T> *)p.u + (size_t)i * n3;
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (size_t t = threadIdx.x; t < n3; t += blockDim.x) {
    const int x = (int)(t % n), y = (int)((t / n) % n), z = (int)(t / ((size_t)n * n));
    const double w = (double)u[t].x * u[t].x + (double)u[t].y * u[t].y;
    double sx, cx, sy, cy, sz, cz;
    sincospi(2.0 * x / n, &sx, &cx);
    sincospi(2.0 * y / n, &sy, &cy);
    sincospi(2.0 * z / n, &sz, &cz);
    acc[0] += w * cx; acc[1] += w * sx; acc[2] += w * cy; acc[3] += w * sy; acc[4] += w * cz; acc[5] += w * sz;
  }
  __shared__ double red[6][256];
  for (int q = 0; q < 6; ++q) red[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int q = 0; q < 6; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < 6; ++q) out[(size_t)i * 6 + q] = red[q][0] / (double)n3;
}

// Per ordered pair (block (i, j), j >= i): S_ij = (1/N) sum_t |u_i(t)|^2 |u_j(t)|^2, the
// overlap of the two orbital densities; S[i][j] = S[j][i].
template <typename T> __global__ void k_pair_overlap(Plan p, double *__restrict__ S) {
  const int i = blockIdx.y, j = blockIdx.x;
  if (j < i) return;
  const size_t n3 = (size_t)p.n * p.n * p.n;
  const cpx<T> *ui = (const cpx<T> *)p.u + (size_t)i * n3, *uj = (const cpx<T> *)p.u + (size_t)j * n3;
  double acc = 0;
  for (size_t t = threadIdx.x; t < n3; t += blockDim.x) {
    const double a = (double)ui[t].x * ui[t].x + (double)ui[t].y * ui[t].y;
    const double b = (double)uj[t].x * uj[t].x + (double)uj[t].y * uj[t].y;
    acc += a * b;
  }
  __shared__ double red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    S[(size_t)i * p.n_occ + j] = red[0] / (double)n3;
    S[(size_t)j * p.n_occ + i] = red[0] / (double)n3;
  }
}

// ---------------------------------------------------------------- k-point sampling
// Sec. II C-D.  Occupied orbitals are composite indices I = k_I n_o + i over the mesh; every
// u_I on the grid is the cell-periodic part of phi_{i k}.  The outer loop runs over the
// supercell momentum transfers Q' = g' + kappa'/n (supercell Miller index M = n g' + kappa',
// kappa' in [0, n)), each primary Q' with its partner -Q' as slots s and s + np.  The
// transformed state of column (kt, s, j) is w = P_v^{kt} e^{-iQ'r} |j kj>: it has crystal
// momentum kt = kj - kappa'_s (mod n), and its periodic part has the coefficients of u_j
// shifted by g'_s + t, t = [kappa_j < kappa'_s] per axis.  A co-density of item (I, column)
// at FFT index g carries the transfer Q = g + (kt - k_I)/n; its Coulomb kernel comes from
// the table of that class, v_cls[(kt - kappa_I) + n - 1][g] = 4 pi/|Q|^2 inside the
// auxiliary sphere and 0 outside.

__device__ __forceinline__ int kp_mod(int a, int n) { const int r = a % n; return r < 0 ? r + n : r; }
__device__ __forceinline__ int kp_index(const Plan &p, int k0, int k1, int k2) {
  return (k0 * p.mesh[1] + k1) * p.mesh[2] + k2;
}
__device__ __forceinline__ void kp_kappa(const Plan &p, int k, int *kap) {
  kap[2] = k % p.mesh[2];
  kap[1] = (k / p.mesh[2]) % p.mesh[1];
  kap[0] = k / (p.mesh[1] * p.mesh[2]);
}
// supercell Miller index of slot s of the slab (primary Q' first, then their negatives)
__device__ __forceinline__ void kp_slot(const Plan &p, int gp0, int np, int s, int *M) {
  const int *m = p.prim_m + 3 * (size_t)(gp0 + (s < np ? s : s - np));
  const int sg = s < np ? 1 : -1;
  M[0] = sg * m[0]; M[1] = sg * m[1]; M[2] = sg * m[2];
}
// class index of an integer shift delta (each component in (-n, n))
__device__ __forceinline__ int kp_class(const Plan &p, const int *d) {
  return ((d[0] + p.mesh[0] - 1) * (2 * p.mesh[1] - 1) + (d[1] + p.mesh[1] - 1)) * (2 * p.mesh[2] - 1) +
         (d[2] + p.mesh[2] - 1);
}
// position in the auxiliary set of the integer vector g, or -1
__device__ __forceinline__ int kp_lut(const Plan &p, int g0, int g1, int g2) {
  const int n = p.n;
  if (2 * abs(g0) >= n || 2 * abs(g1) >= n || 2 * abs(g2) >= n) return -1;
  return p.lut[((size_t)wrapn(g2, n) * n + wrapn(g1, n)) * n + wrapn(g0, n)];
}

// scale factors per k: virtual a of k at [k][n_orb] offset n_o + a, occupied j at [k][j]
template <typename T>
__global__ void k_dscale_k(Plan p, const double *__restrict__ eps, double mu, double tau, T *__restrict__ d) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (a >= p.n_orb) return;
  const double x = (eps[(size_t)k * p.n_orb + a] - mu) * tau;
  d[(size_t)k * p.n_orb + a] = (T)exp(a < p.no_k ? x : -x);
}

// S^T row of column c = (kt nslots + s) n_o + j: the scaled, shifted coefficients of u_{j kj}
template <typename T>
__global__ void k_gather_k(Plan p, int gp0, int np, cpx<T> *__restrict__ st) {
  const int c = blockIdx.y;
  const int no = p.no_k, nslots = 2 * np;
  const int j = c % no, s = (c / no) % nslots, kt = c / (no * nslots);
  int M[3], kt3[3], kj3[3], sh[3];
  kp_slot(p, gp0, np, s, M);
  kp_kappa(p, kt, kt3);
  for (int a = 0; a < 3; ++a) {
    const int ks = kp_mod(M[a], p.mesh[a]);
    kj3[a] = kp_mod(kt3[a] + ks, p.mesh[a]);
    sh[a] = (M[a] - ks) / p.mesh[a] + (kj3[a] < ks ? 1 : 0);
  }
  const int kj = kp_index(p, kj3[0], kj3[1], kj3[2]);
  const T dj = ((const T *)p.dscale)[(size_t)kj * p.n_orb + j];
  const int n = p.n;
  const cpx<T> *cg = (const cpx<T> *)p.cgrid + (size_t)(kj * no + j) * n * n * n;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < p.n_pw; q += gridDim.x * blockDim.x) {
    const int wx = wrapn(p.pw_m[3 * q] + sh[0], n), wy = wrapn(p.pw_m[3 * q + 1] + sh[1], n),
              wz = wrapn(p.pw_m[3 * q + 2] + sh[2], n);
    st[(size_t)c * p.n_pw + q] = cscale(cg[((size_t)wz * n + wy) * n + wx], dj);
  }
}

// Exchange per (primary slot, I, J): item A = (I, w_J^{Q'}), item B = (J, w_I^{-Q'});
// X_IJ = sum_Q v(Q) M_A(Q) M_B(-Q), the partner of A's index g_A at B's index -g_A + Delta.
// Diagonal blocks also store M_II at its canonical index g + [kappa_I < kappa_slot], where
// every item of a slot has Q = g_c - kappa_slot / n (the direct term pairs g_c with -g_c + e).
template <typename T, int N>
__global__ void __launch_bounds__(256) k_zcol_k(Plan p, int gp0, int np, const cpx<T> *__restrict__ tbuf,
                                                cpx<T> *__restrict__ mdiag, double2 *__restrict__ sx) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T> *MA = reinterpret_cast<cpx<T> *>(smem_raw);
  const int NO = p.n_occ, no = p.no_k, nslots = 2 * np;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int gpl = blockIdx.x / (NO * NO);
  const int r = blockIdx.x % (NO * NO);
  const int I = r / NO, J = r % NO;
  const int i = I % no, j = J % no, ki = I / no, kj = J / no;
  int M[3], kI[3], kJ[3], kA[3], kB[3], ktA[3], ktB[3], dA[3], del[3], cA[3], cB[3];
  kp_slot(p, gp0, np, gpl, M);
  kp_kappa(p, ki, kI);
  kp_kappa(p, kj, kJ);
  for (int a = 0; a < 3; ++a) {
    const int n = p.mesh[a];
    kA[a] = kp_mod(M[a], n);
    kB[a] = kp_mod(-M[a], n);
    ktA[a] = kp_mod(kJ[a] - kA[a], n);
    ktB[a] = kp_mod(kI[a] - kB[a], n);
    dA[a] = ktA[a] - kI[a];
    del[a] = (kA[a] != 0 ? 1 : 0) - (kJ[a] < kA[a] ? 1 : 0) - (kI[a] < kB[a] ? 1 : 0);
    cA[a] = kI[a] < kA[a] ? 1 : 0;
    cB[a] = kI[a] < kB[a] ? 1 : 0;
  }
  const size_t colA = ((size_t)kp_index(p, ktA[0], ktA[1], ktA[2]) * nslots + gpl) * no + j;
  const size_t colB = ((size_t)kp_index(p, ktB[0], ktB[1], ktB[2]) * nslots + gpl + np) * no + i;
  const size_t itemA = colA * NO + I, itemB = colB * NO + J;
  const bool diag = (I == J);
  const T *vA = vtab_k<T>(p) + (size_t)kp_class(p, dA) * p.n_aux;
  const int nd = p.n_daux;
  for (int d = tid; d < nd; d += nth) {
    const int4 c = p.daux[d];
    const int off = p.daux_off[d];
    const cpx<T> *src = tbuf + itemA * N * nd + d;
    cpx<T> a[N];
#pragma unroll
    for (int k = 0; k < N; ++k) a[k] = src[(size_t)k * nd];
    LineFFT<T, N, -1>::run(a);
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const int m = freq_of<N>(k);
      if (m >= c.z && m <= c.w) {
        const int g = off + m - c.z;
        MA[g] = a[k];
        if (diag) {
          const int q = kp_lut(p, c.x + cA[0], c.y + cA[1], m + cA[2]);
          if (q >= 0) mdiag[((size_t)gpl * p.n_aux + q) * NO + I] = a[k];
        }
      }
    }
  }
  __syncthreads();
  T accx = T(0), accy = T(0);
  for (int d = tid; d < nd; d += nth) {
    const int4 c = p.daux[d];
    const int off = p.daux_off[d];
    const cpx<T> *src = tbuf + itemB * N * nd + d;
    cpx<T> a[N];
#pragma unroll
    for (int k = 0; k < N; ++k) a[k] = src[(size_t)k * nd];
    LineFFT<T, N, -1>::run(a);
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const int m = freq_of<N>(k);
      if (m >= c.z && m <= c.w) {
        if (diag) {
          const int q = kp_lut(p, c.x + cB[0], c.y + cB[1], m + cB[2]);
          if (q >= 0) mdiag[((size_t)(gpl + np) * p.n_aux + q) * NO + I] = a[k];
        }
        const int qa = kp_lut(p, -c.x + del[0], -c.y + del[1], -m + del[2]);
        if (qa >= 0) {
          const T v = vA[qa];
          const cpx<T> prod = cmul(MA[qa], a[k]);
          accx += v * prod.x;
          accy += v * prod.y;
        }
      }
    }
  }
  block_reduce_store<T>((double)accx, (double)accy, sx + ((size_t)gpl * NO + I) * NO + J, nullptr);
}

// Direct term per (primary slot, I): Y_IJ = sum_{g_c} v(g_c - kappa'/n) M_II(g_c; Q') M_JJ(-g_c + e; -Q'),
// e = [kappa' != 0] per axis, from the canonically stored diagonal co-densities
template <typename T>
__global__ void k_direct_k(Plan p, int np, int gp0, const cpx<T> *__restrict__ mdiag, double2 *__restrict__ yd) {
  const int gpl = blockIdx.x, I = blockIdx.y;
  const int NO = p.n_occ;
  int M[3], e[3], dd[3];
  kp_slot(p, gp0, np, gpl, M);
  for (int a = 0; a < 3; ++a) {
    const int ks = kp_mod(M[a], p.mesh[a]);
    e[a] = ks != 0 ? 1 : 0;
    dd[a] = -ks;
  }
  const T *v = vtab_k<T>(p) + (size_t)kp_class(p, dd) * p.n_aux;
  const cpx<T> *MA = mdiag + (size_t)gpl * p.n_aux * NO;
  const cpx<T> *MB = mdiag + (size_t)(gpl + np) * p.n_aux * NO;
  for (int J = threadIdx.x; J < NO; J += blockDim.x) {
    double ax = 0, ay = 0;
    T cx = T(0), cy = T(0);
    int cnt = 0;
    for (int g = 0; g < p.n_aux; ++g) {
      const T vg = v[g];
      if (vg == T(0)) continue;
      const int qb = kp_lut(p, e[0] - p.aux_m[3 * g], e[1] - p.aux_m[3 * g + 1], e[2] - p.aux_m[3 * g + 2]);
      if (qb < 0) continue;
      const cpx<T> prod = cmul(MA[(size_t)g * NO + I], MB[(size_t)qb * NO + J]);
      cx += vg * prod.x;
      cy += vg * prod.y;
      if ((++cnt & 31) == 0) { ax += (double)cx; ay += (double)cy; cx = cy = T(0); }
    }
    ax += (double)cx; ay += (double)cy;
    yd[((size_t)gpl * NO + I) * NO + J] = make_double2(ax, ay);
  }
}

// e^x_IJ += coef v(Q') (X_IJ + X_JI),  e^d_IJ += -2 coef v(Q') (Y_IJ + Y_JI)
static __global__ void k_accum_k(Plan p, int gp0, int np, double coef, const double2 *__restrict__ sx,
                                 const double2 *__restrict__ yd) {
  const int no = p.n_occ;
  const int ij = blockIdx.x * blockDim.x + threadIdx.x;
  if (ij >= no * no) return;
  const int i = ij / no, j = ij % no;
  double ex = 0, exi = 0, ed = 0, edi = 0;
  for (int gpl = 0; gpl < np; ++gpl) {
    const double vv = coef * p.vprim[gp0 + gpl];
    const double2 a = sx[((size_t)gpl * no + i) * no + j], b = sx[((size_t)gpl * no + j) * no + i];
    const double2 c = yd[((size_t)gpl * no + i) * no + j], d = yd[((size_t)gpl * no + j) * no + i];
    ex += vv * (a.x + b.x);
    exi += vv * (a.y + b.y);
    ed += -2.0 * vv * (c.x + d.x);
    edi += -2.0 * vv * (c.y + d.y);
  }
  p.ex[ij] += ex;
  p.exi[ij] += exi;
  p.ed[ij] += ed;
  p.edi[ij] += edi;
}

// ---------------------------------------------------------------- accumulation (FP64)
//   e^x_ij += coef v(G') (X_ij + X_ji),   e^d_ij += -2 coef v(G') (Y_ij + Y_ji)
// coef = w_k / (Omega^2 N_FFT^2); the sum over the slab runs in a fixed order.
static __global__ void k_accum(Plan p, int gp0, int np, double coef, const double2 *__restrict__ sx,
                        const double2 *__restrict__ yd) {
  const int no = p.n_occ;
  const int ij = blockIdx.x * blockDim.x + threadIdx.x;
  if (ij >= no * no) return;
  const int i = ij / no, j = ij % no;
  double ex = 0, exi = 0, ed = 0, edi = 0;
  for (int gpl = 0; gpl < np; ++gpl) {
    const double vv = coef * p.v_aux64[p.prim[gp0 + gpl]];
    const double2 a = sx[((size_t)gpl * no + i) * no + j], b = sx[((size_t)gpl * no + j) * no + i];
    const double2 c = yd[((size_t)gpl * no + i) * no + j], d = yd[((size_t)gpl * no + j) * no + i];
    ex += vv * (a.x + b.x);
    exi += vv * (a.y + b.y);
    ed += -2.0 * vv * (c.x + d.x);
    edi += -2.0 * vv * (c.y + d.y);
  }
  p.ex[ij] += ex;
  p.exi[ij] += exi;
  p.ed[ij] += ed;
  p.edi[ij] += edi;
}

// level n >= 2 of the extrapolation (blockIdx.y = n - 2): only G' in A_n contribute
static __global__ void k_accum_lev(Plan p, int gp0, int np, double coef) {
  const int no = p.n_occ;
  const int ij = blockIdx.x * blockDim.x + threadIdx.x;
  if (ij >= no * no) return;
  const int i = ij / no, j = ij % no;
  {
    const int n = blockIdx.y + 1;
    const double2 *sx = p.sxl + (size_t)n * p.lev_stride, *yd = p.ydl + (size_t)n * p.lev_stride;
    double ex = 0, ed = 0;
    for (int gpl = 0; gpl < np; ++gpl) {
      const int g = p.prim[gp0 + gpl];
      if (p.aux_lev[g] < n + 1) continue;
      const double vv = coef * p.v_aux64[g];
      const double2 a = sx[((size_t)gpl * no + i) * no + j], b = sx[((size_t)gpl * no + j) * no + i];
      const double2 c = yd[((size_t)gpl * no + i) * no + j], d = yd[((size_t)gpl * no + j) * no + i];
      ex += vv * (a.x + b.x);
      ed += -2.0 * vv * (c.x + d.x);
    }
    p.exl[(size_t)n * no * no + ij] += ex;
    p.edl[(size_t)n * no * no + ij] += ed;
  }
}

// ---------------------------------------------------------------- opposite-spin direct term
// Spin-unrestricted form: the direct energy couples M^a_ii of the alpha channel with M^b_jj
// of the beta channel at the same tau and G' (Eq. MP2direct with s != s').  Per primary G'
// and pair (i alpha, j beta): y = Re[Y(G') + Y(-G')], Y(G') = sum_G v(G) M^a_ii(G;G')
// M^b_jj(-G;-G').  Real orbitals: Y(-G') = conj(Y(G')) and M(-G;-G') = conj(M(G;G')).
template <typename T>
__global__ void k_direct_cross(Plan pa, Plan pb, int np, const cpx<T> *__restrict__ ma,
                               const cpx<T> *__restrict__ mb, double *__restrict__ y) {
  const int gpl = blockIdx.x, i = blockIdx.y;
  const int na = pa.n_occ, nb = pb.n_occ, naux = pa.n_aux;
  const T *v = vtab<T>(pa);
  for (int j = threadIdx.x; j < nb; j += blockDim.x) {
    double acc = 0.0;
    for (int pass = 0; pass < (pa.real_orb ? 1 : 2); ++pass) {
      // general orbitals: pass 0 pairs slot G' of alpha with slot -G' of beta, pass 1 the reverse
      const int sa = pass == 0 ? gpl : gpl + np, sb = pa.real_orb ? gpl : (pass == 0 ? gpl + np : gpl);
      const cpx<T> *A = ma + (size_t)sa * naux * na;
      const cpx<T> *B = mb + (size_t)sb * naux * nb;
      double ax = 0.0;
      T cx = T(0);
      for (int g = 0; g < naux; ++g) {
        const cpx<T> x = A[(size_t)g * na + i];
        cpx<T> prod;
        if (pa.real_orb) prod = cmulconj(x, B[(size_t)g * nb + j]);
        else prod = cmul(x, B[(size_t)pa.aux_neg[g] * nb + j]);
        cx += v[g] * prod.x;
        if ((g & 31) == 31) { ax += (double)cx; cx = T(0); }
      }
      ax += (double)cx;
      acc += pa.real_orb ? 2.0 * ax : ax;
    }
    y[((size_t)gpl * na + i) * nb + j] = acc;
  }
}

// acc[i][j] += -coef v(G') y over the slab's primary G', fixed order
static __global__ void k_accum_cross(Plan pa, int nb, int gp0, int np, double coef, const double *__restrict__ y,
                                     double *__restrict__ acc) {
  const int na = pa.n_occ;
  const int ij = blockIdx.x * blockDim.x + threadIdx.x;
  if (ij >= na * nb) return;
  double s = 0.0;
  for (int gpl = 0; gpl < np; ++gpl) s += -coef * pa.v_aux64[pa.prim[gp0 + gpl]] * y[(size_t)gpl * na * nb + ij];
  acc[ij] += s;
}

// out[0] = sum of n values, fixed order; one block of 256 threads
static __global__ void k_sum(int n, const double *__restrict__ x, double *__restrict__ out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) s += x[k];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0];
}

static __global__ void k_zero_acc(Plan p) {
  const int no2 = p.n_occ * p.n_occ;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < no2; k += gridDim.x * blockDim.x) {
    p.ex[k] = 0; p.exi[k] = 0; p.ed[k] = 0; p.edi[k] = 0;
  }
  if (p.n_lev > 1)
    for (size_t k = blockIdx.x * blockDim.x + threadIdx.x; k < (size_t)p.n_lev * no2; k += gridDim.x * blockDim.x) {
      p.exl[k] = 0; p.edl[k] = 0;
    }
}

// fixed-order level sums: esum_lev[2n] = E_d over A_{n+1}, esum_lev[2n+1] = E_x; one block of 256
static __global__ void k_finish_lev(Plan p) {
  __shared__ double red[2][256];
  const int no2 = p.n_occ * p.n_occ;
  for (int n = 0; n < p.n_lev; ++n) {
    const double *ed = n == 0 ? p.ed : p.edl + (size_t)n * no2;
    const double *ex = n == 0 ? p.ex : p.exl + (size_t)n * no2;
    double sd = 0, sx = 0;
    for (int k = threadIdx.x; k < no2; k += blockDim.x) { sd += ed[k]; sx += ex[k]; }
    red[0][threadIdx.x] = sd;
    red[1][threadIdx.x] = sx;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) {
        red[0][threadIdx.x] += red[0][threadIdx.x + w];
        red[1][threadIdx.x] += red[1][threadIdx.x + w];
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) { p.esum_lev[2 * n] = red[0][0]; p.esum_lev[2 * n + 1] = red[1][0]; }
    __syncthreads();
  }
}

// fixed-order final sums: esum = {E_d, E_x, Im E_d, Im E_x}; one block of 256 threads
static __global__ void k_finish(Plan p) {
  __shared__ double red[4][256];
  const int no2 = p.n_occ * p.n_occ;
  double s[4] = {0, 0, 0, 0};
  for (int k = threadIdx.x; k < no2; k += blockDim.x) {
    s[0] += p.ed[k]; s[1] += p.ex[k]; s[2] += p.edi[k]; s[3] += p.exi[k];
  }
  for (int q = 0; q < 4; ++q) red[q][threadIdx.x] = s[q];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int q = 0; q < 4; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < 4; ++q) p.esum[q] = red[q][0];
}

}  // namespace ltmp2

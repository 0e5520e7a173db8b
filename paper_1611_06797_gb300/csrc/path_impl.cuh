// Launchers of the hot path for one real type T.  Included once per precision by
// kernels_f64.cu / kernels_f32.cu, which explicitly instantiate Path<T>.
#pragma once
#include <mutex>
#include <type_traits>

#include "kernels.cuh"

namespace ltmp2 {

#define LTMP2_FOR_EACH_N(X) X(8) X(10) X(12) X(16) X(18) X(20) X(24) X(25) X(27) X(30) X(32) X(36) X(40)

// Plane kernels: 0 = k_planes (full-plane passes), 1 = k_planes2 (compacted passes),
// 2 = k_planes3 (product in registers, compact intermediate), 3 = k_planes4 (as 2, each
// warp on its own occupied planes without block barriers).
// ib = occupied planes per block (kernel 3: per warp step); 0 picks the default of each kernel.
template <typename T> static int plane_ib_default(const Plan &p, int kernel) {
  const int n = p.n;
  const size_t plane = (size_t)n * (n + 1) * sizeof(cpx<T>);
  const int nxa = p.mxhi_aux - p.mxlo_aux + 1;
  int ib;
  if (kernel == 3) {
    // as many planes per warp step as fill the 32 lanes of the x pass, at least 2 (two
    // planes per warp step were fastest in FP32 on the 24^3 and 36^3 workloads: 20.6 and
    // 790 ms per plane pass against 23.5 and 905 with one), within ~100 KB
    ib = (32 + n - 1) / n;
    if (ib < 2) ib = 2;
    const size_t per = (size_t)kPlaneWarps * plane_stride(n, nxa) * sizeof(cpx<T>);
    while (ib > 1 && plane + ib * per > 100 * 1024) --ib;
  } else if (kernel == 0) {
    ib = (int)((96 * 1024) / plane) - 1;   // about 96 KB of shared memory
    if (ib > 8) ib = 8;
  } else if (kernel == 2) {
    // four planes per block: small blocks, many resident per SM (best on the 24^3 workload
    // in both precisions among 2..16)
    const size_t per = (size_t)n * nxa * sizeof(cpx<T>);
    ib = (int)((100 * 1024 - plane - sizeof(int) * p.n_daux - 64) / per);
    if (ib > 4) ib = 4;
  } else {
    const size_t per = plane + (size_t)p.n_daux * sizeof(cpx<T>);
    ib = (int)((100 * 1024 - plane - 3 * sizeof(int) * (n + 1) - 64) / per);
    if (ib > 384 / n) ib = 384 / n;
  }
  if (ib > p.n_occ) ib = p.n_occ;
  if (ib < 1) ib = 1;
  return ib;
}

template <typename T> static size_t plane_smem(const Plan &p, int kernel, int ib) {
  const int n = p.n;
  const size_t plane = (size_t)n * (n + 1) * sizeof(cpx<T>);
  const int nxa = p.mxhi_aux - p.mxlo_aux + 1;
  if (kernel == 0) return plane * (1 + ib);
  const size_t q = (size_t)plane_stride(n, nxa);
  if (kernel == 2) return plane + (size_t)ib * q * sizeof(cpx<T>) + sizeof(int) * p.n_daux;
  if (kernel == 3) return plane + (size_t)kPlaneWarps * ib * q * sizeof(cpx<T>) + sizeof(int) * p.n_daux;
  return plane * (1 + ib) + (size_t)ib * p.n_daux * sizeof(cpx<T>) + 3 * sizeof(int) * nxa;
}

// launch the plane kernel for the ncols columns of the current slab (z1 -> tbuf)
template <typename T> static cudaError_t launch_planes(const Plan &p, int ncols, int kernel, int ib, cudaStream_t st) {
  if (ib <= 0) ib = plane_ib_default<T>(p, kernel);
  const size_t smem = plane_smem<T>(p, kernel, ib);
  int threads = kernel == 3 ? 32 * kPlaneWarps : ib * p.n;
  if (threads < 64) threads = 64;
  if (threads > 1024 || smem > 200 * 1024) return cudaErrorInvalidValue;
  switch (p.n) {
#define LTMP2_CASE(NN)                                                                                     \
  case NN:                                                                                                 \
    if (kernel == 0)                                                                                       \
      k_planes<T, NN><<<dim3(NN, ncols), threads, smem, st>>>(p, ib, (const cpx<T> *)p.z1, (cpx<T> *)p.tbuf);  \
    else if (kernel == 1)                                                                                  \
      k_planes2<T, NN><<<dim3(NN, ncols), threads, smem, st>>>(p, ib, (const cpx<T> *)p.z1, (cpx<T> *)p.tbuf); \
    else if (kernel == 2)                                                                                  \
      k_planes3<T, NN><<<dim3(NN, ncols), threads, smem, st>>>(p, ib, (const cpx<T> *)p.z1, (cpx<T> *)p.tbuf); \
    else                                                                                                   \
      k_planes4<T, NN><<<dim3(NN, ncols), threads, smem, st>>>(p, ib, (const cpx<T> *)p.z1, (cpx<T> *)p.tbuf); \
    break;
    LTMP2_FOR_EACH_N(LTMP2_CASE)
#undef LTMP2_CASE
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T> bool Path<T>::plane_feasible(const Plan &p, int kernel, int ib) {
  if (kernel < 0 || kernel > 3 || ib < 0) return false;
  if (ib == 0) ib = plane_ib_default<T>(p, kernel);
  const int threads = kernel == 3 ? 32 * kPlaneWarps : ib * p.n;
  return threads <= 1024 && plane_smem<T>(p, kernel, ib) <= 200 * 1024;
}

template <typename T>
cudaError_t Path<T>::plane_pass(const Plan &p, int ncols, int kernel, int ib, cudaStream_t st) {
  return launch_planes<T>(p, ncols, kernel, ib, st);
}

struct ScopedStage {
  StageTimer *tm;
  int st;
  ScopedStage(StageTimer *t, int s) : tm(t), st(s) { if (tm) tm->begin(st); }
  ~ScopedStage() { if (tm) tm->end(st); }
};

template <typename T> cudaError_t Path<T>::init_device() {
  // once per device and process; contexts set up from several host threads serialise here
  static bool done[64] = {false};
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 64 && done[dev]) return cudaSuccess;
  e = upload_twiddles();
  if (e != cudaSuccess) return e;
  // dynamic shared memory limits of the FFT kernels
#define LTMP2_SET_SMEM(NN)                                                                          \
  e = cudaFuncSetAttribute(k_planes<T, NN>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024); \
  if (e != cudaSuccess) return e;                                                                   \
  e = cudaFuncSetAttribute(k_zcol<T, NN, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024); \
  if (e != cudaSuccess) return e;                                                                   \
  e = cudaFuncSetAttribute(k_zcol<T, NN, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024); \
  if (e != cudaSuccess) return e;                                                                   \
  e = cudaFuncSetAttribute(k_planes2<T, NN>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024); \
  if (e != cudaSuccess) return e;                                                                   \
  e = cudaFuncSetAttribute(k_planes3<T, NN>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024); \
  if (e != cudaSuccess) return e;                                                                   \
  e = cudaFuncSetAttribute(k_planes4<T, NN>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024); \
  if (e != cudaSuccess) return e;                                                                   \
  e = cudaFuncSetAttribute(k_zcol_k<T, NN>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024); \
  if (e != cudaSuccess) return e;
  LTMP2_FOR_EACH_N(LTMP2_SET_SMEM)
#undef LTMP2_SET_SMEM
  if (dev < 64) done[dev] = true;
  return cudaSuccess;
}

template <typename T>
cudaError_t Path<T>::setup_occupied(const Plan &p, const void *c_occ_dev, cudaStream_t st) {
  const int n = p.n;
  const size_t n3 = (size_t)n * n * n;
  cudaError_t e = cudaMemsetAsync(p.cgrid, 0, sizeof(cpx<T>) * n3 * p.n_occ, st);
  if (e != cudaSuccess) return e;
  const cpx<T> *c = (const cpx<T> *)c_occ_dev;
  k_scatter_grid<T><<<dim3((p.n_pw + 255) / 256, p.n_occ), 256, 0, st>>>(p, p.n_occ, c, (cpx<T> *)p.cgrid);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // z1 scratch: reuse p.z1 when it is large enough (max_cols >= n_occ always holds)
  cpx<T> *z1 = (cpx<T> *)p.z1;
  const size_t smem = (size_t)n * (n + 1) * sizeof(cpx<T>);
  switch (n) {
#define LTMP2_CASE(NN)                                                                            \
  case NN:                                                                                        \
    k_w_zinv<T, NN><<<dim3((p.n_dorb + 127) / 128, p.n_occ), 128, 0, st>>>(p, p.n_pw, c, z1);     \
    k_planes_store<T, NN><<<dim3(NN, p.n_occ), 128, smem, st>>>(p, z1, (cpx<T> *)p.u, (cpx<T> *)p.ut,       \
                                                                (T *)p.utr);                                  \
    break;
    LTMP2_FOR_EACH_N(LTMP2_CASE)
#undef LTMP2_CASE
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T> cudaError_t Path<T>::overlap_setup(const Plan &p, cudaStream_t st) {
  // r_a transposed into pt ([n_pw][n_v]); pt is free on this route (no Green's function)
  k_transpose<T><<<dim3((p.n_pw + 31) / 32, (p.n_v + 31) / 32), dim3(32, 8), 0, st>>>(p.n_v, p.n_pw, (const T *)p.cv,
                                                                                      (T *)p.pt);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  for (int gp0 = 0; gp0 < p.n_prim; gp0 += p.max_prim) {
    const int np = p.n_prim - gp0 < p.max_prim ? p.n_prim - gp0 : p.max_prim;
    const int ncols = np * p.n_occ;
    // rho^T[(G', j)][a] = sum_q (U e^{-iG'r} phi_j)[q] r_a[q]: U is unitary and r_a = U phi_a
    // is real, so this is <a| e^{-iG'r} |j> (Eq. SCHovrlp), step (i) of Sec. III A
    k_gather_s_real<T><<<dim3((p.n_pw + 255) / 256, ncols), 256, 0, st>>>(p, gp0, np, (cpx<T> *)p.st, true);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    dim3 grid((p.n_v + 63) / 64, (ncols + 63) / 64);
    k_rgemm<T, cpx<T>, true><<<grid, 256, 0, st>>>(ncols, p.n_v, p.n_pw, (const cpx<T> *)p.st, p.n_pw,
                                                    (const T *)p.pt, p.n_v, nullptr,
                                                    (cpx<T> *)p.rt + (size_t)gp0 * p.n_occ * p.n_v, p.n_v);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <typename T>
cudaError_t Path<T>::green(const Plan &p, double tau, cudaStream_t st, StageTimer *tm) {
  ScopedStage s(tm, kStageGreen);
  k_dscale<T><<<(p.n_orb + 255) / 256, 256, 0, st>>>(p.n_orb, p.n_occ, p.eps, p.mu, tau, (T *)p.dscale);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // no Green's function on the paper's route, nor when W goes through the virtual space
  if (p.route == 1 || p.w_virtual) return cudaSuccess;
  if constexpr (std::is_same<T, float>::value) {
    if (p.tc && p.tc->green_on()) {
      // precision form, real basis: P_r on the tensor cores (3xTF32), then the split of P_r
      // into the transformed-state GEMM's operands
      if ((e = tc_green(*p.tc, (const float *)p.dscale + p.n_occ, p.pt, st)) != cudaSuccess) return e;
      return tc_pack_b(*p.tc, p.pt, st);
    }
  }
  const int M = p.n_pw, N = p.n_pw, K = p.nv_tau > 0 ? p.nv_tau : p.n_v;
  dim3 grid((N + 63) / 64, (M + 63) / 64);
  if constexpr (std::is_same<T, double>::value) {
    if (p.oz && p.rvt && oz_green_fits(*p.oz)) {
      // FP64 on the tensor cores: P_r = (R_v'^T D') R_v', then its slices for the W product
      if ((e = oz_green(*p.oz, (const double *)p.rvt, (const double *)p.dscale + p.n_occ, K, (double *)p.pt, st)) !=
          cudaSuccess)
        return e;
      return oz_split_b(*p.oz, (const double *)p.pt, st);
    }
  }
  if (p.real_basis) {
    // P_r[q][p] = sum_a r_a(q) e^{-(e_a-mu)tau} r_a(p), r_a the real coordinates of a
    k_rgemm<T, T, false><<<grid, 256, 0, st>>>(M, N, K, (const T *)p.cv, p.n_pw, (const T *)p.cv, p.n_pw,
                                               (const T *)p.dscale + p.n_occ, (T *)p.pt, p.n_pw);
  } else {
    // P^T[q][p] = sum_a conj(c_a(q)) e^{-(e_a-mu)tau} c_a(p)
    k_cgemm<T, false, true><<<grid, 256, 0, st>>>(M, N, K, (const cpx<T> *)p.cv, p.n_pw,
                                                  (const cpx<T> *)p.cv, p.n_pw,
                                                  (const T *)p.dscale + p.n_occ, (cpx<T> *)p.pt, p.n_pw);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if constexpr (std::is_same<T, float>::value) {
    if (p.tc) return tc_pack_b(*p.tc, p.pt, st);  // split P into TF32 hi/lo operands
  } else {
    if (p.oz) return oz_split_b(*p.oz, (const double *)p.pt, st);   // exact integer slices of P_r
  }
  return cudaSuccess;
}

template <typename T>
cudaError_t Path<T>::slab_pre(const Plan &p, int gp0, int np, cudaStream_t st, StageTimer *tm) {
  const int n = p.n, no = p.n_occ;
  const int nslots = np * p.slots_per_prim();
  const int ncols = nslots * no;
  cudaError_t e;
  if (p.route != 1) {
    ScopedStage s(tm, kStageGatherZ);
    if (p.real_basis)
      k_gather_s_real<T><<<dim3((p.n_pw + 255) / 256, ncols), 256, 0, st>>>(p, gp0, np, (cpx<T> *)p.st);
    else
      k_gather_s<T><<<dim3((p.n_pw + 255) / 256, ncols), 256, 0, st>>>(p, gp0, np, (cpx<T> *)p.st);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  {
    ScopedStage s(tm, kStageWGemm);
    bool done = false;
    if (p.route == 1) {
      // W (real-basis coordinates, before the e^{(e_j-mu)tau} row factor) =
      // sum_a rho^T[(G', j)][a] e^{-(e_a-mu)tau} r_a: step (iii) with the stored overlap densities
      dim3 grid((p.n_pw + 63) / 64, (ncols + 63) / 64);
      const int nv = p.nv_tau > 0 ? p.nv_tau : p.n_v;
      k_rgemm<T, cpx<T>, true><<<grid, 256, 0, st>>>(ncols, p.n_pw, nv,
                                                      (const cpx<T> *)p.rt + (size_t)gp0 * no * p.n_v, p.n_v,
                                                      (const T *)p.cv, p.n_pw, (const T *)p.dscale + p.n_occ,
                                                      (cpx<T> *)p.wt, p.n_pw);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      done = true;
    } else if (p.w_virtual) {
      // X^T = (U S)^T R_v'^T [ncols][nv] in the z1 buffer (free until the z transform; it
      // holds n n_dorb >= n_pw > nv values per column), then W^T = X^T D' R_v'
      if constexpr (std::is_same<T, double>::value) {
        if (p.oz) {
          if ((e = oz_virtual(*p.oz, p.st, ncols, (const double *)p.rvt, (const double *)p.dscale + p.n_occ, p.nv_tau,
                              p.z1, p.wt, st)) != cudaSuccess)
            return e;
          done = true;
        }
      }
    }
    if (p.w_virtual && !done) {
      const int nv = p.nv_tau;
      dim3 gx((nv + 63) / 64, (ncols + 63) / 64);
      k_rgemm<T, cpx<T>, true><<<gx, 256, 0, st>>>(ncols, nv, p.n_pw, (const cpx<T> *)p.st, p.n_pw,
                                                    (const T *)p.rvt, p.n_v, nullptr, (cpx<T> *)p.z1, nv);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      dim3 gw((p.n_pw + 63) / 64, (ncols + 63) / 64);
      k_rgemm<T, cpx<T>, true><<<gw, 256, 0, st>>>(ncols, p.n_pw, nv, (const cpx<T> *)p.z1, nv, (const T *)p.cv,
                                                    p.n_pw, (const T *)p.dscale + p.n_occ, (cpx<T> *)p.wt,
                                                    p.n_pw);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      done = true;
    }
    if constexpr (std::is_same<T, float>::value) {
      if (p.tc && !done) {
        if ((e = tc_wgemm(*p.tc, p.st, ncols, p.wt, st)) != cudaSuccess) return e;
        done = true;
      }
    } else {
      if (p.oz && !done) {   // FP64-accurate products on the tensor cores
        if ((e = oz_wgemm(*p.oz, p.st, ncols, p.wt, st)) != cudaSuccess) return e;
        done = true;
      }
    }
    if (!done) {
      dim3 grid((p.n_pw + 63) / 64, (ncols + 63) / 64);
      if (p.real_basis)
        k_rgemm<T, cpx<T>, true><<<grid, 256, 0, st>>>(ncols, p.n_pw, p.n_pw, (const cpx<T> *)p.st, p.n_pw,
                                                        (const T *)p.pt, p.n_pw, nullptr, (cpx<T> *)p.wt,
                                                        p.n_pw);
      else
        k_cgemm<T, true, false><<<grid, 256, 0, st>>>(ncols, p.n_pw, p.n_pw, (const cpx<T> *)p.st, p.n_pw,
                                                      (const cpx<T> *)p.pt, p.n_pw, nullptr,
                                                      (cpx<T> *)p.wt, p.n_pw);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
  }
  // real basis: W^T back to plane-wave coefficients, into the (now free) S^T buffer
  const cpx<T> *w_pw = (const cpx<T> *)p.wt;
  if (p.real_basis) {
    ScopedStage s(tm, kStageGatherZ);
    k_from_real_basis<T><<<dim3((p.n_pw + 255) / 256, ncols), 256, 0, st>>>(
        p, (const cpx<T> *)p.wt, (cpx<T> *)p.st, p.route == 1 ? (const T *)p.dscale : nullptr);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    w_pw = (const cpx<T> *)p.st;
  }
  switch (n) {
#define LTMP2_CASE(NN)                                                                                  \
  case NN: {                                                                                            \
    ScopedStage s(tm, kStageGatherZ);                                                                   \
    k_w_zinv<T, NN><<<dim3((p.n_dorb + 127) / 128, ncols), 128, 0, st>>>(p, p.n_pw, w_pw, (cpx<T> *)p.z1); \
    if ((e = cudaGetLastError()) != cudaSuccess) return e;                                              \
  } break;
    LTMP2_FOR_EACH_N(LTMP2_CASE)
#undef LTMP2_CASE
    default:
      return cudaErrorInvalidValue;
  }
  return cudaSuccess;
}

template <typename T>
cudaError_t Path<T>::slab(const Plan &p, int gp0, int np, double coef, cudaStream_t st, StageTimer *tm) {
  const int n = p.n, no = p.n_occ;
  const int nslots = np * p.slots_per_prim();
  const int ncols = nslots * no;
  cudaError_t e;
  if ((e = slab_pre(p, gp0, np, st, tm)) != cudaSuccess) return e;
  const bool lev = p.n_lev > 1;
  const size_t smem_col = (lev ? 2 : 1) * (size_t)p.n_aux * sizeof(cpx<T>);
  const int npairs = p.real_orb ? np * (no * (no + 1) / 2) : np * no * no;
  int col_threads = ((p.n_daux + 31) / 32) * 32;
  if (col_threads > 256) col_threads = 256;   // the column kernel's launch bound (FP64 N >= 36 uses ~255 registers)
  switch (n) {
#define LTMP2_CASE(NN)                                                                                  \
  case NN: {                                                                                            \
    {                                                                                                   \
      ScopedStage s(tm, kStagePlane);                                                                   \
      if ((e = launch_planes<T>(p, ncols, p.plane_kernel, p.plane_ib, st)) != cudaSuccess) return e;    \
    }                                                                                                   \
    {                                                                                                   \
      ScopedStage s(tm, kStageColumn);                                                                  \
      if (lev)                                                                                          \
        k_zcol<T, NN, true><<<npairs, col_threads, smem_col, st>>>(p, gp0, np, (const cpx<T> *)p.tbuf,  \
                                                                   (cpx<T> *)p.mdiag, p.sx);            \
      else                                                                                              \
        k_zcol<T, NN, false><<<npairs, col_threads, smem_col, st>>>(p, gp0, np, (const cpx<T> *)p.tbuf, \
                                                                    (cpx<T> *)p.mdiag, p.sx);           \
      if ((e = cudaGetLastError()) != cudaSuccess) return e;                                            \
    }                                                                                                   \
  } break;
    LTMP2_FOR_EACH_N(LTMP2_CASE)
#undef LTMP2_CASE
    default:
      return cudaErrorInvalidValue;
  }
  return slab_post(p, gp0, np, coef, st, tm);
}

template <typename T>
cudaError_t Path<T>::slab_post(const Plan &p, int gp0, int np, double coef, cudaStream_t st, StageTimer *tm) {
  const int no = p.n_occ;
  const bool lev = p.n_lev > 1;
  cudaError_t e;
  {
    ScopedStage s(tm, kStageDirect);
    int th = no < 128 ? ((no + 31) / 32) * 32 : 128;
    // FP32: the shared-memory tiled kernel (1.6x faster on the 24^3 workload); FP64 is
    // bound by the FP64 pipe either way and the one-warp-per-(G', i) kernel is 12 % faster
    bool done = false;
    if constexpr (std::is_same<T, float>::value) {
      if (!lev && p.tc && p.tc->direct_on()) {   // real orbitals: one tensor-core product per G'
        if ((e = tc_direct(*p.tc, p.mdiag, p.v_aux32, np, p.yd, st)) != cudaSuccess) return e;
        done = true;
      }
    }
    if (done) {
    } else if (lev) {
      k_direct<T, true><<<dim3(np, no), th, 0, st>>>(p, np, (const cpx<T> *)p.mdiag, p.yd);
    } else if (std::is_same<T, float>::value) {
      const int t = (no + 31) / 32;
      k_direct_tiled<T><<<dim3(np, t, t), 256, 0, st>>>(p, np, (const cpx<T> *)p.mdiag, p.yd);
    } else {
      k_direct<T, false><<<dim3(np, no), th, 0, st>>>(p, np, (const cpx<T> *)p.mdiag, p.yd);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  {
    ScopedStage s(tm, kStageAccum);
    k_accum<<<(no * no + 127) / 128, 128, 0, st>>>(p, gp0, np, coef, p.sx, p.yd);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (lev) {
      k_accum_lev<<<dim3((no * no + 31) / 32, p.n_lev - 1), 32, 0, st>>>(p, gp0, np, coef);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

template <typename T> cudaError_t Path<T>::green_k(const Plan &p, double tau, cudaStream_t st, StageTimer *tm) {
  ScopedStage s(tm, kStageGreen);
  k_dscale_k<T><<<dim3((p.n_orb + 255) / 256, p.nk), 256, 0, st>>>(p, p.eps, p.mu, tau, (T *)p.dscale);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t pw2 = (size_t)p.n_pw * p.n_pw;
  dim3 grid((p.n_pw + 63) / 64, (p.n_pw + 63) / 64);
  for (int k = 0; k < p.nk; ++k) {
    // P^T_k[q][p] = sum_a conj(c_{a k}(q)) e^{-(e_{a k}-mu)tau} c_{a k}(p)
    const cpx<T> *cv = (const cpx<T> *)p.cv + (size_t)k * p.n_v * p.n_pw;
    k_cgemm<T, false, true><<<grid, 256, 0, st>>>(p.n_pw, p.n_pw, p.n_v, cv, p.n_pw, cv, p.n_pw,
                                                  (const T *)p.dscale + (size_t)k * p.n_orb + p.no_k,
                                                  (cpx<T> *)p.pt + k * pw2, p.n_pw);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <typename T>
cudaError_t Path<T>::slab_k(const Plan &p, int gp0, int np, double coef, cudaStream_t st, StageTimer *tm) {
  const int n = p.n, NO = p.n_occ;
  const int nslots = 2 * np;
  const int ncols = nslots * NO;          // nk blocks of nslots * n_o columns, one block per kt
  const int rows_k = nslots * p.no_k;
  cudaError_t e;
  {
    ScopedStage s(tm, kStageGatherZ);
    k_gather_k<T><<<dim3((p.n_pw + 255) / 256, ncols), 256, 0, st>>>(p, gp0, np, (cpx<T> *)p.st);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  {
    ScopedStage s(tm, kStageWGemm);
    const size_t pw2 = (size_t)p.n_pw * p.n_pw;
    dim3 grid((p.n_pw + 63) / 64, (rows_k + 63) / 64);
    for (int kt = 0; kt < p.nk; ++kt) {
      const size_t row0 = (size_t)kt * rows_k * p.n_pw;
      k_cgemm<T, true, false><<<grid, 256, 0, st>>>(rows_k, p.n_pw, p.n_pw, (const cpx<T> *)p.st + row0, p.n_pw,
                                                    (const cpx<T> *)p.pt + kt * pw2, p.n_pw, nullptr,
                                                    (cpx<T> *)p.wt + row0, p.n_pw);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
  }
  const size_t smem_col = (size_t)p.n_aux * sizeof(cpx<T>);
  const int npairs = np * NO * NO;
  int col_threads = ((p.n_daux + 31) / 32) * 32;
  if (col_threads > 256) col_threads = 256;
  switch (n) {
#define LTMP2_CASE(NN)                                                                                 \
  case NN: {                                                                                           \
    {                                                                                                  \
      ScopedStage s(tm, kStageGatherZ);                                                                \
      k_w_zinv<T, NN><<<dim3((p.n_dorb + 127) / 128, ncols), 128, 0, st>>>(p, p.n_pw, (const cpx<T> *)p.wt, \
                                                                          (cpx<T> *)p.z1);              \
      if ((e = cudaGetLastError()) != cudaSuccess) return e;                                           \
    }                                                                                                  \
    {                                                                                                  \
      ScopedStage s(tm, kStagePlane);                                                                  \
      if ((e = launch_planes<T>(p, ncols, p.plane_kernel, p.plane_ib, st)) != cudaSuccess) return e;   \
    }                                                                                                  \
    {                                                                                                  \
      ScopedStage s(tm, kStageColumn);                                                                 \
      k_zcol_k<T, NN><<<npairs, col_threads, smem_col, st>>>(p, gp0, np, (const cpx<T> *)p.tbuf,       \
                                                             (cpx<T> *)p.mdiag, p.sx);                 \
      if ((e = cudaGetLastError()) != cudaSuccess) return e;                                           \
    }                                                                                                  \
  } break;
    LTMP2_FOR_EACH_N(LTMP2_CASE)
#undef LTMP2_CASE
    default:
      return cudaErrorInvalidValue;
  }
  {
    ScopedStage s(tm, kStageDirect);
    const int th = NO < 128 ? ((NO + 31) / 32) * 32 : 128;
    k_direct_k<T><<<dim3(np, NO), th, 0, st>>>(p, np, gp0, (const cpx<T> *)p.mdiag, p.yd);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  {
    ScopedStage s(tm, kStageAccum);
    k_accum_k<<<(NO * NO + 127) / 128, 128, 0, st>>>(p, gp0, np, coef, p.sx, p.yd);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// ---------------------------------------------------------------- batching form: persistent stages
// Thread blocks of kPersistThreads stay resident and take items from a device counter:
// plane items (system, column, z) and column items (system, pair) of every active system of
// the round, each run by the same body as the system's own kernel (dispatch on its grid).
template <typename T>
__global__ void __launch_bounds__(kPersistThreads) k_planes_persist(const Plan *__restrict__ plans, BatchRound r,
                                                                     int *__restrict__ counter) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_item;
  // the round's tables in shared memory: indexed by the item's system, which a kernel
  // parameter array would have to copy to local memory for
  __shared__ BatchRound sr;
  if (threadIdx.x == 0) sr = r;
  const int total = r.first[r.nsys];
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int item = s_item;
    if (item >= total) return;
    int e = 0;
    while (item >= sr.first[e + 1]) ++e;
    const Plan &p = plans[sr.sys[e]];
    const int local = item - sr.first[e];
    const int z = local % p.n, col = local / p.n;
    switch (p.n) {
#define LTMP2_CASE(NN)                                                                                        \
  case NN:                                                                                                    \
    planes3_body<T, NN>(p, sr.ib[e], z, col, (const cpx<T> *)p.z1, (cpx<T> *)p.tbuf, smem_raw);              \
    break;
      LTMP2_FOR_EACH_N(LTMP2_CASE)
#undef LTMP2_CASE
      default:
        break;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kPersistThreads) k_zcol_persist(const Plan *__restrict__ plans, BatchRound r,
                                                                   int *__restrict__ counter) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_item;
  // the round's tables in shared memory: indexed by the item's system, which a kernel
  // parameter array would have to copy to local memory for
  __shared__ BatchRound sr;
  if (threadIdx.x == 0) sr = r;
  const int total = r.first[r.nsys];
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int item = s_item;
    if (item >= total) return;
    int e = 0;
    while (item >= sr.first[e + 1]) ++e;
    const Plan &p = plans[sr.sys[e]];
    const int local = item - sr.first[e];
    switch (p.n) {
#define LTMP2_CASE(NN)                                                                                        \
  case NN:                                                                                                    \
    zcol_body<T, NN, false>(p, sr.gp0[e], sr.np[e], local, (const cpx<T> *)p.tbuf, (cpx<T> *)p.mdiag, p.sx,   \
                            smem_raw);                                                                        \
    break;
      LTMP2_FOR_EACH_N(LTMP2_CASE)
#undef LTMP2_CASE
      default:
        break;
    }
  }
}

template <typename T> size_t Path<T>::plane_smem_for(const Plan &p, int ib) { return plane_smem<T>(p, 2, ib); }

template <typename T> cudaError_t Path<T>::persist_attributes(size_t plane_smem_b, size_t col_smem_b) {
  cudaError_t e = cudaFuncSetAttribute(k_planes_persist<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)plane_smem_b);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_zcol_persist<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)col_smem_b);
}

// resident blocks of the persistent kernel: every SM filled to its occupancy
template <typename T> int Path<T>::persist_blocks(bool planes, size_t smem) {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  const cudaError_t e = planes
      ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_planes_persist<T>, kPersistThreads, smem)
      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_zcol_persist<T>, kPersistThreads, smem);
  if (e != cudaSuccess) return 0;
  return sms * (per > 0 ? per : 1);
}

template <typename T>
cudaError_t Path<T>::planes_persist(const Plan *d_plans, const BatchRound &r, int *counter, int blocks, size_t smem,
                                    cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  k_planes_persist<T><<<blocks, kPersistThreads, smem, st>>>(d_plans, r, counter);
  return cudaGetLastError();
}

template <typename T>
cudaError_t Path<T>::zcol_persist(const Plan *d_plans, const BatchRound &r, int *counter, int blocks, size_t smem,
                                  cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  k_zcol_persist<T><<<blocks, kPersistThreads, smem, st>>>(d_plans, r, counter);
  return cudaGetLastError();
}

template <typename T>
cudaError_t Path<T>::descriptors(const Plan &p, double *moments, double *overlap, cudaStream_t st) {
  k_orb_moments<T><<<p.n_occ, 256, 0, st>>>(p, moments);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_pair_overlap<T><<<dim3(p.n_occ, p.n_occ), 256, 0, st>>>(p, overlap);
  return cudaGetLastError();
}

template <typename T>
cudaError_t Path<T>::direct_cross(const Plan &pa, const Plan &pb, int gp0, int np, double coef, double *y,
                                  double *acc, cudaStream_t st) {
  const int th = pb.n_occ < 128 ? ((pb.n_occ + 31) / 32) * 32 : 128;
  k_direct_cross<T><<<dim3(np, pa.n_occ), th, 0, st>>>(pa, pb, np, (const cpx<T> *)pa.mdiag,
                                                       (const cpx<T> *)pb.mdiag, y);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_accum_cross<<<(pa.n_occ * pb.n_occ + 127) / 128, 128, 0, st>>>(pa, pb.n_occ, gp0, np, coef, y, acc);
  return cudaGetLastError();
}

template <typename T> cudaError_t Path<T>::sum(int n, const double *x, double *out, cudaStream_t st) {
  k_sum<<<1, 256, 0, st>>>(n, x, out);
  return cudaGetLastError();
}

template <typename T> cudaError_t Path<T>::zero_acc(const Plan &p, cudaStream_t st) {
  k_zero_acc<<<(p.n_occ * p.n_occ + 255) / 256, 256, 0, st>>>(p);
  return cudaGetLastError();
}

template <typename T> cudaError_t Path<T>::finish(const Plan &p, cudaStream_t st, StageTimer *tm) {
  ScopedStage s(tm, kStageAccum);
  k_finish<<<1, 256, 0, st>>>(p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || p.n_lev < 2) return e;
  k_finish_lev<<<1, 256, 0, st>>>(p);
  return cudaGetLastError();
}

}  // namespace ltmp2

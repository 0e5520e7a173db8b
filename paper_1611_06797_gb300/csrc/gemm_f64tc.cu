// Host side of the FP64 tensor-core GEMM (exact integer slices, gemm_f64tc.cuh): slice
// buffers and tensor maps of a context, the per-tau split of P_r, the per-slab product
// W^T = S^T P_r, and ltmp2_dgemm_nt (the same product on caller matrices, for tests).
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/ltmp2.h"
#include "gemm_f64tc.cuh"
#include "plan.h"

namespace ltmp2 {

int tc_make_map_sw64(CUtensorMap *m, float *base, int rows, int kpad, int box_rows, int box_k);

namespace {

struct OzMaps {
  CUtensorMap a, b, bv;
};

int kpad_of(int k) { return ((k + oz::BK - 1) / oz::BK) * oz::BK; }
int stacked_rows(int rows) { return 2 * (((rows + 63) / 64) * 64); }

cudaError_t set_attributes() {
  static std::once_flag once;
  static cudaError_t e = cudaSuccess;
  std::call_once(once, [] {
    e = cudaFuncSetAttribute(oz::k_dgemm_oz<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, oz::SMEM);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(oz::k_dgemm_oz<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, oz::SMEM);
  });
  return e;
}

int check_flag(int *err) {
  int flag = 0;
  if (cudaMemcpy(&flag, err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return LTMP2_ERR_CUDA;
  if (flag) {
    cudaMemset(err, 0, sizeof(int));
    return LTMP2_ERR_TIMEOUT;
  }
  return LTMP2_OK;
}

}  // namespace

size_t oz_bytes(int rows_cap, int npw, int nv) {
  const size_t kp = (size_t)kpad_of(npw), ar = (size_t)stacked_rows(rows_cap);
  return sizeof(float) * kp * oz::S * (ar + (size_t)npw + (size_t)nv) +
         sizeof(double) * (ar + (size_t)npw + (size_t)nv) + 1024;
}

cudaError_t oz_init(OzResources &r, void *mem, int rows_cap, int npw, int nv) {
  cudaError_t e = set_attributes();
  if (e != cudaSuccess) return e;
  r.rows_cap = rows_cap;
  r.npw = npw;
  r.nv = nv;
  r.kpad = kpad_of(npw);
  r.arows = stacked_rows(rows_cap);
  const size_t kp = (size_t)r.kpad;
  char *p = static_cast<char *>(mem);
  r.a = reinterpret_cast<float *>(p);
  p += sizeof(float) * kp * oz::S * r.arows;
  r.b = reinterpret_cast<float *>(p);
  p += sizeof(float) * kp * oz::S * npw;
  r.bv = reinterpret_cast<float *>(p);
  p += sizeof(float) * kp * oz::S * nv;
  r.sa = reinterpret_cast<double *>(p);
  p += sizeof(double) * r.arows;
  r.sb = reinterpret_cast<double *>(p);
  p += sizeof(double) * npw;
  r.sbv = reinterpret_cast<double *>(p);
  p += sizeof(double) * nv;
  r.err = reinterpret_cast<int *>(p);
  if ((e = cudaMemset(r.err, 0, sizeof(int))) != cudaSuccess) return e;
  OzMaps *m = new OzMaps();
  if (tc_make_map_sw64(&m->a, r.a, oz::S * r.arows, r.kpad, oz::BM, oz::BK) ||
      tc_make_map_sw64(&m->b, r.b, oz::S * npw, r.kpad, oz::BN, oz::BK) ||
      (nv > 0 && tc_make_map_sw64(&m->bv, r.bv, oz::S * nv, r.kpad, oz::BN, oz::BK))) {
    delete m;
    return cudaErrorInvalidValue;
  }
  r.maps = m;
  return cudaSuccess;
}

cudaError_t oz_split_cv(const OzResources &r, const double *cv, cudaStream_t st) {
  if (r.nv < 1) return cudaSuccess;
  oz::k_oz_split_rows<<<r.nv, 256, 0, st>>>(cv, r.nv, r.npw, r.npw, nullptr, r.kpad, r.kpad, r.nv, r.bv, r.sbv);
  return cudaGetLastError();
}

bool oz_green_fits(const OzResources &r) { return r.maps && r.nv > 0 && r.npw <= r.arows; }

cudaError_t oz_green(const OzResources &r, const double *rvt, const double *dv, int nv, double *pr, cudaStream_t st) {
  if (!oz_green_fits(r) || nv < 1 || nv > r.nv) return cudaErrorInvalidValue;
  const OzMaps &m = *static_cast<const OzMaps *>(r.maps);
  const int kf = kpad_of(nv);
  // A = R_v'^T D' (rows q, columns a < nv), B = R_v'^T: P_r = A B^T
  oz::k_oz_split_rows<<<(r.npw + oz::BM - 1) / oz::BM * oz::BM, 256, 0, st>>>(rvt, r.npw, nv, r.nv, dv, kf, r.kpad,
                                                                             r.arows, r.a, r.sa);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  oz::k_oz_split_rows<<<r.npw, 256, 0, st>>>(rvt, r.npw, nv, r.nv, nullptr, kf, r.kpad, r.npw, r.b, r.sb);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  dim3 grid((r.npw + oz::BN - 1) / oz::BN, (r.npw + oz::BM - 1) / oz::BM);
  oz::k_dgemm_oz<false><<<grid, 160, oz::SMEM, st>>>(m.a, m.b, r.npw, r.npw, kf / oz::BK, r.arows, r.npw, r.sa, r.sb,
                                                     pr, r.npw, r.err);
  return cudaGetLastError();
}

cudaError_t oz_virtual(const OzResources &r, const void *st_in, int rows, const double *rvt, const double *dv, int nv,
                       void *x, void *wt, cudaStream_t st) {
  if (rows > r.rows_cap || !r.maps || nv < 1 || nv > r.nv) return cudaErrorInvalidValue;
  const OzMaps &m = *static_cast<const OzMaps *>(r.maps);
  const int ar = stacked_rows(rows), kf = kpad_of(nv);
  dim3 g1((nv + oz::BN - 1) / oz::BN, ar / oz::BM), g2((r.npw + oz::BN - 1) / oz::BN, ar / oz::BM);
  // X^T = (U S)^T R_v'^T: A = the gathered states (K = n_pw), B = the first nv rows of R_v
  oz::k_oz_split_stacked<<<ar / 2, 256, 0, st>>>(static_cast<const double2 *>(st_in), rows, r.npw, r.npw, r.kpad,
                                                 r.kpad, r.arows, r.a, r.sa);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  oz::k_dgemm_oz<true><<<g1, 160, oz::SMEM, st>>>(m.a, m.bv, rows, nv, r.kpad / oz::BK, r.arows, r.nv, r.sa, r.sbv,
                                                  static_cast<double *>(x), nv, r.err);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // W^T = X^T (D' R_v'): A = X (K = nv), B = R_v'^T D' (rows p, columns a < nv)
  oz::k_oz_split_stacked<<<ar / 2, 256, 0, st>>>(static_cast<const double2 *>(x), rows, nv, nv, kf, r.kpad, r.arows,
                                                 r.a, r.sa);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  oz::k_oz_split_rows<<<r.npw, 256, 0, st>>>(rvt, r.npw, nv, r.nv, dv, kf, r.kpad, r.npw, r.b, r.sb);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  oz::k_dgemm_oz<true><<<g2, 160, oz::SMEM, st>>>(m.a, m.b, rows, r.npw, kf / oz::BK, r.arows, r.npw, r.sa, r.sb,
                                                  static_cast<double *>(wt), r.npw, r.err);
  return cudaGetLastError();
}

void oz_release(OzResources &r) {
  delete static_cast<OzMaps *>(r.maps);
  r.maps = nullptr;
}

cudaError_t oz_split_b(const OzResources &r, const double *pr, cudaStream_t st) {
  oz::k_oz_split_rows<<<r.npw, 256, 0, st>>>(pr, r.npw, r.npw, r.npw, nullptr, r.kpad, r.kpad, r.npw, r.b, r.sb);
  return cudaGetLastError();
}

cudaError_t oz_wgemm(const OzResources &r, const void *st_in, int rows, void *wt, cudaStream_t st) {
  if (rows > r.rows_cap || !r.maps) return cudaErrorInvalidValue;
  const OzMaps &m = *static_cast<const OzMaps *>(r.maps);
  const int ar = stacked_rows(rows);
  oz::k_oz_split_stacked<<<ar / 2, 256, 0, st>>>(static_cast<const double2 *>(st_in), rows, r.npw, r.npw, r.kpad,
                                                 r.kpad, r.arows, r.a, r.sa);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  dim3 grid((r.npw + oz::BN - 1) / oz::BN, ar / oz::BM);
  oz::k_dgemm_oz<true><<<grid, 160, oz::SMEM, st>>>(m.a, m.b, rows, r.npw, r.kpad / oz::BK, r.arows, r.npw, r.sa,
                                                    r.sb, static_cast<double *>(wt), r.npw, r.err);
  return cudaGetLastError();
}

int oz_check(const OzResources &r) { return check_flag(r.err); }

}  // namespace ltmp2

extern "C" int ltmp2_dgemm_nt(int m, int n, int k, const double *a, int lda, const double *b, int ldb, double *c,
                              int ldc) {
  using namespace ltmp2;
  if (m < 1 || n < 1 || k < 1 || !a || !b || !c || lda < k || ldb < k || ldc < n) return LTMP2_ERR_INVALID_ARG;
  cudaError_t e = set_attributes();
  if (e != cudaSuccess) return LTMP2_ERR_CUDA;
  const int kpad = kpad_of(k), ar = ((m + oz::BM - 1) / oz::BM) * oz::BM;
  float *pa = nullptr, *pb = nullptr;
  double *sa = nullptr, *sb = nullptr;
  int *err = nullptr;
  int rc = LTMP2_OK;
  auto cleanup = [&] {
    cudaFree(pa);
    cudaFree(pb);
    cudaFree(sa);
    cudaFree(sb);
    cudaFree(err);
  };
  if (cudaMalloc(&pa, sizeof(float) * (size_t)oz::S * ar * kpad) != cudaSuccess ||
      cudaMalloc(&pb, sizeof(float) * (size_t)oz::S * n * kpad) != cudaSuccess ||
      cudaMalloc(&sa, sizeof(double) * ar) != cudaSuccess || cudaMalloc(&sb, sizeof(double) * n) != cudaSuccess ||
      cudaMalloc(&err, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    cleanup();
    return LTMP2_ERR_OOM;
  }
  OzMaps maps;
  if (tc_make_map_sw64(&maps.a, pa, oz::S * ar, kpad, oz::BM, oz::BK) ||
      tc_make_map_sw64(&maps.b, pb, oz::S * n, kpad, oz::BN, oz::BK)) {
    cleanup();
    return LTMP2_ERR_INVALID_ARG;
  }
  cudaMemset(err, 0, sizeof(int));
  oz::k_oz_split_rows<<<ar, 256>>>(a, m, k, lda, nullptr, kpad, kpad, ar, pa, sa);
  oz::k_oz_split_rows<<<n, 256>>>(b, n, k, ldb, nullptr, kpad, kpad, n, pb, sb);
  dim3 grid((n + oz::BN - 1) / oz::BN, ar / oz::BM);
  oz::k_dgemm_oz<false><<<grid, 160, oz::SMEM>>>(maps.a, maps.b, m, n, kpad / oz::BK, ar, n, sa, sb, c, ldc, err);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) rc = LTMP2_ERR_CUDA;
  if (!rc) rc = check_flag(err);
  cleanup();
  return rc;
}

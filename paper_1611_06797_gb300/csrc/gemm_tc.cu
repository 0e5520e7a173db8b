// Host side of the tcgen05 3xTF32 transformed-state GEMM: operand buffers, TMA tensor
// maps (built once per context) and the launchers used by the precision form.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include "gemm_tc.cuh"
#include "plan.h"

namespace ltmp2 {

namespace {
// cuTensorMapEncodeTiled through the runtime's driver entry point, so the library does
// not link libcuda directly (it still loads on hosts without a GPU driver).
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

int make_map(CUtensorMap *m, float *base, int rows, int kpad, int box_rows) {
  cuuint64_t dims[2] = {(cuuint64_t)kpad, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)kpad * sizeof(float)};
  cuuint32_t box[2] = {(cuuint32_t)tc::BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1u, 1u};
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return -1;
  const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, estr,
                                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : -1;
}
}  // namespace

int tc_variant_bn(int variant) { return variant <= 1 ? 128 : 64; }  // variant 4: drained, 64

int tc_kpad(int npw) { return ((2 * npw + tc::BK - 1) / tc::BK) * tc::BK; }

size_t tc_bytes(int rows_cap, int npw) {
  const size_t kp = (size_t)tc_kpad(npw);
  return sizeof(float) * kp * (4 * (size_t)rows_cap + 2 * (size_t)npw) + 256;
}

cudaError_t tc_init(TcResources &r, void *mem, int rows_cap, int npw, int variant) {
  r.variant = variant;
  r.rows_cap = rows_cap;
  r.npw = npw;
  r.kpad = tc_kpad(npw);
  const size_t a = (size_t)rows_cap * r.kpad, b = (size_t)npw * r.kpad;
  float *f = static_cast<float *>(mem);
  r.a1h = f; r.a1l = f + a; r.a2h = f + 2 * a; r.a2l = f + 3 * a;
  r.bh = f + 4 * a; r.bl = f + 4 * a + b;
  r.err = reinterpret_cast<int *>(f + 4 * a + 2 * b);
  tc::TcMaps *mp = new tc::TcMaps();
  const int bn = tc_variant_bn(r.variant);
  if (make_map(&mp->a1h, r.a1h, rows_cap, r.kpad, tc::BM) || make_map(&mp->a1l, r.a1l, rows_cap, r.kpad, tc::BM) ||
      make_map(&mp->a2h, r.a2h, rows_cap, r.kpad, tc::BM) || make_map(&mp->a2l, r.a2l, rows_cap, r.kpad, tc::BM) ||
      make_map(&mp->bh, r.bh, npw, r.kpad, bn) || make_map(&mp->bl, r.bl, npw, r.kpad, bn)) {
    delete mp;
    return cudaErrorInvalidValue;
  }
  r.maps = mp;
  cudaError_t e;
#define LTMP2_TC_ATTR(BN, NR)                                                                  \
  e = cudaFuncSetAttribute(tc::k_tc_cgemm<BN, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                           tc::TcCfg<BN, NR>::SMEM_BYTES);                                     \
  if (e != cudaSuccess) return e;
  LTMP2_TC_ATTR(128, 1)
  LTMP2_TC_ATTR(128, 2)
  LTMP2_TC_ATTR(64, 2)
  LTMP2_TC_ATTR(64, 4)
#undef LTMP2_TC_ATTR
  e = cudaFuncSetAttribute(tc::k_tc_cgemm_drain<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           tc::TcCfg<64, 2>::SMEM_BYTES);
  if (e != cudaSuccess) return e;
  return cudaMemset(r.err, 0, sizeof(int));
}

void tc_release(TcResources &r) {
  delete static_cast<tc::TcMaps *>(r.maps);
  r.maps = nullptr;
}

cudaError_t tc_pack_b(const TcResources &r, const void *pt, cudaStream_t st) {
  tc::k_pack_b<<<dim3((r.kpad / 2 + 255) / 256, r.npw), 256, 0, st>>>(static_cast<const float2 *>(pt), r.npw,
                                                                        r.kpad, r.bh, r.bl);
  return cudaGetLastError();
}

cudaError_t tc_wgemm(const TcResources &r, const void *st_in, int rows, void *wt, cudaStream_t st) {
  if (rows > r.rows_cap) return cudaErrorInvalidValue;
  tc::k_pack_a<<<dim3((r.kpad / 2 + 255) / 256, rows), 256, 0, st>>>(static_cast<const float2 *>(st_in), rows,
                                                                       r.npw, r.kpad, r.a1h, r.a1l, r.a2h, r.a2l);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const tc::TcMaps &m = *static_cast<const tc::TcMaps *>(r.maps);
  const int variant = r.variant;
#define LTMP2_TC_LAUNCH(BN, NR)                                                                              \
  {                                                                                                          \
    dim3 grid((r.npw + BN - 1) / BN, (rows + tc::BM - 1) / tc::BM);                                          \
    tc::k_tc_cgemm<BN, NR><<<grid, 128, tc::TcCfg<BN, NR>::SMEM_BYTES, st>>>(                                \
        m.a1h, m.a1l, m.a2h, m.a2l, m.bh, m.bl, rows, r.npw, r.kpad / tc::BK, static_cast<float2 *>(wt), r.npw, \
        r.err);                                                                                              \
  }
  if (variant == 0) LTMP2_TC_LAUNCH(128, 1)
  else if (variant == 1) LTMP2_TC_LAUNCH(128, 2)
  else if (variant == 2) LTMP2_TC_LAUNCH(64, 2)
  else if (variant == 3) LTMP2_TC_LAUNCH(64, 4)
  else {
    dim3 grid((r.npw + 63) / 64, (rows + tc::BM - 1) / tc::BM);
    tc::k_tc_cgemm_drain<64><<<grid, 160, tc::TcCfg<64, 2>::SMEM_BYTES, st>>>(
        m.a1h, m.a1l, m.a2h, m.a2l, m.bh, m.bl, rows, r.npw, r.kpad / tc::BK, static_cast<float2 *>(wt), r.npw,
        r.err);
  }
#undef LTMP2_TC_LAUNCH
  return cudaGetLastError();
}

}  // namespace ltmp2

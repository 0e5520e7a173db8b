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

int make_map(CUtensorMap *m, float *base, int rows, int kpad, int box_rows, int box_k = tc::BK,
             CUtensorMapSwizzle sw = CU_TENSOR_MAP_SWIZZLE_128B) {
  cuuint64_t dims[2] = {(cuuint64_t)kpad, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)kpad * sizeof(float)};
  cuuint32_t box[2] = {(cuuint32_t)box_k, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1u, 1u};
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return -1;
  const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, estr,
                                            CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
                                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : -1;
}
}  // namespace

// 64-byte-swizzled K-major fp32 operand map (the FP64 tensor-core GEMM's slices use it too)
int tc_make_map_sw64(CUtensorMap *m, float *base, int rows, int kpad, int box_rows, int box_k) {
  return make_map(m, base, rows, kpad, box_rows, box_k, CU_TENSOR_MAP_SWIZZLE_64B);
}

// Layouts the autotuner chooses from: 4 drained (separate Re / Im operands, N 64, two-stage
// ring), 5 stacked Re / Im rows with a three-stage 64-byte-swizzle ring (the default and
// the only layout for real orbitals).
int tc_variant_bn(int variant) { return variant == 5 ? tc::S_BN : 64; }

int tc_kpad(int npw) { return ((2 * npw + tc::BK - 1) / tc::BK) * tc::BK; }

static int rows_pad(int rows) { return ((rows + 127) / 128) * 128; }

size_t tc_bytes(int rows_cap, int npw) {
  const size_t kp = (size_t)tc_kpad(npw);
  return sizeof(float) * kp * (4 * (size_t)rows_pad(rows_cap) + 2 * (size_t)npw) + 256;
}

cudaError_t tc_init(TcResources &r, void *mem, int rows_cap, int npw, int variant, bool real) {
  if (variant != 4 && variant != 5) return cudaErrorInvalidValue;
  if (real && variant != 5) return cudaErrorInvalidValue;  // only the stacked kernel has a real form
  r.variant = variant;
  r.real = real;
  r.rows_cap = rows_cap;
  r.npw = npw;
  // real basis: K = n_pw (a multiple of the 32-element k block), at most the complex size
  r.kpad = real ? ((npw + tc::BK - 1) / tc::BK) * tc::BK : tc_kpad(npw);
  const int rp = rows_pad(rows_cap);
  const size_t a = (size_t)rp * r.kpad, b = (size_t)npw * r.kpad;
  float *f = static_cast<float *>(mem);
  r.a1h = f; r.a1l = f + a; r.a2h = f + 2 * a; r.a2l = f + 3 * a;
  r.bh = f + 4 * a; r.bl = f + 4 * a + b;
  r.err = reinterpret_cast<int *>(f + 4 * a + 2 * b);
  tc::TcMaps *mp = new tc::TcMaps();
  int bad = 0;
  if (variant == 5) {
    // stacked operand: hi in a1h and lo in a1l, 2 rp rows each (spanning a1h..a2l)
    r.a1l = f + 2 * a;
    bad |= make_map(&mp->a1h, r.a1h, 2 * rp, r.kpad, 128, tc::S_BK, CU_TENSOR_MAP_SWIZZLE_64B);
    bad |= make_map(&mp->a1l, r.a1l, 2 * rp, r.kpad, 128, tc::S_BK, CU_TENSOR_MAP_SWIZZLE_64B);
    bad |= make_map(&mp->bh, r.bh, npw, r.kpad, tc::S_BN, tc::S_BK, CU_TENSOR_MAP_SWIZZLE_64B);
    bad |= make_map(&mp->bl, r.bl, npw, r.kpad, tc::S_BN, tc::S_BK, CU_TENSOR_MAP_SWIZZLE_64B);
  } else {
    const int bn = tc_variant_bn(variant);
    bad |= make_map(&mp->a1h, r.a1h, rows_cap, r.kpad, tc::BM) | make_map(&mp->a1l, r.a1l, rows_cap, r.kpad, tc::BM);
    bad |= make_map(&mp->a2h, r.a2h, rows_cap, r.kpad, tc::BM) | make_map(&mp->a2l, r.a2l, rows_cap, r.kpad, tc::BM);
    bad |= make_map(&mp->bh, r.bh, npw, r.kpad, bn) | make_map(&mp->bl, r.bl, npw, r.kpad, bn);
  }
  if (bad) {
    delete mp;
    return cudaErrorInvalidValue;
  }
  r.maps = mp;
  cudaError_t e = cudaFuncSetAttribute(tc::k_tc_cgemm_drain<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           tc::TcCfg<64, 2>::SMEM_BYTES);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(tc::k_tc_cgemm_stacked, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::S_SMEM);
  if (e != cudaSuccess) return e;
  return cudaMemset(r.err, 0, sizeof(int));
}

void tc_release(TcResources &r) {
  delete static_cast<tc::TcMaps *>(r.maps);
  r.maps = nullptr;
  delete static_cast<tc::TcMaps *>(r.gmaps);
  r.gmaps = nullptr;
  delete static_cast<tc::TcMaps *>(r.dmaps);
  r.dmaps = nullptr;
  r.green = r.direct = false;   // their tensor maps are gone: set up again before any use
}

static int kpad_of(int k) { return ((k + tc::BK - 1) / tc::BK) * tc::BK; }

size_t tc_green_bytes(int npw, int nv) {
  const size_t kp = (size_t)kpad_of(nv);
  const size_t arows = 2 * (size_t)rows_pad(((npw + 1) / 2 + 63) / 64 * 64);
  return sizeof(float) * ((size_t)npw * nv + kp * (2 * arows + 2 * (size_t)npw)) + 1024;
}

cudaError_t tc_green_init(TcResources &r, void *mem, const float *cv, int nv, cudaStream_t st) {
  if (!r.real || r.variant != 5) return cudaErrorInvalidValue;
  const int npw = r.npw;
  r.nv = nv;
  r.kpad_v = kpad_of(nv);
  r.grows = (npw + 1) / 2;
  const size_t arows = 2 * (size_t)rows_pad((r.grows + 63) / 64 * 64);
  const size_t kp = (size_t)r.kpad_v;
  float *f = static_cast<float *>(mem);
  r.rvt = f;
  f += ((size_t)npw * nv + 63) / 64 * 64;
  r.gah = f; f += arows * kp;
  r.gal = f; f += arows * kp;
  r.gbh = f; f += (size_t)npw * kp;
  r.gbl = f;
  tc::TcMaps *mp = new tc::TcMaps();
  int bad = 0;
  bad |= make_map(&mp->a1h, r.gah, (int)arows, r.kpad_v, 128, tc::S_BK, CU_TENSOR_MAP_SWIZZLE_64B);
  bad |= make_map(&mp->a1l, r.gal, (int)arows, r.kpad_v, 128, tc::S_BK, CU_TENSOR_MAP_SWIZZLE_64B);
  bad |= make_map(&mp->bh, r.gbh, npw, r.kpad_v, tc::S_BN, tc::S_BK, CU_TENSOR_MAP_SWIZZLE_64B);
  bad |= make_map(&mp->bl, r.gbl, npw, r.kpad_v, tc::S_BN, tc::S_BK, CU_TENSOR_MAP_SWIZZLE_64B);
  if (bad) {
    delete mp;
    return cudaErrorInvalidValue;
  }
  r.gmaps = mp;
  tc::k_transpose_f<<<dim3((npw + 31) / 32, (nv + 31) / 32), dim3(32, 8), 0, st>>>(nv, npw, cv, r.rvt);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  tc::k_pack_rows<<<dim3((r.kpad_v + 255) / 256, npw), 256, 0, st>>>(r.rvt, nv, r.kpad_v, r.gbh, r.gbl);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  r.green = r.use_green = true;
  return cudaSuccess;
}

cudaError_t tc_green(const TcResources &r, const float *dv, void *pt, cudaStream_t st) {
  const tc::TcMaps &m = *static_cast<const tc::TcMaps *>(r.gmaps);
  const int r64 = (r.grows + 63) / 64 * 64;
  tc::k_pack_green_a<<<dim3((r.kpad_v + 255) / 256, r64), 256, 0, st>>>(r.rvt, dv, r.npw, r.nv, r.kpad_v, r.gah,
                                                                        r.gal);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  dim3 grid((r.npw + tc::S_BN - 1) / tc::S_BN, r64 / 64);
  tc::k_tc_cgemm_stacked<<<grid, 160, tc::S_SMEM, st>>>(m.a1h, m.a1l, m.bh, m.bl, r.grows, r.npw,
                                                        r.kpad_v / tc::S_BK, static_cast<float2 *>(pt), r.npw, r.err);
  return cudaGetLastError();
}

size_t tc_direct_bytes(int no, int naux, int slots) {
  const size_t kp = (size_t)kpad_of(naux);
  const size_t r64 = ((size_t)no + 63) / 64 * 64;
  return sizeof(float) * kp * (2 * 2 * r64 * slots + 2 * 2 * (size_t)no * slots) +
         sizeof(float2) * (size_t)slots * no * 2 * no + 1024;
}

cudaError_t tc_direct_init(TcResources &r, void *mem, int no, int naux, int slots) {
  r.dno = no;
  r.dnaux = naux;
  r.dslots = slots;
  r.dkpad = kpad_of(naux);
  r.dr64 = (no + 63) / 64 * 64;
  const size_t kp = (size_t)r.dkpad, arows = 2 * (size_t)r.dr64 * slots, brows = 2 * (size_t)no * slots;
  float *f = static_cast<float *>(mem);
  r.dah = f; f += arows * kp;
  r.dal = f; f += arows * kp;
  r.dbh = f; f += brows * kp;
  r.dbl = f; f += brows * kp;
  r.dc = reinterpret_cast<float2 *>(f);
  tc::TcMaps *mp = new tc::TcMaps();
  int bad = 0;
  bad |= make_map(&mp->a1h, r.dah, (int)arows, r.dkpad, 128, tc::S_BK, CU_TENSOR_MAP_SWIZZLE_64B);
  bad |= make_map(&mp->a1l, r.dal, (int)arows, r.dkpad, 128, tc::S_BK, CU_TENSOR_MAP_SWIZZLE_64B);
  bad |= make_map(&mp->bh, r.dbh, (int)brows, r.dkpad, tc::S_BN, tc::S_BK, CU_TENSOR_MAP_SWIZZLE_64B);
  bad |= make_map(&mp->bl, r.dbl, (int)brows, r.dkpad, tc::S_BN, tc::S_BK, CU_TENSOR_MAP_SWIZZLE_64B);
  if (bad) {
    delete mp;
    return cudaErrorInvalidValue;
  }
  r.dmaps = mp;
  r.direct = r.use_direct = true;
  return cudaSuccess;
}

cudaError_t tc_direct(const TcResources &r, const void *mdiag, const float *v, int np, double2 *yd, cudaStream_t st) {
  if (np > r.dslots) return cudaErrorInvalidValue;
  const tc::TcMaps &m = *static_cast<const tc::TcMaps *>(r.dmaps);
  tc::k_pack_direct<<<dim3(r.dkpad / 32, r.dr64 / 32, np), dim3(32, 8), 0, st>>>(
      static_cast<const float2 *>(mdiag), v, r.dnaux, r.dno, r.dkpad, r.dr64, r.dah, r.dal, r.dbh, r.dbl);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int no = r.dno;
  dim3 grid((2 * no + tc::S_BN - 1) / tc::S_BN, r.dr64 / 64, np);
  tc::k_tc_cgemm_stacked<<<grid, 160, tc::S_SMEM, st>>>(m.a1h, m.a1l, m.bh, m.bl, no, 2 * no, r.dkpad / tc::S_BK,
                                                        r.dc, 2 * no, r.err, 2 * r.dr64, 2 * no,
                                                        (long long)no * 2 * no);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  tc::k_direct_combine<<<dim3((no * no + 255) / 256, np), 256, 0, st>>>(r.dc, no, yd);
  return cudaGetLastError();
}

cudaError_t tc_pack_b(const TcResources &r, const void *pt, cudaStream_t st) {
  if (r.green_on()) {   // the pair-interleaved output of tc_green
    tc::k_pack_b_pairs<<<dim3((r.kpad + 255) / 256, r.npw), 256, 0, st>>>(static_cast<const float2 *>(pt), r.npw,
                                                                            r.kpad, r.bh, r.bl);
    return cudaGetLastError();
  }
  if (r.real) {
    tc::k_pack_b_real<<<dim3((r.kpad + 255) / 256, r.npw), 256, 0, st>>>(static_cast<const float *>(pt), r.npw,
                                                                           r.kpad, r.bh, r.bl);
    return cudaGetLastError();
  }
  tc::k_pack_b<<<dim3((r.kpad / 2 + 255) / 256, r.npw), 256, 0, st>>>(static_cast<const float2 *>(pt), r.npw,
                                                                        r.kpad, r.bh, r.bl);
  return cudaGetLastError();
}

cudaError_t tc_wgemm(const TcResources &r, const void *st_in, int rows, void *wt, cudaStream_t st) {
  if (rows > r.rows_cap) return cudaErrorInvalidValue;
  const tc::TcMaps &m = *static_cast<const tc::TcMaps *>(r.maps);
  const int variant = r.variant;
  cudaError_t e;
  if (variant == 5) {
    const int r64 = ((rows + 63) / 64) * 64;   // zero-filled up to a whole 64-row block
    if (r.real)
      tc::k_pack_a_stacked_real<<<dim3((r.kpad + 255) / 256, r64), 256, 0, st>>>(
          static_cast<const float2 *>(st_in), rows, r.npw, r.kpad, r.a1h, r.a1l);
    else
      tc::k_pack_a_stacked<<<dim3((r.kpad / 2 + 255) / 256, r64), 256, 0, st>>>(
        static_cast<const float2 *>(st_in), rows, r.npw, r.kpad, r.a1h, r.a1l);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    dim3 grid((r.npw + tc::S_BN - 1) / tc::S_BN, r64 / 64);
    tc::k_tc_cgemm_stacked<<<grid, 160, tc::S_SMEM, st>>>(m.a1h, m.a1l, m.bh, m.bl, rows, r.npw, r.kpad / tc::S_BK,
                                                          static_cast<float2 *>(wt), r.npw, r.err);
    return cudaGetLastError();
  }
  tc::k_pack_a<<<dim3((r.kpad / 2 + 255) / 256, rows), 256, 0, st>>>(static_cast<const float2 *>(st_in), rows,
                                                                       r.npw, r.kpad, r.a1h, r.a1l, r.a2h, r.a2l);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  dim3 grid((r.npw + 63) / 64, (rows + tc::BM - 1) / tc::BM);
  tc::k_tc_cgemm_drain<64><<<grid, 160, tc::TcCfg<64, 2>::SMEM_BYTES, st>>>(
      m.a1h, m.a1l, m.a2h, m.a2l, m.bh, m.bl, rows, r.npw, r.kpad / tc::BK, static_cast<float2 *>(wt), r.npw,
      r.err);
  return cudaGetLastError();
}

cudaError_t tc_wait_selftest(int *err, unsigned long long limit_ns, cudaStream_t st) {
  tc::k_wait_selftest<<<1, 32, 0, st>>>(err, limit_ns);
  return cudaGetLastError();
}

}  // namespace ltmp2

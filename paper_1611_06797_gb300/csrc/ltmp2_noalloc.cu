// ltmp2_energy_noalloc: the energy of ltmp2_setup + ltmp2_energy in one call that
// makes no device allocation.
//
// Some callers cannot call cudaMalloc: a process running under a fixed device-memory
// budget that is already spent by its own pool, code that must not trigger the
// implicit device synchronisation cudaMalloc/cudaFree can cause (a latency-critical
// loop sharing the GPU with other streams), or a plug-in whose host application owns
// all device memory.  For small systems this entry point keeps every device buffer
// of the path (input copies, index tables, Green's function, transformed states,
// FFT intermediates, pair sums, accumulators) inside one file-scope device array
// of kNoAllocScratchBytes bytes.  The array is part of the library image: every GPU
// that loads the library holds it until the process exits.
//
// The kernels are the ones ltmp2_energy launches; only the memory they run in differs.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <type_traits>
#include <vector>

#include "../../include/ltmp2.h"
#include "fft.cuh"
#include "host_plan.h"
#include "plan.h"

using namespace ltmp2;

namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)32 << 20;  // 32 MiB
constexpr size_t kAlign = 256;

}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

std::mutex g_scratch_mutex;
void *g_scratch_ptr[64] = {nullptr};

// Device address of the scratch array on the current device (host code cannot use the
// array's name as an address).  Looked up once per device and cached; a cudaDeviceReset
// of that device invalidates the cached address, so calls after a reset are not
// supported.
int scratch_base(void **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return LTMP2_ERR_CUDA;
  }
  if (dev < 0 || dev >= 64) return LTMP2_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return LTMP2_ERR_CUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return LTMP2_OK;
}

struct Arena {
  unsigned char *base;
  size_t used = 0, cap;
  Arena(void *b, size_t c) : base(static_cast<unsigned char *>(b)), cap(c) {}
  // reserve bytes (rounded up to kAlign); nullptr when the array is full
  void *take(size_t bytes) {
    const size_t need = (std::max<size_t>(bytes, 1) + kAlign - 1) / kAlign * kAlign;
    if (used + need > cap) return nullptr;
    void *p = base + used;
    used += need;
    return p;
  }
  size_t left() const { return cap - used; }
};

int copy_in(void *dst, const void *src, size_t bytes, cudaStream_t st) {
  if (cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) {
    cudaGetLastError();
    return LTMP2_ERR_CUDA;
  }
  return LTMP2_OK;
}

template <typename T>
int run_noalloc(const ltmp2_system *sys, Plan &p, Arena &ar, const std::vector<int> &order, int n_tau,
                const double *tau, const double *w, cudaStream_t st, double *e_d, double *e_x, double *e_pair) {
  struct C2 { T x, y; };
  const size_t cs = sizeof(C2);
  const size_t n3 = (size_t)p.n * p.n * p.n;
  // coefficients in the path's plane-wave order
  std::vector<C2> hv((size_t)p.n_v * p.n_pw), ho((size_t)p.n_occ * p.n_pw);
  for (int r = 0; r < p.n_orb; ++r)
    for (int q = 0; q < p.n_pw; ++q) {
      const double *c = sys->coeff + ((size_t)r * p.n_pw + order[q]) * 2;
      const C2 v = {(T)c[0], (T)c[1]};
      if (r < p.n_occ) ho[(size_t)r * p.n_pw + q] = v;
      else hv[(size_t)(r - p.n_occ) * p.n_pw + q] = v;
    }
  // real orbitals: the virtuals' real-basis coordinates (see the real-basis kernels)
  std::vector<T> hr;
  if (p.real_basis) {
    hr.resize((size_t)p.n_v * p.n_pw);
    const T r2 = (T)1.4142135623730950488016887242097;
    for (int r = 0; r < p.n_v; ++r)
      for (int q = 0; q < p.n_pw; ++q) {
        const int *mq = sys->miller + 3 * order[q];
        const C2 v = hv[(size_t)r * p.n_pw + q];
        const bool zero = mq[0] == 0 && mq[1] == 0 && mq[2] == 0;
        const bool prim = mq[0] != 0 ? mq[0] > 0 : (mq[1] != 0 ? mq[1] > 0 : mq[2] > 0);
        hr[(size_t)r * p.n_pw + q] = zero ? v.x : (prim ? r2 * v.x : r2 * v.y);
      }
  }
  void *cocc = ar.take(ho.size() * cs);
  p.cv = p.real_basis ? ar.take(hr.size() * sizeof(T)) : ar.take(hv.size() * cs);
  p.cgrid = ar.take(cs * n3 * p.n_occ);
  p.u = ar.take(cs * n3 * p.n_occ);
  p.ut = ar.take(cs * n3 * p.n_occ);
  p.dscale = ar.take(sizeof(T) * p.n_orb);
  p.pt = ar.take((p.real_basis ? sizeof(T) : cs) * (size_t)p.n_pw * p.n_pw);
  const size_t no2 = (size_t)p.n_occ * p.n_occ;
  p.ex = (double *)ar.take(no2 * sizeof(double));
  p.ed = (double *)ar.take(no2 * sizeof(double));
  p.exi = (double *)ar.take(no2 * sizeof(double));
  p.edi = (double *)ar.take(no2 * sizeof(double));
  p.esum = (double *)ar.take(4 * sizeof(double));
  if (!cocc || !p.cv || !p.cgrid || !p.u || !p.ut || !p.dscale || !p.pt || !p.ex || !p.ed || !p.exi || !p.edi || !p.esum)
    return LTMP2_ERR_UNSUPPORTED;
  // slab of primary G' sized to what is left of the array
  const int spp = p.slots_per_prim();
  const size_t cols_pp = (size_t)spp * p.n_occ;
  const size_t per_prim = cs * cols_pp * (2 * (size_t)p.n_pw + (size_t)p.n * p.n_dorb +
                                          (size_t)p.n_occ * p.n * p.n_daux) +
                          cs * spp * (size_t)p.n_aux * p.n_occ + 2 * sizeof(double2) * no2 + 8 * kAlign;
  const size_t z1_min = cs * (size_t)p.n_occ * p.n * p.n_dorb + kAlign;
  if (ar.left() < z1_min + per_prim) return LTMP2_ERR_UNSUPPORTED;
  long long mp = (long long)((ar.left() - z1_min) / per_prim);
  mp = std::min<long long>(mp, std::max<long long>(1, 4096 / (long long)cols_pp));
  mp = std::min<long long>(mp, p.n_prim);
  p.max_prim = (int)std::max<long long>(1, mp);
  const size_t max_cols = cols_pp * p.max_prim;
  p.st = ar.take(cs * max_cols * p.n_pw);
  p.wt = ar.take(cs * max_cols * p.n_pw);
  p.z1 = ar.take(cs * std::max(max_cols, (size_t)p.n_occ) * p.n * p.n_dorb);
  p.tbuf = ar.take(cs * max_cols * p.n_occ * p.n * p.n_daux);
  p.mdiag = ar.take(cs * (size_t)spp * p.max_prim * p.n_aux * p.n_occ);
  p.sx = (double2 *)ar.take(sizeof(double2) * (size_t)p.max_prim * no2);
  p.yd = (double2 *)ar.take(sizeof(double2) * (size_t)p.max_prim * no2);
  if (!p.st || !p.wt || !p.z1 || !p.tbuf || !p.mdiag || !p.sx || !p.yd) return LTMP2_ERR_UNSUPPORTED;

  int rc;
  if ((rc = copy_in(cocc, ho.data(), ho.size() * cs, st))) return rc;
  if (p.real_basis) {
    if ((rc = copy_in(p.cv, hr.data(), hr.size() * sizeof(T), st))) return rc;
  } else {
    if ((rc = copy_in(p.cv, hv.data(), hv.size() * cs, st))) return rc;
  }
  if (Path<T>::init_device() != cudaSuccess) return LTMP2_ERR_CUDA;
  if (Path<T>::setup_occupied(p, cocc, st) != cudaSuccess) return LTMP2_ERR_CUDA;
  // the energy loop of ltmp2_energy, in the same order
  if (Path<T>::zero_acc(p, st) != cudaSuccess) return LTMP2_ERR_CUDA;
  const double nfft = (double)n3;
  for (int k = 0; k < n_tau; ++k) {
    if (Path<T>::green(p, tau[k], st, nullptr) != cudaSuccess) return LTMP2_ERR_CUDA;
    const double coef = w[k] / (p.omega * p.omega * nfft * nfft);
    for (int g0 = 0; g0 < p.n_prim; g0 += p.max_prim) {
      const int np = std::min(p.max_prim, p.n_prim - g0);
      if (Path<T>::slab(p, g0, np, coef, st, nullptr) != cudaSuccess) return LTMP2_ERR_CUDA;
    }
  }
  if (Path<T>::finish(p, st, nullptr) != cudaSuccess) return LTMP2_ERR_CUDA;
  double es[4];
  std::vector<double> ed(no2), ex(no2);
  if (cudaMemcpyAsync(es, p.esum, sizeof(es), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(ed.data(), p.ed, no2 * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(ex.data(), p.ex, no2 * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return LTMP2_ERR_CUDA;
  }
  *e_d = es[0];
  *e_x = es[1];
  if (e_pair)
    for (size_t k = 0; k < no2; ++k) e_pair[k] = ed[k] + ex[k];
  return LTMP2_OK;
}

int energy_noalloc(const ltmp2_system *sys, int n_tau, const double *tau, const double *w, double *e_direct,
                   double *e_exchange, double *e_pair, void *stream) {
  if (!sys || !e_direct || !e_exchange || !tau || !w || n_tau < 1) return LTMP2_ERR_INVALID_ARG;
  for (int k = 0; k < n_tau; ++k)
    if (!(tau[k] > 0.0) || !std::isfinite(tau[k]) || !std::isfinite(w[k])) return LTMP2_ERR_INVALID_ARG;
  // the same validation and tables as ltmp2_setup; the CUDA-core GEMM flag is implied here
  HostPlan hp;
  int rc = build_host_plan(sys, LTMP2_FLAG_REAL_ORBITALS, hp);
  if (rc) return rc;
  void *base = nullptr;
  if ((rc = scratch_base(&base))) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Arena ar(base, kNoAllocScratchBytes);
  Plan p = hp.p;
  std::vector<double> heps(sys->eps, sys->eps + sys->n_orb);
  auto put = [&](auto **dst, const auto &vec) -> int {
    using X = typename std::remove_reference<decltype(vec)>::type::value_type;
    void *q = ar.take(vec.size() * sizeof(X));
    if (!q) return LTMP2_ERR_UNSUPPORTED;
    *dst = reinterpret_cast<typename std::remove_reference<decltype(*dst)>::type>(q);
    return copy_in(q, vec.data(), vec.size() * sizeof(X), st);
  };
  if ((rc = put(&p.dorb, hp.dorb))) return rc;
  if ((rc = put(&p.dorb_off, hp.dorb_off))) return rc;
  if ((rc = put(&p.daux, hp.daux))) return rc;
  if ((rc = put(&p.daux_off, hp.daux_off))) return rc;
  if ((rc = put(&p.pw_m, hp.pw_m))) return rc;
  if (p.real_basis && (rc = put(&p.pw_pair, hp.pw_pair))) return rc;
  if ((rc = put(&p.aux_m, hp.aux_m))) return rc;
  if ((rc = put(&p.aux_neg, hp.aux_neg))) return rc;
  if ((rc = put(&p.prim, hp.prim))) return rc;
  if ((rc = put(&p.v_aux64, hp.v64))) return rc;
  if ((rc = put(&p.v_aux32, hp.v32))) return rc;
  if ((rc = put(&p.eps, heps))) return rc;
  return sys->precision == LTMP2_FP64
             ? run_noalloc<double>(sys, p, ar, hp.order, n_tau, tau, w, st, e_direct, e_exchange, e_pair)
             : run_noalloc<float>(sys, p, ar, hp.order, n_tau, tau, w, st, e_direct, e_exchange, e_pair);
}

}  // namespace

extern "C" int ltmp2_energy_noalloc(const ltmp2_system *sys, int n_tau, const double *tau, const double *w,
                                    double *e_direct, double *e_exchange, double *e_pair, void *stream) {
  // host-side containers may throw; nothing may cross the C boundary
  try {
    return energy_noalloc(sys, n_tau, tau, w, e_direct, e_exchange, e_pair, stream);
  } catch (const std::bad_alloc &) {
    return LTMP2_ERR_OOM;
  } catch (...) {
    return LTMP2_ERR_INVALID_ARG;
  }
}

// C ABI of the LTMP2 hot path: input validation, index tables, device memory,
// the tau / G'-slab driver loop and per-stage timing.  The arithmetic of the
// path runs in the kernels of kernels_f64.cu / kernels_f32.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <type_traits>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "../../include/ltmp2.h"
#include "fft.cuh"
#include "host_plan.h"
#include "plan.h"

using namespace ltmp2;

namespace {

struct EventTimer final : StageTimer {
  bool on = false;
  cudaStream_t stream = nullptr;
  std::vector<cudaEvent_t> pool;
  std::vector<std::tuple<int, cudaEvent_t, cudaEvent_t>> pending;
  std::vector<cudaEvent_t> open;  // begin events by stage
  double ms[LTMP2_NUM_STAGES] = {0};
  long long launches[LTMP2_NUM_STAGES] = {0};
  EventTimer() : open(LTMP2_NUM_STAGES, nullptr) {}
  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  void begin(int stage) override {
    if (!on) return;
    cudaEvent_t e = get();
    cudaEventRecord(e, stream);
    open[stage] = e;
  }
  void end(int stage) override {
    if (!on || !open[stage]) return;
    cudaEvent_t e = get();
    cudaEventRecord(e, stream);
    pending.emplace_back(stage, open[stage], e);
    open[stage] = nullptr;
  }
  void collect() {
    for (auto &t : pending) {
      float x = 0.f;
      cudaEventSynchronize(std::get<2>(t));
      if (cudaEventElapsedTime(&x, std::get<1>(t), std::get<2>(t)) == cudaSuccess) {
        ms[std::get<0>(t)] += x;
        launches[std::get<0>(t)] += 1;
      }
      pool.push_back(std::get<1>(t));
      pool.push_back(std::get<2>(t));
    }
    pending.clear();
  }
  ~EventTimer() override {
    for (auto e : pool) cudaEventDestroy(e);
    for (auto &t : pending) {
      cudaEventDestroy(std::get<1>(t));
      cudaEventDestroy(std::get<2>(t));
    }
  }
};

}  // namespace

struct ltmp2_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  Plan p;
  std::vector<void *> allocs;
  EventTimer timer;
  double last_imag[2] = {0, 0};
  int slab_capacity = 0;
  double lattice[9] = {0};
  long long kernel_launches = 0;
  unsigned char *d_keep = nullptr;   // screened-pair mask and kept lists (learned form)
  int *d_keep_list = nullptr, *d_keep_count = nullptr;
  TcResources tc;
  void *tc_mem = nullptr;   // operand buffers of the tensor-core GEMM (owned via allocs)
  OzResources oz;           // FP64 path: slices of the tensor-core FP64 GEMM (memory owned via allocs)
  double ecut_aux = 0.0;               // E_aux of A (Hartree)
  std::vector<double> aux_g2;          // |G|^2 of A in internal order
  // internal cutoff extrapolation: level cutoffs, |A_n| (G != 0), device buffers
  std::vector<double> lev_ecut;
  std::vector<int> lev_count;
  bool lev_alloc = false, lev_done = false;
  // spin-unrestricted pairing (this context as the alpha channel): opposite-spin scratch
  double *d_cross_y = nullptr, *d_cross_acc = nullptr, *d_cross_sum = nullptr;
  int cross_nb = 0;
  int *d_selftest_err = nullptr;   // error word of the failure-path self-test
  unsigned long long fingerprint = 0;  // hash of the set-up inputs (ltmp2_fingerprint)
  unsigned long long mask_hash = 0;    // hash of the pair mask, 0 = every pair kept
  void *k_cocc = nullptr;              // k-point context: occupied coefficients (owned via allocs)
  std::vector<double> eps_host;        // orbital energies, ascending (Gamma-point contexts)
  int virt_mode = LTMP2_VIRTUALS_AUTO; // ltmp2_set_virtual_cut
  double virt_log2 = 64.0;
  ~ltmp2_ctx() {
    tc_release(tc);
    oz_release(oz);
    for (void *q : allocs) cudaFree(q);
  }
};

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return LTMP2_OK;
  if (e == cudaErrorMemoryAllocation) return LTMP2_ERR_OOM;
  return LTMP2_ERR_CUDA;
}

template <typename X> int dalloc(ltmp2_ctx *c, X **ptr, size_t count) {
  void *q = nullptr;
  cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(X));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? LTMP2_ERR_OOM : LTMP2_ERR_CUDA;
  }
  c->allocs.push_back(q);
  *ptr = static_cast<X *>(q);
  return LTMP2_OK;
}

int dalloc_bytes(ltmp2_ctx *c, void **ptr, size_t bytes) {
  void *q = nullptr;
  cudaError_t e = cudaMalloc(&q, std::max<size_t>(bytes, 16));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? LTMP2_ERR_OOM : LTMP2_ERR_CUDA;
  }
  c->allocs.push_back(q);
  *ptr = q;
  return LTMP2_OK;
}

template <typename T> struct CT { T x, y; };

template <typename T>
int upload_coeff(ltmp2_ctx *c, const double *coeff, int n_pw, int row0, int rows,
                 const std::vector<int> &order, void **dst) {
  std::vector<CT<T>> h((size_t)rows * n_pw);
  for (int r = 0; r < rows; ++r)
    for (int q = 0; q < n_pw; ++q) {
      const double *src = coeff + ((size_t)(row0 + r) * n_pw + order[q]) * 2;
      h[(size_t)r * n_pw + q] = {(T)src[0], (T)src[1]};
    }
  int rc = dalloc_bytes(c, dst, h.size() * sizeof(CT<T>));
  if (rc) return rc;
  return cuda_status(cudaMemcpy(*dst, h.data(), h.size() * sizeof(CT<T>), cudaMemcpyHostToDevice));
}

// Real-basis coordinates of real orbitals (x(-G) = conj x(G)) in internal order: slot q
// of a primary G_q holds sqrt2 Re x(q), the slot of -G_q holds sqrt2 Im x(-G_q), and
// G = 0 holds Re x(0) (the unitary map U of the real-basis kernels).
template <typename T>
int upload_real_coeff(ltmp2_ctx *c, const ltmp2_system *sys, int row0, int rows, const std::vector<int> &order,
                      void **dst) {
  const int n_pw = sys->n_pw;
  const double r2 = 1.4142135623730950488016887242097;
  std::vector<T> h((size_t)rows * n_pw);
  for (int q = 0; q < n_pw; ++q) {
    const int o = order[q];
    const int *m = sys->miller + 3 * o;
    const int kind = (m[0] == 0 && m[1] == 0 && m[2] == 0)
                         ? 0
                         : ((m[0] != 0 ? m[0] > 0 : (m[1] != 0 ? m[1] > 0 : m[2] > 0)) ? 1 : 2);
    for (int r = 0; r < rows; ++r) {
      const double *src = sys->coeff + ((size_t)(row0 + r) * n_pw + o) * 2;
      h[(size_t)r * n_pw + q] = (T)(kind == 0 ? src[0] : (kind == 1 ? r2 * src[0] : r2 * src[1]));
    }
  }
  int rc = dalloc_bytes(c, dst, h.size() * sizeof(T));
  if (rc) return rc;
  return cuda_status(cudaMemcpy(*dst, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
}

// R_v^T [n_pw][n_v] in the real basis, for the transformed states through the virtual space
template <typename T>
int upload_real_coeff_t(ltmp2_ctx *c, const ltmp2_system *sys, const std::vector<int> &order, void **dst) {
  const int n_pw = sys->n_pw, no = sys->n_occ, nv = sys->n_orb - sys->n_occ;
  const double r2 = 1.4142135623730950488016887242097;
  std::vector<T> h((size_t)nv * n_pw);
  for (int q = 0; q < n_pw; ++q) {
    const int o = order[q];
    const int *m = sys->miller + 3 * o;
    const int kind = (m[0] == 0 && m[1] == 0 && m[2] == 0)
                         ? 0
                         : ((m[0] != 0 ? m[0] > 0 : (m[1] != 0 ? m[1] > 0 : m[2] > 0)) ? 1 : 2);
    for (int a = 0; a < nv; ++a) {
      const double *src = sys->coeff + ((size_t)(no + a) * n_pw + o) * 2;
      h[(size_t)q * nv + a] = (T)(kind == 0 ? src[0] : (kind == 1 ? r2 * src[0] : r2 * src[1]));
    }
  }
  int rc = dalloc_bytes(c, dst, h.size() * sizeof(T));
  if (rc) return rc;
  return cuda_status(cudaMemcpy(*dst, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
}

template <typename T> int setup_precision(ltmp2_ctx *c, const ltmp2_system *sys, const std::vector<int> &order) {
  Plan &p = c->p;
  cudaError_t e = Path<T>::init_device();
  if (e != cudaSuccess) return cuda_status(e);
  const size_t cs = sizeof(CT<T>);
  const size_t n3 = (size_t)p.n * p.n * p.n;
  int rc;
  if (p.real_basis) {
    if ((rc = upload_real_coeff<T>(c, sys, p.n_occ, p.n_v, order, &p.cv))) return rc;
  } else {
    if ((rc = upload_coeff<T>(c, sys->coeff, p.n_pw, p.n_occ, p.n_v, order, &p.cv))) return rc;
  }
  // CUDA-core GEMMs in the real basis: R_v^T as well, for the large-tau transformed states
  const bool simt = std::is_same<T, double>::value || (sys->flags & LTMP2_FLAG_SIMT_GEMM);
  if (p.real_basis && simt && p.n_v > 0 && (rc = upload_real_coeff_t<T>(c, sys, order, &p.rvt))) return rc;
  void *cocc = nullptr;
  if ((rc = upload_coeff<T>(c, sys->coeff, p.n_pw, 0, p.n_occ, order, &cocc))) return rc;
  if ((rc = dalloc_bytes(c, &p.cgrid, cs * n3 * p.n_occ))) return rc;
  if ((rc = dalloc_bytes(c, &p.u, cs * n3 * p.n_occ))) return rc;
  if ((rc = dalloc_bytes(c, &p.ut, cs * n3 * p.n_occ))) return rc;
  if (p.real_basis && (rc = dalloc_bytes(c, &p.utr, sizeof(T) * n3 * p.n_occ))) return rc;
  if ((rc = dalloc_bytes(c, &p.dscale, sizeof(T) * p.n_orb))) return rc;
  // real basis: one extra row, for the pair-interleaved Green's function of the tensor-core build
  if ((rc = dalloc_bytes(c, &p.pt, (p.real_basis ? sizeof(T) * (size_t)(p.n_pw + 1) : cs * (size_t)p.n_pw) * p.n_pw)))
    return rc;
  // slab capacity from the free memory
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  const int spp = p.slots_per_prim();
  const size_t cols_pp = (size_t)spp * p.n_occ;
  const size_t per_prim = cs * cols_pp * (2 * (size_t)p.n_pw + (size_t)p.n * p.n_dorb +
                                          (size_t)p.n_occ * p.n * p.n_daux) +
                          cs * spp * (size_t)p.n_aux * p.n_occ + 2 * sizeof(double2) * (size_t)p.n_occ * p.n_occ;
  size_t budget = std::min<size_t>(free_b / 3, (size_t)16 << 30);
  long long mp = (long long)(budget / std::max<size_t>(per_prim, 1));
  const long long by_cols = std::max<long long>(1, 4096 / (long long)cols_pp);
  mp = std::min<long long>(mp, by_cols);
  mp = std::min<long long>(mp, p.n_prim);
  if (mp < 1) mp = 1;
  p.max_prim = (int)mp;
  c->slab_capacity = p.max_prim;
  const size_t max_cols = cols_pp * p.max_prim;
  if ((rc = dalloc_bytes(c, &p.st, cs * max_cols * p.n_pw))) return rc;
  if ((rc = dalloc_bytes(c, &p.wt, cs * max_cols * p.n_pw))) return rc;
  if ((rc = dalloc_bytes(c, &p.z1, cs * std::max(max_cols, (size_t)p.n_occ) * p.n * p.n_dorb))) return rc;
  if ((rc = dalloc_bytes(c, &p.tbuf, cs * max_cols * p.n_occ * p.n * p.n_daux))) return rc;
  if ((rc = dalloc_bytes(c, &p.mdiag, cs * (size_t)spp * p.max_prim * p.n_aux * p.n_occ))) return rc;
  if ((rc = dalloc(c, &p.sx, (size_t)p.max_prim * p.n_occ * p.n_occ))) return rc;
  if ((rc = dalloc(c, &p.yd, (size_t)p.max_prim * p.n_occ * p.n_occ))) return rc;
  if (std::is_same<T, float>::value && !(sys->flags & LTMP2_FLAG_SIMT_GEMM)) {
    void *tcmem = nullptr;
    if ((rc = dalloc_bytes(c, &tcmem, tc_bytes((int)max_cols, p.n_pw)))) return rc;
    c->tc_mem = tcmem;
    e = tc_init(c->tc, tcmem, (int)max_cols, p.n_pw, 5, p.real_basis);
    if (e != cudaSuccess) return cuda_status(e);
    if (p.real_basis) {
      // the direct-term products on the tensor cores, one per primary G' of a slab (the
      // Green's function stays on the CUDA cores unless ltmp2_set_tuning asks otherwise)
      void *dmem = nullptr;
      if ((rc = dalloc_bytes(c, &dmem, tc_direct_bytes(p.n_occ, p.n_aux, p.max_prim)))) return rc;
      e = tc_direct_init(c->tc, dmem, p.n_occ, p.n_aux, p.max_prim);
      if (e != cudaSuccess) return cuda_status(e);
    }
    p.tc = &c->tc;
  }
  if (std::is_same<T, double>::value && p.real_basis && !(sys->flags & LTMP2_FLAG_SIMT_GEMM)) {
    // the transformed-state GEMM with FP64 accuracy on the tensor cores (exact integer slices)
    void *omem = nullptr;
    if ((rc = dalloc_bytes(c, &omem, oz_bytes((int)max_cols, p.n_pw, p.n_v)))) return rc;
    e = oz_init(c->oz, omem, (int)max_cols, p.n_pw, p.n_v);
    if (e == cudaSuccess) e = oz_split_cv(c->oz, (const double *)p.cv, c->stream);   // R_v, once
    if (e != cudaSuccess) return cuda_status(e);
    p.oz = &c->oz;
  }
  e = Path<T>::setup_occupied(p, cocc, c->stream);
  if (e != cudaSuccess) return cuda_status(e);
  e = cudaStreamSynchronize(c->stream);
  return cuda_status(e);
}

// k-point context: per-k virtual coefficients, composite occupied orbitals, per-k Green's
// functions, slab buffers (two slots per primary Q', N_k n_occ columns per slot)
template <typename T>
int setup_precision_k(ltmp2_ctx *c, const ltmp2_kpoint_system *sys, const std::vector<int> &order) {
  Plan &p = c->p;
  cudaError_t e = Path<T>::init_device();
  if (e != cudaSuccess) return cuda_status(e);
  const size_t cs = sizeof(CT<T>);
  const size_t n3 = (size_t)p.n * p.n * p.n;
  const int nk = p.nk, no = p.no_k, npw = p.n_pw, norb = p.n_orb;
  int rc;
  {
    std::vector<CT<T>> hv((size_t)nk * p.n_v * npw), ho((size_t)nk * no * npw);
    for (int k = 0; k < nk; ++k)
      for (int r = 0; r < norb; ++r)
        for (int q = 0; q < npw; ++q) {
          const double *src = sys->coeff + (((size_t)k * norb + r) * npw + order[q]) * 2;
          const CT<T> v = {(T)src[0], (T)src[1]};
          if (r < no) ho[((size_t)k * no + r) * npw + q] = v;
          else hv[((size_t)k * p.n_v + r - no) * npw + q] = v;
        }
    if ((rc = dalloc_bytes(c, &p.cv, hv.size() * cs))) return rc;
    if ((rc = cuda_status(cudaMemcpy(p.cv, hv.data(), hv.size() * cs, cudaMemcpyHostToDevice)))) return rc;
    void *cocc = nullptr;
    if ((rc = dalloc_bytes(c, &cocc, ho.size() * cs))) return rc;
    if ((rc = cuda_status(cudaMemcpy(cocc, ho.data(), ho.size() * cs, cudaMemcpyHostToDevice)))) return rc;
    c->k_cocc = cocc;
  }
  if ((rc = dalloc_bytes(c, &p.cgrid, cs * n3 * p.n_occ))) return rc;
  if ((rc = dalloc_bytes(c, &p.u, cs * n3 * p.n_occ))) return rc;
  if ((rc = dalloc_bytes(c, &p.ut, cs * n3 * p.n_occ))) return rc;
  if ((rc = dalloc_bytes(c, &p.dscale, sizeof(T) * (size_t)nk * norb))) return rc;
  if ((rc = dalloc_bytes(c, &p.pt, cs * (size_t)nk * npw * npw))) return rc;
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  const size_t cols_pp = 2 * (size_t)p.n_occ;
  const size_t per_prim = cs * cols_pp * (2 * (size_t)npw + (size_t)p.n * p.n_dorb + (size_t)p.n_occ * p.n * p.n_daux) +
                          cs * 2 * (size_t)p.n_aux * p.n_occ + 2 * sizeof(double2) * (size_t)p.n_occ * p.n_occ;
  const size_t budget = std::min<size_t>(free_b / 3, (size_t)16 << 30);
  long long mp = (long long)(budget / std::max<size_t>(per_prim, 1));
  mp = std::min<long long>(mp, std::max<long long>(1, 4096 / (long long)cols_pp));
  mp = std::min<long long>(mp, p.n_prim);
  if (mp < 1) mp = 1;
  p.max_prim = (int)mp;
  c->slab_capacity = p.max_prim;
  const size_t max_cols = cols_pp * p.max_prim;
  if ((rc = dalloc_bytes(c, &p.st, cs * max_cols * npw))) return rc;
  if ((rc = dalloc_bytes(c, &p.wt, cs * max_cols * npw))) return rc;
  if ((rc = dalloc_bytes(c, &p.z1, cs * std::max(max_cols, (size_t)p.n_occ) * p.n * p.n_dorb))) return rc;
  if ((rc = dalloc_bytes(c, &p.tbuf, cs * max_cols * p.n_occ * p.n * p.n_daux))) return rc;
  // positions of the diagonal co-densities outside a slot's sphere are never written: zero them once
  const size_t mbytes = cs * 2 * (size_t)p.max_prim * p.n_aux * p.n_occ;
  if ((rc = dalloc_bytes(c, &p.mdiag, mbytes))) return rc;
  if ((rc = cuda_status(cudaMemset(p.mdiag, 0, mbytes)))) return rc;
  if ((rc = dalloc(c, &p.sx, (size_t)p.max_prim * p.n_occ * p.n_occ))) return rc;
  if ((rc = dalloc(c, &p.yd, (size_t)p.max_prim * p.n_occ * p.n_occ))) return rc;
  e = Path<T>::setup_occupied(p, c->k_cocc, c->stream);
  if (e != cudaSuccess) return cuda_status(e);
  return cuda_status(cudaStreamSynchronize(c->stream));
}

// Launch (without waiting) everything one energy evaluation does on `stream`.  Usable
// inside stream capture: no allocation, copy or synchronisation happens here.
// Per tau (Eq. SCHLT's factor e^{-(e_a-mu)tau}): the virtuals whose weight is at least
// 2^-L of the LUMO's.  Energies ascend, so they are the first nv; the rest contribute
// below the rounding of an FP64 product over the kept ones and are left out.  W goes
// through the virtual space when its two products (4 n_pw nv multiply-adds per column)
// undercut the product with the Green's function (2 n_pw^2) by 10 %.
constexpr double kVirtualRouteRatio = 0.9;
int tau_virtuals(const ltmp2_ctx *c, double tau, bool *w_virtual) {
  const Plan &p = c->p;
  *w_virtual = false;
  if (c->virt_mode == LTMP2_VIRTUALS_ALL || p.nk > 0 || p.n_v < 1 || c->eps_host.size() != (size_t)p.n_orb)
    return p.n_v;
  const double *ev = c->eps_host.data() + p.n_occ;
  const double cut = ev[0] + c->virt_log2 * 0.69314718055994530942 / tau;
  const int nv = std::max(1, (int)(std::upper_bound(ev, ev + p.n_v, cut) - ev));
  if (p.rvt && p.route == 0 &&
      (c->virt_mode == LTMP2_VIRTUALS_SPACE || 2.0 * nv <= kVirtualRouteRatio * p.n_pw))
    *w_virtual = true;
  return nv;
}
void set_tau_virtuals(const ltmp2_ctx *c, Plan &p, double tau) {
  bool wv = false;
  p.nv_tau = tau_virtuals(c, tau, &wv);
  p.w_virtual = wv;
}
// back to every virtual and the Green's function when the tau loop ends
struct TauVirtualsReset {
  Plan &p;
  ~TauVirtualsReset() {
    p.nv_tau = 0;
    p.w_virtual = false;
  }
};

template <typename T>
int enqueue_energy(ltmp2_ctx *c, cudaStream_t stream, int n_tau, const double *tau, const double *w, int gp_begin,
                   int gp_end, StageTimer *tm, long long *launches) {
  Plan &p = c->p;
  TauVirtualsReset reset{p};
  cudaError_t e = Path<T>::zero_acc(p, stream);
  if (e != cudaSuccess) return cuda_status(e);
  *launches += Path<T>::frame_launches(p);  // zero + final reduction(s)
  const double nfft = (double)p.n * p.n * p.n;
  // k-point sampling: Omega = N_k Omega_0 (the Born-von Karman supercell), the unit-cell
  // transforms are 1/N_k of the supercell's, and the energy is per unit cell (one more 1/N_k)
  const double nk = p.nk > 0 ? (double)p.nk : 1.0;
  for (int k = 0; k < n_tau; ++k) {
    if (p.nk == 0) set_tau_virtuals(c, p, tau[k]);
    e = p.nk > 0 ? Path<T>::green_k(p, tau[k], stream, tm) : Path<T>::green(p, tau[k], stream, tm);
    if (e != cudaSuccess) return cuda_status(e);
    *launches += p.nk > 0 ? Path<T>::green_k_launches(p) : Path<T>::green_launches(p);
    const double coef = w[k] / (nk * nk * nk * p.omega * p.omega * nfft * nfft);
    for (int g0 = gp_begin; g0 < gp_end; g0 += p.max_prim) {
      const int np = std::min(p.max_prim, gp_end - g0);
      e = p.nk > 0 ? Path<T>::slab_k(p, g0, np, coef, stream, tm) : Path<T>::slab(p, g0, np, coef, stream, tm);
      if (e != cudaSuccess) return cuda_status(e);
      *launches += p.nk > 0 ? Path<T>::slab_k_launches(p) : Path<T>::slab_launches(p);
    }
  }
  e = Path<T>::finish(p, stream, tm);
  return cuda_status(e);
}

// After the work is complete: a bounded wait inside the tensor-core GEMM that ran out is
// reported (and the flag cleared).
int check_tc_flag(ltmp2_ctx *c) {
  if (c->p.oz) {
    const int rc = oz_check(c->oz);
    if (rc) return rc;
  }
  if (!c->p.tc) return LTMP2_OK;
  int flag = 0;
  cudaError_t e = cudaMemcpy(&flag, c->p.tc->err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_status(e);
  if (flag) {
    cudaMemset(c->p.tc->err, 0, sizeof(int));
    return LTMP2_ERR_TIMEOUT;
  }
  return LTMP2_OK;
}

template <typename T>
int run_energy(ltmp2_ctx *c, int n_tau, const double *tau, const double *w, int gp_begin, int gp_end) {
  StageTimer *tm = c->timer.on ? &c->timer : nullptr;
  c->timer.stream = c->stream;
  int rc = enqueue_energy<T>(c, c->stream, n_tau, tau, w, gp_begin, gp_end, tm, &c->kernel_launches);
  if (rc) return rc;
  c->lev_done = c->p.n_lev > 1;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (tm) c->timer.collect();
  if (e != cudaSuccess) return cuda_status(e);
  return check_tc_flag(c);
}

int check_tau(int n_tau, const double *tau, const double *w) {
  if (n_tau < 1 || !tau || !w) return LTMP2_ERR_INVALID_ARG;
  for (int k = 0; k < n_tau; ++k)
    if (!(tau[k] > 0.0) || !std::isfinite(tau[k]) || !std::isfinite(w[k])) return LTMP2_ERR_INVALID_ARG;
  return LTMP2_OK;
}

int energy_common(ltmp2_ctx *ctx, int n_tau, const double *tau, const double *w, int gp_begin, int gp_end,
                  double *e_d, double *e_x, std::vector<double> *ed_pair, std::vector<double> *ex_pair) {
  if (!ctx) return LTMP2_ERR_INVALID_ARG;
  int rc = check_tau(n_tau, tau, w);
  if (rc) return rc;
  if (gp_begin < 0 || gp_end > ctx->p.n_prim || gp_begin > gp_end) return LTMP2_ERR_INVALID_ARG;
  DeviceGuard g(ctx->device);
  rc = ctx->p.precision == LTMP2_FP64 ? run_energy<double>(ctx, n_tau, tau, w, gp_begin, gp_end)
                                      : run_energy<float>(ctx, n_tau, tau, w, gp_begin, gp_end);
  if (rc) return rc;
  double es[4];
  cudaError_t e = cudaMemcpy(es, ctx->p.esum, sizeof(es), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_status(e);
  const size_t no2 = (size_t)ctx->p.n_occ * ctx->p.n_occ;
  if (ed_pair) {
    ed_pair->resize(no2);
    e = cudaMemcpy(ed_pair->data(), ctx->p.ed, no2 * sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_status(e);
  }
  if (ex_pair) {
    ex_pair->resize(no2);
    e = cudaMemcpy(ex_pair->data(), ctx->p.ex, no2 * sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_status(e);
  }
  ctx->last_imag[0] = es[2];
  ctx->last_imag[1] = es[3];
  if (e_d) *e_d = es[0];
  if (e_x) *e_x = es[1];
  return LTMP2_OK;
}


// ---------------------------------------------------------------- autotuner
// Slab size (primary G' per pass) and tensor-core GEMM variant, chosen by timing one
// slab per candidate; cached per (grid, N_pw, N_occ, |A|, precision, real) bucket.
struct TuneKey {
  int n, n_pw, n_occ, n_aux, precision, real;
  bool operator<(const TuneKey &o) const {
    return std::tie(n, n_pw, n_occ, n_aux, precision, real) <
           std::tie(o.n, o.n_pw, o.n_occ, o.n_aux, o.precision, o.real);
  }
};
std::mutex g_tune_mutex;
struct TuneVal {
  int slab, variant, plane_kernel, plane_ib;
};
std::map<TuneKey, TuneVal> g_tune_cache;

int apply_tuning(ltmp2_ctx *c, int slab, int variant, int plane_kernel, int plane_ib) {
  if (slab < 1 || slab > c->slab_capacity) return LTMP2_ERR_INVALID_ARG;
  c->p.max_prim = slab;
  c->p.plane_kernel = plane_kernel;
  c->p.plane_ib = plane_ib;
  if (c->p.tc && variant >= 0 && variant != c->tc.variant) {
    tc_release(c->tc);
    cudaError_t e = tc_init(c->tc, c->tc_mem, c->tc.rows_cap, c->p.n_pw, variant, c->tc.real);
    if (e != cudaSuccess) return cuda_status(e);
  }
  return LTMP2_OK;
}

template <typename T> int tune_ctx(ltmp2_ctx *c, int *slab_out, int *var_out) {
  Plan &p = c->p;
  const TuneKey key{p.n, p.n_pw, p.n_occ, p.n_aux, p.precision, p.real_orb ? 1 : 0};
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      const TuneVal &v = it->second;
      int rc = apply_tuning(c, std::min(v.slab, c->slab_capacity), v.variant, v.plane_kernel, v.plane_ib);
      *slab_out = p.max_prim;
      *var_out = p.tc ? c->tc.variant : -1;
      return rc;
    }
  }
  std::vector<int> slabs;
  for (int sl = std::min(c->slab_capacity, p.n_prim); sl >= 1 && slabs.size() < 4; sl /= 2) slabs.push_back(sl);
  std::vector<int> variants =
      p.tc ? (c->tc.real ? std::vector<int>{5} : std::vector<int>{5, 4}) : std::vector<int>{-1};
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return LTMP2_ERR_CUDA;
  double best = 1e300;
  int best_slab = slabs.front(), best_var = variants.front();
  int rc = LTMP2_OK;
  for (int v : variants) {
    if ((rc = apply_tuning(c, slabs.front(), v, p.plane_kernel, p.plane_ib))) break;
    if (Path<T>::green(p, 1.0, c->stream, nullptr) != cudaSuccess) { rc = LTMP2_ERR_CUDA; break; }
    for (int sl : slabs) {
      p.max_prim = sl;
      // one untimed pass, then two timed ones (weight 0: accumulators unchanged)
      for (int rep = 0; rep < 3 && !rc; ++rep) {
        if (rep == 1) cudaEventRecord(a, c->stream);
        if (Path<T>::slab(p, 0, sl, 0.0, c->stream, nullptr) != cudaSuccess) rc = LTMP2_ERR_CUDA;
      }
      if (rc) break;
      cudaEventRecord(b, c->stream);
      if (cudaEventSynchronize(b) != cudaSuccess) { rc = LTMP2_ERR_CUDA; break; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, a, b);
      const double per_prim = ms / (2.0 * sl);
      if (per_prim < best) { best = per_prim; best_slab = sl; best_var = v; }
    }
    if (rc) break;
  }
  // plane kernel and its block size, timed alone on the columns of one warm slab
  int best_pk = 0, best_ib = 0;
  if (!rc) rc = apply_tuning(c, best_slab, best_var, p.plane_kernel, p.plane_ib);
  if (!rc && Path<T>::slab(p, 0, best_slab, 0.0, c->stream, nullptr) != cudaSuccess) rc = LTMP2_ERR_CUDA;
  if (!rc) {
    const int ncols = best_slab * p.slots_per_prim() * p.n_occ;
    double best_plane = 1e300;
    static const int kIbs[2][4] = {{2, 4, 8, 16}, {1, 2, 3, 4}};   // planes per block; kernel 3: per warp step
    for (int pk = 0; pk < 4 && !rc; ++pk)
      for (int ibk = 0; ibk < 4; ++ibk) {
        const int ib = kIbs[pk == 3 ? 1 : 0][ibk];
        if (ib > p.n_occ) continue;
        if (Path<T>::plane_pass(p, ncols, pk, ib, c->stream) != cudaSuccess) {  // infeasible shape
          cudaGetLastError();
          continue;
        }
        cudaEventRecord(a, c->stream);
        for (int rep = 0; rep < 2; ++rep) Path<T>::plane_pass(p, ncols, pk, ib, c->stream);
        cudaEventRecord(b, c->stream);
        if (cudaEventSynchronize(b) != cudaSuccess) { rc = LTMP2_ERR_CUDA; break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (ms < best_plane) { best_plane = ms; best_pk = pk; best_ib = ib; }
      }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (!rc) rc = check_tc_flag(c);
  if (!rc) rc = apply_tuning(c, best_slab, best_var, best_pk, best_ib);
  if (rc) return rc;
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache[key] = {best_slab, best_var, best_pk, best_ib};
  }
  *slab_out = best_slab;
  *var_out = p.tc ? best_var : -1;
  return LTMP2_OK;
}

}  // namespace

// ---------------------------------------------------------------- batching form
// Every system's whole evaluation (all tau, all slabs) captured into one CUDA graph: one
// branch per system on its own forked stream, joined at the end.  A run is one graph
// launch; the graph is replayed by ltmp2_batch_run.
struct ltmp2_batch {
  int device = 0;
  bool persistent = false;        // shared persistent FFT stages per round (else one branch per system)
  void *d_plans = nullptr;        // persistent mode: the systems' plans on the device
  int *d_counters = nullptr;      // persistent mode: the two work-queue counters
  std::vector<ltmp2_ctx *> ctxs;
  std::vector<long long> launches;
  cudaStream_t origin = nullptr;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> events;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  ~ltmp2_batch() {
    cudaFree(d_plans);
    cudaFree(d_counters);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    for (auto e : events) cudaEventDestroy(e);
    for (auto st : streams) cudaStreamDestroy(st);
    if (origin) cudaStreamDestroy(origin);
  }
};

namespace {
}  // namespace

namespace {
// descriptors of every unordered occupied pair (see ltmp2_pair_descriptors)
int pair_descriptors(ltmp2_ctx *ctx, double *desc) {
  if (!ctx || !desc) return LTMP2_ERR_INVALID_ARG;
  Plan &p = ctx->p;
  const int no = p.n_occ;
  DeviceGuard g(ctx->device);
  double *dmom = nullptr, *dov = nullptr;
  if (cudaMalloc(&dmom, sizeof(double) * 6 * no) != cudaSuccess ||
      cudaMalloc(&dov, sizeof(double) * (size_t)no * no) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(dmom);
    return LTMP2_ERR_OOM;
  }
  cudaError_t e = p.precision == LTMP2_FP64 ? Path<double>::descriptors(p, dmom, dov, ctx->stream)
                                            : Path<float>::descriptors(p, dmom, dov, ctx->stream);
  std::vector<double> mom(6 * (size_t)no), ov((size_t)no * no), eps(p.n_orb);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpy(mom.data(), dmom, sizeof(double) * mom.size(), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(ov.data(), dov, sizeof(double) * ov.size(), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(eps.data(), p.eps, sizeof(double) * eps.size(), cudaMemcpyDeviceToHost);
  cudaFree(dmom);
  cudaFree(dov);
  if (e != cudaSuccess) return cuda_status(e);
  // periodic centroid (fractional) and spread (bohr) of each occupied density
  const double tp = 6.283185307179586476925286766559;
  std::vector<double> frac(3 * (size_t)no), spread(no);
  for (int i = 0; i < no; ++i) {
    double s2 = 0;
    for (int k = 0; k < 3; ++k) {
      const double re = mom[6 * i + 2 * k], im = mom[6 * i + 2 * k + 1];
      double f = std::atan2(im, re) / tp;
      frac[3 * i + k] = f - std::floor(f);
      const double mag = std::max(std::sqrt(re * re + im * im), 1e-12);
      const double sig = std::sqrt(-2.0 * std::log(std::min(mag, 1.0))) / tp;   // fractional units
      const double alen = std::sqrt(ctx->lattice[3 * k] * ctx->lattice[3 * k] + ctx->lattice[3 * k + 1] * ctx->lattice[3 * k + 1] +
                                    ctx->lattice[3 * k + 2] * ctx->lattice[3 * k + 2]);
      s2 += (sig * alen) * (sig * alen);
    }
    spread[i] = std::sqrt(s2);
  }
  size_t row = 0;
  for (int i = 0; i < no; ++i)
    for (int j = i; j < no; ++j, ++row) {
      double r[3] = {0, 0, 0};
      for (int k = 0; k < 3; ++k) {
        double df = frac[3 * i + k] - frac[3 * j + k];
        df -= std::floor(df + 0.5);
        for (int c = 0; c < 3; ++c) r[c] += df * ctx->lattice[3 * k + c];
      }
      const double dist = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
      double *f = desc + row * LTMP2_NUM_DESC;
      f[0] = eps[i] - p.mu;
      f[1] = eps[j] - p.mu;
      f[2] = std::log10(std::max(ov[(size_t)i * no + j], 1e-300) /
                        std::sqrt(std::max(ov[(size_t)i * no + i] * ov[(size_t)j * no + j], 1e-300)));
      f[3] = dist;
      f[4] = spread[i];
      f[5] = spread[j];
      f[6] = (i == j) ? 1.0 : 0.0;
      f[7] = dist / (spread[i] + spread[j] + 1e-3);
    }
  return LTMP2_OK;
}
}  // namespace

// Batching form, persistent mode: rounds of (tau, slab) across the systems; per round each
// active system's pre-FFT phase on its own branch, then one persistent plane launch and one
// persistent column launch over the items of every active system, then each system's direct
// term and accumulation.  Captured on b->origin.
namespace {
template <typename T>
int capture_rounds(ltmp2_batch *b, ltmp2_ctx *const *ctxs, int n, const int *n_tau, const double *const *tau,
                   const double *const *w) {
  std::vector<Plan> plans(n);
  std::vector<int> ib(n), nslab(n), rounds(n);
  size_t smem_p = 0, smem_c = 0;
  int rmax = 0;
  for (int i = 0; i < n; ++i) {
    const Plan &p = ctxs[i]->p;
    plans[i] = p;
    ib[i] = std::max(1, std::min(kPersistThreads / p.n, p.n_occ));
    smem_p = std::max(smem_p, Path<T>::plane_smem_for(p, ib[i]));
    smem_c = std::max(smem_c, (size_t)p.n_aux * sizeof(CT<T>));
    nslab[i] = (p.n_prim + p.max_prim - 1) / p.max_prim;
    rounds[i] = n_tau[i] * nslab[i];
    rmax = std::max(rmax, rounds[i]);
  }
  if (smem_p > 200 * 1024 || smem_c > 200 * 1024) return LTMP2_ERR_UNSUPPORTED;
  if (cudaMalloc(&b->d_plans, sizeof(Plan) * n) != cudaSuccess || cudaMalloc(&b->d_counters, 2 * sizeof(int)) != cudaSuccess)
    return LTMP2_ERR_OOM;
  int rc = cuda_status(cudaMemcpy(b->d_plans, plans.data(), sizeof(Plan) * n, cudaMemcpyHostToDevice));
  if (!rc) rc = cuda_status(Path<T>::persist_attributes(smem_p, smem_c));
  const int blocks_p = Path<T>::persist_blocks(true, smem_p), blocks_c = Path<T>::persist_blocks(false, smem_c);
  if (!rc && (blocks_p < 1 || blocks_c < 1)) rc = LTMP2_ERR_CUDA;
  if (rc) return rc;
  const Plan *dp = static_cast<const Plan *>(b->d_plans);
  if (cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return LTMP2_ERR_CUDA;
  rc = cuda_status(cudaEventRecord(b->events[n], b->origin));
  for (int i = 0; i < n && !rc; ++i) {
    rc = cuda_status(cudaStreamWaitEvent(b->streams[i], b->events[n], 0));
    if (!rc) rc = cuda_status(Path<T>::zero_acc(ctxs[i]->p, b->streams[i]));
    b->launches[i] += 1;
  }
  long long shared = 0;
  for (int r = 0; r < rmax && !rc; ++r) {
    BatchRound rp, rcol;
    std::vector<int> act, gp0(n), np(n);
    for (int i = 0; i < n; ++i)
      if (r < rounds[i]) act.push_back(i);
    for (int i : act) {
      const Plan &p = ctxs[i]->p;
      const int k = r / nslab[i], j = r % nslab[i];
      gp0[i] = j * p.max_prim;
      np[i] = std::min(p.max_prim, p.n_prim - gp0[i]);
      if (j == 0) {
        if ((rc = cuda_status(Path<T>::green(p, tau[i][k], b->streams[i], nullptr)))) break;
        b->launches[i] += Path<T>::green_launches(p);
      }
      if ((rc = cuda_status(Path<T>::slab_pre(p, gp0[i], np[i], b->streams[i], nullptr)))) break;
      const int post = 2 + (p.tc && p.tc->direct ? 2 : 0);                       // direct term(s) + accumulation
      b->launches[i] += Path<T>::slab_launches(p) - 2 - post;                    // all but plane, column and post
      if ((rc = cuda_status(cudaEventRecord(b->events[i], b->streams[i])))) break;
      if ((rc = cuda_status(cudaStreamWaitEvent(b->origin, b->events[i], 0)))) break;
    }
    if (rc) break;
    rp.nsys = rcol.nsys = (int)act.size();
    for (int e = 0; e < rp.nsys; ++e) {
      const int i = act[e];
      const Plan &p = ctxs[i]->p;
      const int ncols = np[i] * p.slots_per_prim() * p.n_occ;
      const int npairs = p.real_orb ? np[i] * (p.n_occ * (p.n_occ + 1) / 2) : np[i] * p.n_occ * p.n_occ;
      rp.sys[e] = rcol.sys[e] = i;
      rp.gp0[e] = rcol.gp0[e] = gp0[i];
      rp.np[e] = rcol.np[e] = np[i];
      rp.ib[e] = rcol.ib[e] = ib[i];
      rp.first[e + 1] = rp.first[e] + p.n * ncols;
      rcol.first[e + 1] = rcol.first[e] + npairs;
    }
    if ((rc = cuda_status(Path<T>::planes_persist(dp, rp, b->d_counters, blocks_p, smem_p, b->origin)))) break;
    if ((rc = cuda_status(Path<T>::zcol_persist(dp, rcol, b->d_counters + 1, blocks_c, smem_c, b->origin)))) break;
    shared += 2;
    if ((rc = cuda_status(cudaEventRecord(b->events[n], b->origin)))) break;
    for (int i : act) {
      const Plan &p = ctxs[i]->p;
      const int k = r / nslab[i];
      const double nfft = (double)p.n * p.n * p.n;
      const double coef = w[i][k] / (p.omega * p.omega * nfft * nfft);
      if ((rc = cuda_status(cudaStreamWaitEvent(b->streams[i], b->events[n], 0)))) break;
      if ((rc = cuda_status(Path<T>::slab_post(p, gp0[i], np[i], coef, b->streams[i], nullptr)))) break;
      b->launches[i] += 2 + (p.tc && p.tc->direct_on() ? 2 : 0);
      if (r == rounds[i] - 1) {
        if ((rc = cuda_status(Path<T>::finish(p, b->streams[i], nullptr)))) break;
        b->launches[i] += 1;
      }
    }
  }
  for (int i = 0; i < n && !rc; ++i) {
    rc = cuda_status(cudaEventRecord(b->events[i], b->streams[i]));
    if (!rc) rc = cuda_status(cudaStreamWaitEvent(b->origin, b->events[i], 0));
  }
  b->launches[0] += shared;
  const cudaError_t ec = cudaStreamEndCapture(b->origin, &b->graph);
  if (rc) return rc;
  return cuda_status(ec);
}
}  // namespace

// spin-unrestricted form: both channels on the alpha context's stream
namespace {
template <typename T>
int enqueue_uhf(ltmp2_ctx *a, ltmp2_ctx *b, int n_tau, const double *tau, const double *w, long long *launches) {
  Plan &pa = a->p, &pb = b->p;
  TauVirtualsReset ra{pa}, rb{pb};
  cudaStream_t st = a->stream;
  cudaError_t e;
  if ((e = Path<T>::zero_acc(pa, st)) != cudaSuccess || (e = Path<T>::zero_acc(pb, st)) != cudaSuccess)
    return cuda_status(e);
  if ((e = cudaMemsetAsync(a->d_cross_acc, 0, sizeof(double) * pa.n_occ * pb.n_occ, st)) != cudaSuccess)
    return cuda_status(e);
  *launches += 2;
  const double nfft = (double)pa.n * pa.n * pa.n;
  for (int k = 0; k < n_tau; ++k) {
    set_tau_virtuals(a, pa, tau[k]);
    set_tau_virtuals(b, pb, tau[k]);
    if ((e = Path<T>::green(pa, tau[k], st, nullptr)) != cudaSuccess) return cuda_status(e);
    if ((e = Path<T>::green(pb, tau[k], st, nullptr)) != cudaSuccess) return cuda_status(e);
    *launches += Path<T>::green_launches(pa) + Path<T>::green_launches(pb);
    const double coef = w[k] / (pa.omega * pa.omega * nfft * nfft);
    for (int g0 = 0; g0 < pa.n_prim; g0 += pa.max_prim) {
      const int np = std::min(pa.max_prim, pa.n_prim - g0);
      // each channel: its exchange and same-spin direct sums, and its diagonal co-densities
      if ((e = Path<T>::slab(pa, g0, np, coef, st, nullptr)) != cudaSuccess) return cuda_status(e);
      if ((e = Path<T>::slab(pb, g0, np, coef, st, nullptr)) != cudaSuccess) return cuda_status(e);
      if ((e = Path<T>::direct_cross(pa, pb, g0, np, coef, a->d_cross_y, a->d_cross_acc, st)) != cudaSuccess)
        return cuda_status(e);
      *launches += Path<T>::slab_launches(pa) + Path<T>::slab_launches(pb) + 2;
    }
  }
  if ((e = Path<T>::finish(pa, st, nullptr)) != cudaSuccess || (e = Path<T>::finish(pb, st, nullptr)) != cudaSuccess)
    return cuda_status(e);
  if ((e = Path<T>::sum(pa.n_occ * pb.n_occ, a->d_cross_acc, a->d_cross_sum, st)) != cudaSuccess)
    return cuda_status(e);
  *launches += 3;
  return LTMP2_OK;
}
}  // namespace

extern "C" {

const char *ltmp2_strerror(int code) {
  switch (code) {
    case LTMP2_OK: return "success";
    case LTMP2_ERR_INVALID_ARG: return "invalid argument";
    case LTMP2_ERR_GAP: return "HOMO-LUMO gap below 1e-6 Ha";
    case LTMP2_ERR_NOT_ORTHONORMAL: return "orbitals are not orthonormal";
    case LTMP2_ERR_GRID: return "unsupported FFT grid or plane-wave set";
    case LTMP2_ERR_OOM: return "device memory exhausted";
    case LTMP2_ERR_CUDA: return "CUDA error";
    case LTMP2_ERR_TIMEOUT: return "device wait timed out";
    case LTMP2_ERR_UNSUPPORTED: return "unsupported option";
    case LTMP2_ERR_NO_CONVERGENCE: return "Laplace grid fit did not converge";
    case LTMP2_ERR_NOT_REAL: return "orbitals are not real in real space";
    default: return "unknown status";
  }
}

int ltmp2_setup(const ltmp2_system *sys, ltmp2_ctx **out) {
  if (!sys || !out) return LTMP2_ERR_INVALID_ARG;
  *out = nullptr;
  try {
  HostPlan hp;
  int rc = build_host_plan(sys, LTMP2_FLAG_REAL_ORBITALS | LTMP2_FLAG_SIMT_GEMM, hp);
  if (rc) return rc;
  const int no = sys->n_occ;
  std::unique_ptr<ltmp2_ctx> owner(new (std::nothrow) ltmp2_ctx());
  ltmp2_ctx *c = owner.get();
  if (!c) return LTMP2_ERR_OOM;
  if (cudaGetDevice(&c->device) != cudaSuccess) {
    cudaGetLastError();
    return LTMP2_ERR_CUDA;
  }
  Plan &p = c->p;
  p = hp.p;
  // plane kernel: FP32, the warp-autonomous one (fastest on the 24^3 and 36^3 workloads);
  // FP64, the block-synchronous one (FP64-issue bound either way, and 17 % faster)
  p.plane_kernel = sys->precision == LTMP2_FP32 ? 3 : 2;
  std::memcpy(c->lattice, sys->lattice, sizeof(c->lattice));
  c->ecut_aux = hp.ecut_aux;
  c->aux_g2 = hp.aux_g2;
  c->fingerprint = hp.fingerprint;
  const std::vector<int> &order = hp.order;
  auto up = [&](auto **dptr, const auto &vec) -> int {
    using X = typename std::remove_reference<decltype(vec)>::type::value_type;
    int r = dalloc(c, dptr, vec.size());
    if (r) return r;
    return cuda_status(cudaMemcpy(*dptr, vec.data(), vec.size() * sizeof(X), cudaMemcpyHostToDevice));
  };
  std::vector<double> heps(sys->eps, sys->eps + sys->n_orb);
  c->eps_host = heps;
  if (!rc) rc = up(&p.dorb, hp.dorb);
  if (!rc) rc = up(&p.dorb_off, hp.dorb_off);
  if (!rc) rc = up(&p.daux, hp.daux);
  if (!rc) rc = up(&p.daux_off, hp.daux_off);
  if (!rc) rc = up(&p.pw_m, hp.pw_m);
  if (!rc && p.real_basis) rc = up(&p.pw_pair, hp.pw_pair);   // internal position of -G_q
  if (!rc) rc = up(&p.aux_m, hp.aux_m);
  if (!rc) rc = up(&p.aux_neg, hp.aux_neg);
  if (!rc) rc = up(&p.prim, hp.prim);
  if (!rc) rc = up(&p.v_aux64, hp.v64);
  if (!rc) rc = up(&p.v_aux32, hp.v32);
  if (!rc) rc = up(&p.eps, heps);
  const size_t no2 = (size_t)no * no;
  if (!rc) rc = dalloc(c, &p.ex, no2);
  if (!rc) rc = dalloc(c, &p.ed, no2);
  if (!rc) rc = dalloc(c, &p.exi, no2);
  if (!rc) rc = dalloc(c, &p.edi, no2);
  if (!rc) rc = dalloc(c, &p.esum, 4);
  if (!rc)
    rc = (sys->precision == LTMP2_FP64) ? setup_precision<double>(c, sys, order)
                                        : setup_precision<float>(c, sys, order);
  if (rc) {
    cudaGetLastError();
    return rc;
  }
  *out = owner.release();
  return LTMP2_OK;
  } catch (const std::bad_alloc &) {
    return LTMP2_ERR_OOM;
  } catch (...) {
    return LTMP2_ERR_INVALID_ARG;
  }
}

int ltmp2_setup_kpoints(const ltmp2_kpoint_system *sys, ltmp2_ctx **out) {
  if (!sys || !out) return LTMP2_ERR_INVALID_ARG;
  *out = nullptr;
  try {
    HostPlan hp;
    KPointHost kh;
    int rc = build_kpoint_host_plan(sys, hp, kh);
    if (rc) return rc;
    std::unique_ptr<ltmp2_ctx> owner(new (std::nothrow) ltmp2_ctx());
    ltmp2_ctx *c = owner.get();
    if (!c) return LTMP2_ERR_OOM;
    if (cudaGetDevice(&c->device) != cudaSuccess) {
      cudaGetLastError();
      return LTMP2_ERR_CUDA;
    }
    Plan &p = c->p;
    p = hp.p;
    std::memcpy(c->lattice, sys->lattice, sizeof(c->lattice));
    c->ecut_aux = hp.ecut_aux;
    c->fingerprint = hp.fingerprint;
    auto up = [&](auto **dptr, const auto &vec) -> int {
      using X = typename std::remove_reference<decltype(vec)>::type::value_type;
      int r = dalloc(c, dptr, vec.size());
      if (r) return r;
      return cuda_status(cudaMemcpy(*dptr, vec.data(), vec.size() * sizeof(X), cudaMemcpyHostToDevice));
    };
    std::vector<double> heps(sys->eps, sys->eps + (size_t)p.nk * p.n_orb);
    int *d_prim = nullptr, *d_lut = nullptr;
    double *d_vprim = nullptr, *d_vc64 = nullptr, *d_eps = nullptr;
    float *d_vc32 = nullptr;
    if (!rc) rc = up(&p.dorb, hp.dorb);
    if (!rc) rc = up(&p.dorb_off, hp.dorb_off);
    if (!rc) rc = up(&p.daux, hp.daux);
    if (!rc) rc = up(&p.daux_off, hp.daux_off);
    if (!rc) rc = up(&p.pw_m, hp.pw_m);
    if (!rc) rc = up(&p.aux_m, hp.aux_m);
    if (!rc) rc = up(&d_prim, kh.prim_m);
    if (!rc) rc = up(&d_vprim, kh.vprim);
    if (!rc) rc = up(&d_vc64, kh.vcls64);
    if (!rc) rc = up(&d_vc32, kh.vcls32);
    if (!rc) rc = up(&d_lut, kh.lut);
    if (!rc) rc = up(&d_eps, heps);
    p.prim_m = d_prim;
    p.vprim = d_vprim;
    p.vcls64 = d_vc64;
    p.vcls32 = d_vc32;
    p.lut = d_lut;
    p.eps = d_eps;
    const size_t no2 = (size_t)p.n_occ * p.n_occ;
    if (!rc) rc = dalloc(c, &p.ex, no2);
    if (!rc) rc = dalloc(c, &p.ed, no2);
    if (!rc) rc = dalloc(c, &p.exi, no2);
    if (!rc) rc = dalloc(c, &p.edi, no2);
    if (!rc) rc = dalloc(c, &p.esum, 4);
    if (!rc)
      rc = (sys->precision == LTMP2_FP64) ? setup_precision_k<double>(c, sys, hp.order)
                                          : setup_precision_k<float>(c, sys, hp.order);
    if (rc) {
      cudaGetLastError();
      return rc;
    }
    *out = owner.release();
    return LTMP2_OK;
  } catch (const std::bad_alloc &) {
    return LTMP2_ERR_OOM;
  } catch (...) {
    return LTMP2_ERR_INVALID_ARG;
  }
}

int ltmp2_set_stream(ltmp2_ctx *ctx, void *stream) {
  if (!ctx) return LTMP2_ERR_INVALID_ARG;
  ctx->stream = static_cast<cudaStream_t>(stream);
  return LTMP2_OK;
}

int ltmp2_energy(ltmp2_ctx *ctx, int n_tau, const double *tau, const double *w, double *e_direct,
                 double *e_exchange, double *e_pair) {
  if (!ctx || !e_direct || !e_exchange) return LTMP2_ERR_INVALID_ARG;
  std::vector<double> ed, ex;
  int rc = energy_common(ctx, n_tau, tau, w, 0, ctx->p.n_prim, e_direct, e_exchange, e_pair ? &ed : nullptr,
                         e_pair ? &ex : nullptr);
  if (rc) return rc;
  if (e_pair)
    for (size_t k = 0; k < ed.size(); ++k) e_pair[k] = ed[k] + ex[k];
  return LTMP2_OK;
}

int ltmp2_energy_partial(ltmp2_ctx *ctx, int n_tau, const double *tau, const double *w, int gp_begin,
                         int gp_end, double *e_direct, double *e_exchange, double *e_pair_direct,
                         double *e_pair_exchange) {
  if (!ctx || !e_direct || !e_exchange) return LTMP2_ERR_INVALID_ARG;
  std::vector<double> ed, ex;
  int rc = energy_common(ctx, n_tau, tau, w, gp_begin, gp_end, e_direct, e_exchange,
                         e_pair_direct ? &ed : nullptr, e_pair_exchange ? &ex : nullptr);
  if (rc) return rc;
  if (e_pair_direct) std::memcpy(e_pair_direct, ed.data(), ed.size() * sizeof(double));
  if (e_pair_exchange) std::memcpy(e_pair_exchange, ex.data(), ex.size() * sizeof(double));
  return LTMP2_OK;
}

int ltmp2_set_slab_size(ltmp2_ctx *ctx, int n) {
  if (!ctx) return LTMP2_ERR_INVALID_ARG;
  if (n > ctx->slab_capacity) return LTMP2_ERR_INVALID_ARG;
  ctx->p.max_prim = (n <= 0) ? ctx->slab_capacity : n;
  return ctx->p.max_prim;
}

int ltmp2_num_primary_gprime(const ltmp2_ctx *ctx) { return ctx ? ctx->p.n_prim : LTMP2_ERR_INVALID_ARG; }

int ltmp2_sizes(const ltmp2_ctx *ctx, int *n_aux, int *n_pw, int *n_occ, int *grid_n) {
  if (!ctx) return LTMP2_ERR_INVALID_ARG;
  if (n_aux) *n_aux = ctx->p.n_aux - 1;  // the internal table carries G = 0 with v = 0
  if (n_pw) *n_pw = ctx->p.n_pw;
  if (n_occ) *n_occ = ctx->p.n_occ;
  if (grid_n) *grid_n = ctx->p.n;
  return LTMP2_OK;
}

int ltmp2_last_imag(const ltmp2_ctx *ctx, double *im_direct, double *im_exchange) {
  if (!ctx) return LTMP2_ERR_INVALID_ARG;
  if (im_direct) *im_direct = ctx->last_imag[0];
  if (im_exchange) *im_exchange = ctx->last_imag[1];
  return LTMP2_OK;
}

int ltmp2_kernel_launches(const ltmp2_ctx *ctx, long long *count) {
  if (!ctx || !count) return LTMP2_ERR_INVALID_ARG;
  *count = ctx->kernel_launches;
  return LTMP2_OK;
}

int ltmp2_fingerprint(const ltmp2_ctx *ctx, unsigned long long *out) {
  if (!ctx || !out) return LTMP2_ERR_INVALID_ARG;
  unsigned long long h = ctx->fingerprint;
  if (ctx->mask_hash) h = (h ^ ctx->mask_hash) * 0xff51afd7ed558ccdull;
  *out = h;
  return LTMP2_OK;
}

int ltmp2_sum_partials(int n, int n_occ, const double *e, const double *pd, const double *px, double *e_out,
                       double *pd_out, double *px_out) {
  if (n < 0 || n_occ < 1 || (n > 0 && !e) || !e_out) return LTMP2_ERR_INVALID_ARG;
  if ((pd_out && n > 0 && !pd) || (px_out && n > 0 && !px)) return LTMP2_ERR_INVALID_ARG;
  const size_t no2 = (size_t)n_occ * n_occ;
  double ed = 0.0, ex = 0.0;
  for (int c = 0; c < n; ++c) {
    ed += e[2 * c];
    ex += e[2 * c + 1];
  }
  if (!std::isfinite(ed) || !std::isfinite(ex)) return LTMP2_ERR_INVALID_ARG;
  for (int q = 0; q < 2; ++q) {
    double *out = q == 0 ? pd_out : px_out;
    const double *in = q == 0 ? pd : px;
    if (!out) continue;
    for (size_t k = 0; k < no2; ++k) {
      double s = 0.0;
      for (int c = 0; c < n; ++c) s += in[(size_t)c * no2 + k];
      out[k] = s;
    }
  }
  e_out[0] = ed;
  e_out[1] = ex;
  return LTMP2_OK;
}

int ltmp2_set_profiling(ltmp2_ctx *ctx, int on) {
  if (!ctx) return LTMP2_ERR_INVALID_ARG;
  ctx->timer.on = (on != 0);
  return LTMP2_OK;
}

int ltmp2_stage_times(const ltmp2_ctx *ctx, int n, double *ms, long long *launches) {
  if (!ctx || n < 0) return LTMP2_ERR_INVALID_ARG;
  for (int s = 0; s < std::min(n, LTMP2_NUM_STAGES); ++s) {
    if (ms) ms[s] = ctx->timer.ms[s];
    if (launches) launches[s] = ctx->timer.launches[s];
  }
  return LTMP2_OK;
}

int ltmp2_reset_stage_times(ltmp2_ctx *ctx) {
  if (!ctx) return LTMP2_ERR_INVALID_ARG;
  for (int s = 0; s < LTMP2_NUM_STAGES; ++s) {
    ctx->timer.ms[s] = 0;
    ctx->timer.launches[s] = 0;
  }
  return LTMP2_OK;
}

void ltmp2_destroy(ltmp2_ctx *ctx) {
  if (!ctx) return;
  DeviceGuard g(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  delete ctx;
}

int ltmp2_autotune(ltmp2_ctx *ctx, int *slab, int *gemm_variant) {
  if (ctx && ctx->p.nk > 0) return LTMP2_ERR_UNSUPPORTED;   // no k-point form
  if (!ctx) return LTMP2_ERR_INVALID_ARG;
  DeviceGuard g(ctx->device);
  int sl = 0, var = -1;
  const int rc = ctx->p.precision == LTMP2_FP64 ? tune_ctx<double>(ctx, &sl, &var) : tune_ctx<float>(ctx, &sl, &var);
  if (rc) return rc;
  if (slab) *slab = sl;
  if (gemm_variant) *gemm_variant = var;
  return LTMP2_OK;
}

int ltmp2_set_pair_mask(ltmp2_ctx *ctx, const unsigned char *keep) {
  if (ctx && ctx->p.nk > 0) return LTMP2_ERR_UNSUPPORTED;   // no k-point form
  if (!ctx) return LTMP2_ERR_INVALID_ARG;
  Plan &p = ctx->p;
  if (!keep) {
    p.pair_keep = nullptr;
    p.keep_list = nullptr;
    p.keep_count = nullptr;
    ctx->mask_hash = 0;
    return LTMP2_OK;
  }
  const int no = p.n_occ;
  for (int i = 0; i < no; ++i) {
    if (!keep[i * no + i]) return LTMP2_ERR_INVALID_ARG;
    for (int j = 0; j < i; ++j)
      if ((keep[i * no + j] != 0) != (keep[j * no + i] != 0)) return LTMP2_ERR_INVALID_ARG;
  }
  DeviceGuard g(ctx->device);
  int rc = LTMP2_OK;
  if (!ctx->d_keep) {
    if ((rc = dalloc(ctx, &ctx->d_keep, (size_t)no * no))) return rc;
    if ((rc = dalloc(ctx, &ctx->d_keep_list, (size_t)no * no))) return rc;
    if ((rc = dalloc(ctx, &ctx->d_keep_count, (size_t)no))) return rc;
  }
  std::vector<unsigned char> k01((size_t)no * no);
  std::vector<int> list((size_t)no * no, 0), count(no, 0);
  for (int j = 0; j < no; ++j)
    for (int i = 0; i < no; ++i) {
      k01[(size_t)i * no + j] = keep[(size_t)i * no + j] ? 1 : 0;
      if (keep[(size_t)i * no + j]) list[(size_t)j * no + count[j]++] = i;
    }
  if (cudaMemcpy(ctx->d_keep, k01.data(), k01.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(ctx->d_keep_list, list.data(), list.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(ctx->d_keep_count, count.data(), count.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
    return LTMP2_ERR_CUDA;
  p.pair_keep = ctx->d_keep;
  p.keep_list = ctx->d_keep_list;
  p.keep_count = ctx->d_keep_count;
  // the mask changes the exchange energy, so it enters the fingerprint
  unsigned long long h = 0xcbf29ce484222325ull;
  for (unsigned char b : k01) h = (h ^ b) * 0x100000001b3ull;
  ctx->mask_hash = h | 1ull;
  return LTMP2_OK;
}

int ltmp2_pair_descriptors(ltmp2_ctx *ctx, double *desc) {
  if (ctx && ctx->p.nk > 0) return LTMP2_ERR_UNSUPPORTED;   // no k-point form
  if (!ctx || !desc) return LTMP2_ERR_INVALID_ARG;
  try {
    return pair_descriptors(ctx, desc);
  } catch (const std::bad_alloc &) {
    return LTMP2_ERR_OOM;
  }
}

int ltmp2_get_tuning(const ltmp2_ctx *ctx, int *values) {
  if (!ctx || !values) return LTMP2_ERR_INVALID_ARG;
  values[0] = ctx->p.max_prim;
  values[1] = ctx->p.tc ? ctx->tc.variant : -1;
  values[2] = ctx->p.plane_kernel;
  values[3] = ctx->p.plane_ib;
  values[4] = ctx->p.tc && ctx->tc.real ? (ctx->tc.green_on() ? 1 : 0) : -1;
  values[5] = ctx->p.tc && ctx->tc.direct ? (ctx->tc.use_direct ? 1 : 0) : -1;
  return LTMP2_OK;
}

int ltmp2_set_tuning(ltmp2_ctx *ctx, const int *values) {
  if (ctx && ctx->p.nk > 0) return LTMP2_ERR_UNSUPPORTED;   // no k-point form
  if (!ctx || !values) return LTMP2_ERR_INVALID_ARG;
  Plan &p = ctx->p;
  const int slab = values[0] < 0 ? p.max_prim : values[0];
  int variant = values[1];
  const int pk = values[2] < 0 ? p.plane_kernel : values[2];
  const int ib = values[3] < 0 ? p.plane_ib : values[3];
  if (slab < 1 || slab > ctx->slab_capacity) return LTMP2_ERR_INVALID_ARG;
  if (variant >= 0) {
    if (!p.tc || (variant != 4 && variant != 5) || (ctx->tc.real && variant != 5)) return LTMP2_ERR_INVALID_ARG;
  }
  if (values[4] > 1 || values[5] > 1) return LTMP2_ERR_INVALID_ARG;
  if ((values[4] >= 0 && !(p.tc && ctx->tc.real)) || (values[5] >= 0 && !(p.tc && ctx->tc.direct)))
    return LTMP2_ERR_INVALID_ARG;
  const bool ok = p.precision == LTMP2_FP64 ? Path<double>::plane_feasible(p, pk, ib)
                                             : Path<float>::plane_feasible(p, pk, ib);
  if (!ok) return LTMP2_ERR_INVALID_ARG;
  DeviceGuard g(ctx->device);
  int rc = apply_tuning(ctx, slab, variant, pk, ib);
  if (rc) return rc;
  if (values[4] == 1 && !ctx->tc.green) {
    // first use: R_v^T and its split, once (the Green's function on the tensor cores)
    void *gmem = nullptr;
    if ((rc = dalloc_bytes(ctx, &gmem, tc_green_bytes(p.n_pw, p.n_v)))) return rc;
    cudaError_t e = tc_green_init(ctx->tc, gmem, (const float *)p.cv, p.n_v, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_status(e);
  }
  if (values[4] >= 0) ctx->tc.use_green = values[4] == 1;
  if (values[5] >= 0) ctx->tc.use_direct = values[5] == 1;
  return LTMP2_OK;
}

int ltmp2_batch_create(ltmp2_ctx *const *ctxs, int n, const int *n_tau, const double *const *tau,
                       const double *const *w, ltmp2_batch **out) {
  if (ctxs && n > 0)
    for (int k = 0; k < n; ++k)
      if (ctxs[k] && ctxs[k]->p.nk > 0) return LTMP2_ERR_UNSUPPORTED;   // no k-point form
  if (!ctxs || !n_tau || !tau || !w || !out || n < 1) return LTMP2_ERR_INVALID_ARG;
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i]) return LTMP2_ERR_INVALID_ARG;
    if (ctxs[i]->device != ctxs[0]->device) return LTMP2_ERR_INVALID_ARG;
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return LTMP2_ERR_INVALID_ARG;
    const int rc = check_tau(n_tau[i], tau[i], w[i]);
    if (rc) return rc;
  }
  DeviceGuard g(ctxs[0]->device);
  ltmp2_batch *b = new (std::nothrow) ltmp2_batch();
  if (!b) return LTMP2_ERR_OOM;
  b->device = ctxs[0]->device;
  b->ctxs.assign(ctxs, ctxs + n);
  b->launches.assign(n, 0);
  auto fail = [&](int rc) {
    cudaGetLastError();
    delete b;
    return rc;
  };
  if (cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking) != cudaSuccess) return fail(LTMP2_ERR_CUDA);
  b->streams.resize(n, nullptr);
  b->events.resize(n + 1, nullptr);
  for (int i = 0; i < n; ++i)
    if (cudaStreamCreateWithFlags(&b->streams[i], cudaStreamNonBlocking) != cudaSuccess) return fail(LTMP2_ERR_CUDA);
  for (auto &e : b->events)
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return fail(LTMP2_ERR_CUDA);
  // persistent shared FFT stages when every system allows them (Gamma point, one precision, no
  // cutoff levels, the Green's-function route) and the systems need similar numbers of
  // (tau, slab) rounds; else one graph branch per system.  Rounds keep the systems in
  // lockstep: when one system needs many more rounds than the others, most rounds hold that
  // system alone and the lockstep only adds synchronisation (the 8-system workload: 6 to
  // 850 rounds, 0.59x the systems run one after another; independent branches: about 1x).
  bool persist = n <= kBatchMax;
  int rmin = 0, rmax = 0;
  for (int i = 0; i < n; ++i) {
    const Plan &p = ctxs[i]->p;
    persist = persist && p.nk == 0 && p.n_lev < 2 && p.route == 0 && p.precision == ctxs[0]->p.precision;
    const int rounds = n_tau[i] * ((p.n_prim + p.max_prim - 1) / p.max_prim);
    rmin = i == 0 ? rounds : std::min(rmin, rounds);
    rmax = std::max(rmax, rounds);
  }
  persist = persist && rmax <= 2 * rmin;
  if (persist) {
    b->persistent = true;
    const int prc = ctxs[0]->p.precision == LTMP2_FP64 ? capture_rounds<double>(b, ctxs, n, n_tau, tau, w)
                                                      : capture_rounds<float>(b, ctxs, n, n_tau, tau, w);
    if (prc) return fail(prc);
    if (cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess) return fail(LTMP2_ERR_CUDA);
    *out = b;
    return LTMP2_OK;
  }
  if (cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return fail(LTMP2_ERR_CUDA);
  int rc = cuda_status(cudaEventRecord(b->events[n], b->origin));
  for (int i = 0; i < n && !rc; ++i) {
    ltmp2_ctx *c = ctxs[i];
    rc = cuda_status(cudaStreamWaitEvent(b->streams[i], b->events[n], 0));
    if (!rc)
      rc = c->p.precision == LTMP2_FP64
               ? enqueue_energy<double>(c, b->streams[i], n_tau[i], tau[i], w[i], 0, c->p.n_prim, nullptr,
                                        &b->launches[i])
               : enqueue_energy<float>(c, b->streams[i], n_tau[i], tau[i], w[i], 0, c->p.n_prim, nullptr,
                                       &b->launches[i]);
    if (!rc) rc = cuda_status(cudaEventRecord(b->events[i], b->streams[i]));
    if (!rc) rc = cuda_status(cudaStreamWaitEvent(b->origin, b->events[i], 0));
  }
  const cudaError_t ec = cudaStreamEndCapture(b->origin, &b->graph);
  if (rc) return fail(rc);
  if (ec != cudaSuccess) return fail(LTMP2_ERR_CUDA);
  if (cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess) return fail(LTMP2_ERR_CUDA);
  *out = b;
  return LTMP2_OK;
}

int ltmp2_batch_run(ltmp2_batch *b, double *e_direct, double *e_exchange) {
  if (!b || !e_direct || !e_exchange) return LTMP2_ERR_INVALID_ARG;
  DeviceGuard g(b->device);
  cudaStream_t st = b->ctxs[0]->stream;
  cudaError_t e = cudaGraphLaunch(b->exec, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_status(e);
  for (size_t i = 0; i < b->ctxs.size(); ++i) {
    ltmp2_ctx *c = b->ctxs[i];
    int rc = check_tc_flag(c);
    if (rc) return rc;
    double es[4];
    e = cudaMemcpy(es, c->p.esum, sizeof(es), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_status(e);
    e_direct[i] = es[0];
    e_exchange[i] = es[1];
    c->last_imag[0] = es[2];
    c->last_imag[1] = es[3];
    c->kernel_launches += b->launches[i];
  }
  return LTMP2_OK;
}

int ltmp2_batch_kernel_nodes(const ltmp2_batch *b, long long *count) {
  if (!b || !count) return LTMP2_ERR_INVALID_ARG;
  long long t = 0;
  for (long long x : b->launches) t += x;
  *count = t;
  return LTMP2_OK;
}

int ltmp2_batch_mode(const ltmp2_batch *b, int *persistent) {
  if (!b || !persistent) return LTMP2_ERR_INVALID_ARG;
  *persistent = b->persistent ? 1 : 0;
  return LTMP2_OK;
}

void ltmp2_batch_destroy(ltmp2_batch *b) {
  if (!b) return;
  DeviceGuard g(b->device);
  delete b;
}

int ltmp2_energy_batch(ltmp2_ctx *const *ctxs, int n, const int *n_tau, const double *const *tau,
                       const double *const *w, double *e_direct, double *e_exchange) {
  if (!ctxs || n < 1 || !e_direct || !e_exchange) return LTMP2_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i]) return LTMP2_ERR_INVALID_ARG;
    const int rc = ltmp2_autotune(ctxs[i], nullptr, nullptr);
    if (rc) return rc;
  }
  ltmp2_batch *b = nullptr;
  int rc = ltmp2_batch_create(ctxs, n, n_tau, tau, w, &b);
  if (rc) return rc;
  rc = ltmp2_batch_run(b, e_direct, e_exchange);
  ltmp2_batch_destroy(b);
  return rc;
}

// ---------------------------------------------------------------- failure-path self-test
int ltmp2_selftest_wait(ltmp2_ctx *ctx, int budget_us) {
  if (!ctx || budget_us < 1 || budget_us > 1000000) return LTMP2_ERR_INVALID_ARG;
  DeviceGuard g(ctx->device);
  int rc;
  if (!ctx->d_selftest_err && (rc = dalloc(ctx, &ctx->d_selftest_err, 1))) return rc;
  cudaError_t e = cudaMemsetAsync(ctx->d_selftest_err, 0, sizeof(int), ctx->stream);
  if (e == cudaSuccess) e = tc_wait_selftest(ctx->d_selftest_err, 1000ull * (unsigned long long)budget_us, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  int flag = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&flag, ctx->d_selftest_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_status(e);
  ctx->kernel_launches += 1;
  return flag ? LTMP2_ERR_TIMEOUT : LTMP2_OK;
}

// ---------------------------------------------------------------- spin-unrestricted form
int ltmp2_energy_uhf(ltmp2_ctx *alpha, ltmp2_ctx *beta, int n_tau, const double *tau, const double *w,
                     double *e_direct, double *e_exchange, double *e_spin) {
  if ((alpha && alpha->p.nk > 0) || (beta && beta->p.nk > 0)) return LTMP2_ERR_UNSUPPORTED;   // no k-point form
  if (!alpha || !beta || alpha == beta || !e_direct || !e_exchange) return LTMP2_ERR_INVALID_ARG;
  int rc = check_tau(n_tau, tau, w);
  if (rc) return rc;
  Plan &pa = alpha->p, &pb = beta->p;
  // the two channels must share the cell, grid, plane waves and auxiliary set
  if (alpha->device != beta->device || pa.precision != pb.precision || pa.n != pb.n || pa.n_pw != pb.n_pw ||
      pa.n_aux != pb.n_aux || pa.n_prim != pb.n_prim || pa.real_orb != pb.real_orb ||
      alpha->aux_g2 != beta->aux_g2 || std::memcmp(alpha->lattice, beta->lattice, sizeof(alpha->lattice)) != 0)
    return LTMP2_ERR_INVALID_ARG;
  if (pa.n_lev > 1 || pb.n_lev > 1 || pa.pair_keep || pb.pair_keep) return LTMP2_ERR_UNSUPPORTED;
  DeviceGuard g(alpha->device);
  // a common slab size; restored afterwards
  const int keep_a = pa.max_prim, keep_b = pb.max_prim;
  const int slab = std::min(keep_a, keep_b);
  if (!alpha->d_cross_y || alpha->cross_nb != pb.n_occ) {
    const size_t nab = (size_t)pa.n_occ * pb.n_occ;
    if ((rc = dalloc(alpha, &alpha->d_cross_y, (size_t)alpha->slab_capacity * nab))) return rc;
    if ((rc = dalloc(alpha, &alpha->d_cross_acc, nab))) return rc;
    if ((rc = dalloc(alpha, &alpha->d_cross_sum, 1))) return rc;
    alpha->cross_nb = pb.n_occ;
  }
  pa.max_prim = pb.max_prim = slab;
  rc = pa.precision == LTMP2_FP64 ? enqueue_uhf<double>(alpha, beta, n_tau, tau, w, &alpha->kernel_launches)
                                  : enqueue_uhf<float>(alpha, beta, n_tau, tau, w, &alpha->kernel_launches);
  cudaError_t e = cudaStreamSynchronize(alpha->stream);
  pa.max_prim = keep_a;
  pb.max_prim = keep_b;
  if (rc) return rc;
  if (e != cudaSuccess) return cuda_status(e);
  if ((rc = check_tc_flag(alpha)) || (rc = check_tc_flag(beta))) return rc;
  double ea[4], eb[4], ecross = 0.0;
  if ((e = cudaMemcpy(ea, pa.esum, sizeof(ea), cudaMemcpyDeviceToHost)) != cudaSuccess ||
      (e = cudaMemcpy(eb, pb.esum, sizeof(eb), cudaMemcpyDeviceToHost)) != cudaSuccess ||
      (e = cudaMemcpy(&ecross, alpha->d_cross_sum, sizeof(double), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_status(e);
  // each channel's sums follow the closed-shell weights (direct 2, exchange 1 per spin sum):
  // the spin-unrestricted weights are 1/2 per (s, s') and 1/2 per s
  *e_direct = 0.25 * (ea[0] + eb[0]) + ecross;
  *e_exchange = 0.5 * (ea[1] + eb[1]);
  if (e_spin) {
    e_spin[0] = 0.25 * ea[0] + 0.5 * ea[1];
    e_spin[1] = 0.25 * eb[0] + 0.5 * eb[1];
    e_spin[2] = ecross;
  }
  return LTMP2_OK;
}

// ---------------------------------------------------------------- transformed-state route
int ltmp2_set_route(ltmp2_ctx *ctx, int route) {
  if (ctx && ctx->p.nk > 0) return LTMP2_ERR_UNSUPPORTED;   // no k-point form
  if (!ctx || (route != LTMP2_ROUTE_GREEN && route != LTMP2_ROUTE_OVERLAP)) return LTMP2_ERR_INVALID_ARG;
  Plan &p = ctx->p;
  if (route == LTMP2_ROUTE_GREEN) {
    p.route = 0;
    return LTMP2_OK;
  }
  if (!p.real_basis) return LTMP2_ERR_UNSUPPORTED;
  DeviceGuard g(ctx->device);
  const size_t cs = p.precision == LTMP2_FP64 ? 16 : 8;
  int rc;
  if (!p.rt && (rc = dalloc_bytes(ctx, &p.rt, cs * (size_t)p.n_prim * p.n_occ * p.n_v))) return rc;
  cudaError_t e = p.precision == LTMP2_FP64 ? Path<double>::overlap_setup(p, ctx->stream)
                                             : Path<float>::overlap_setup(p, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_status(e);
  ctx->kernel_launches += 1 + 2 * ((p.n_prim + p.max_prim - 1) / p.max_prim);
  p.route = 1;
  return LTMP2_OK;
}

// ---------------------------------------------------------------- virtuals per Laplace point
int ltmp2_set_virtual_cut(ltmp2_ctx *ctx, int mode, double log2_cut) {
  if (ctx && ctx->p.nk > 0) return LTMP2_ERR_UNSUPPORTED;   // no k-point form
  if (!ctx || mode < LTMP2_VIRTUALS_ALL || mode > LTMP2_VIRTUALS_SPACE || !(log2_cut >= 53.0) ||
      !(log2_cut <= 1100.0))
    return LTMP2_ERR_INVALID_ARG;
  ctx->virt_mode = mode;
  ctx->virt_log2 = log2_cut;
  return LTMP2_OK;
}

int ltmp2_tau_virtuals(ltmp2_ctx *ctx, int n_tau, const double *tau, int *n_virt, int *w_virtual) {
  if (!ctx || !n_virt || !tau || n_tau < 1) return LTMP2_ERR_INVALID_ARG;
  for (int k = 0; k < n_tau; ++k)
    if (!(tau[k] > 0.0) || !std::isfinite(tau[k])) return LTMP2_ERR_INVALID_ARG;
  for (int k = 0; k < n_tau; ++k) {
    bool wv = false;
    n_virt[k] = tau_virtuals(ctx, tau[k], &wv);
    if (w_virtual) w_virtual[k] = wv ? 1 : 0;
  }
  return LTMP2_OK;
}

// ---------------------------------------------------------------- internal cutoff extrapolation
static_assert(kMaxLevels == LTMP2_MAX_LEVELS, "level capacity");
int ltmp2_set_extrapolation(ltmp2_ctx *ctx, int n_c, double alpha) {
  if (ctx && ctx->p.nk > 0) return LTMP2_ERR_UNSUPPORTED;   // no k-point form
  if (!ctx) return LTMP2_ERR_INVALID_ARG;
  Plan &p = ctx->p;
  ctx->lev_done = false;
  if (n_c <= 1) {
    p.n_lev = 0;
    ctx->lev_ecut.clear();
    ctx->lev_count.clear();
    return LTMP2_OK;
  }
  if (n_c > kMaxLevels || !(alpha > 1.0) || !std::isfinite(alpha)) return LTMP2_ERR_INVALID_ARG;
  const size_t cs = p.precision == LTMP2_FP64 ? 16 : 8;
  if (2 * (size_t)p.n_aux * cs > 200 * 1024) return LTMP2_ERR_UNSUPPORTED;  // column kernel's shared memory
  DeviceGuard g(ctx->device);
  const int naux = p.n_aux, no = p.n_occ;
  std::vector<double> ecut(n_c);
  for (int n = 0; n < n_c; ++n) ecut[n] = ctx->ecut_aux / std::pow(alpha, (double)n);
  // L(G) = number of nested spheres that contain G (G = 0, which never contributes, gets n_c)
  std::vector<unsigned char> lev(naux);
  std::vector<int> count(n_c, 0);
  for (int k = 0; k < naux; ++k) {
    int L = 1;
    const double e = 0.5 * ctx->aux_g2[k];
    if (ctx->aux_g2[k] == 0.0) L = n_c;
    else
      while (L < n_c && e <= ecut[L]) ++L;
    lev[k] = (unsigned char)L;
    if (ctx->aux_g2[k] != 0.0)
      for (int n = 0; n < L; ++n) ++count[n];
  }
  std::vector<int> order(naux), start(n_c + 1, 0);
  for (int k = 0; k < naux; ++k) order[k] = k;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return lev[a] < lev[b]; });
  for (int n = 0; n <= n_c; ++n) {
    int k = 0;
    while (k < naux && lev[order[k]] <= n) ++k;
    start[n] = k;
  }
  int rc;
  if (!ctx->lev_alloc) {
    p.lev_stride = (size_t)ctx->slab_capacity * no * no;
    unsigned char *al = nullptr;
    int *lo = nullptr, *ls = nullptr;
    if ((rc = dalloc(ctx, &p.sxl, (size_t)kMaxLevels * p.lev_stride))) return rc;
    if ((rc = dalloc(ctx, &p.ydl, (size_t)kMaxLevels * p.lev_stride))) return rc;
    if ((rc = dalloc(ctx, &p.exl, (size_t)kMaxLevels * no * no))) return rc;
    if ((rc = dalloc(ctx, &p.edl, (size_t)kMaxLevels * no * no))) return rc;
    if ((rc = dalloc(ctx, &p.esum_lev, (size_t)2 * kMaxLevels))) return rc;
    if ((rc = dalloc(ctx, &al, (size_t)naux))) return rc;
    if ((rc = dalloc(ctx, &lo, (size_t)naux))) return rc;
    if ((rc = dalloc(ctx, &ls, (size_t)kMaxLevels + 1))) return rc;
    p.aux_lev = al;
    p.lev_order = lo;
    p.lev_start = ls;
    ctx->lev_alloc = true;
  }
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpy((void *)p.aux_lev, lev.data(), naux, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy((void *)p.lev_order, order.data(), naux * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy((void *)p.lev_start, start.data(), (n_c + 1) * sizeof(int), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_status(e);
  p.n_lev = n_c;
  ctx->lev_ecut = ecut;
  ctx->lev_count = count;
  return LTMP2_OK;
}

int ltmp2_level_energies(const ltmp2_ctx *ctx, double *ecut_aux, int *n_aux, double *e_direct,
                         double *e_exchange) {
  if (!ctx || ctx->p.n_lev < 2) return LTMP2_ERR_INVALID_ARG;
  const int nl = ctx->p.n_lev;
  for (int n = 0; n < nl; ++n) {
    if (ecut_aux) ecut_aux[n] = ctx->lev_ecut[n];
    if (n_aux) n_aux[n] = ctx->lev_count[n];
  }
  if (!e_direct && !e_exchange) return LTMP2_OK;
  if (!ctx->lev_done) return LTMP2_ERR_INVALID_ARG;
  DeviceGuard g(ctx->device);
  double es[2 * kMaxLevels];
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpy(es, ctx->p.esum_lev, 2 * nl * sizeof(double), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_status(e);
  for (int n = 0; n < nl; ++n) {
    if (e_direct) e_direct[n] = es[2 * n];
    if (e_exchange) e_exchange[n] = es[2 * n + 1];
  }
  return LTMP2_OK;
}

int ltmp2_extrapolate(int n, const double *ecut_aux, const double *energy, double *e_inf, double *slope,
                      double *sigma) {
  if (n < 2 || !ecut_aux || !energy || !e_inf) return LTMP2_ERR_INVALID_ARG;
  double sx = 0, sy = 0, sxx = 0, sxy = 0;
  std::vector<double> x(n);
  for (int k = 0; k < n; ++k) {
    if (!(ecut_aux[k] > 0.0) || !std::isfinite(ecut_aux[k]) || !std::isfinite(energy[k])) return LTMP2_ERR_INVALID_ARG;
    x[k] = std::pow(ecut_aux[k], -1.5);
    sx += x[k]; sy += energy[k]; sxx += x[k] * x[k]; sxy += x[k] * energy[k];
  }
  const double det = n * sxx - sx * sx;
  if (!(std::fabs(det) > 0.0)) return LTMP2_ERR_INVALID_ARG;   // all cutoffs equal
  const double b = (n * sxy - sx * sy) / det, a = (sy - b * sx) / n;
  *e_inf = a;
  if (slope) *slope = b;
  if (sigma) {
    double r2 = 0;
    for (int k = 0; k < n; ++k) r2 += (energy[k] - a - b * x[k]) * (energy[k] - a - b * x[k]);
    *sigma = n > 2 ? std::sqrt(r2 / (n - 2) * sxx / det) : 0.0;
  }
  return LTMP2_OK;
}

}  // extern "C"

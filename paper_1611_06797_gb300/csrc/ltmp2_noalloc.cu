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
#include <map>
#include <mutex>
#include <type_traits>
#include <vector>

#include "../../include/ltmp2.h"
#include "fft.cuh"
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
// array's name as an address).  Looked up once per device.
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

struct NaCol {
  int m1, m2, zlo, zhi, off;
};

bool na_columns(const std::vector<std::array<int, 3>> &m, std::vector<NaCol> &cols, std::vector<int> &order) {
  const int n = (int)m.size();
  order.resize(n);
  for (int k = 0; k < n; ++k) order[k] = k;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return m[a] < m[b]; });
  cols.clear();
  for (int k = 0; k < n; ++k) {
    const auto &q = m[order[k]];
    if (cols.empty() || cols.back().m1 != q[0] || cols.back().m2 != q[1]) {
      cols.push_back({q[0], q[1], q[2], q[2], k});
    } else {
      if (q[2] != cols.back().zhi + 1) return false;
      cols.back().zhi = q[2];
    }
  }
  return true;
}

double na_g2(const double B[9], int a, int b, int c) {
  const double x = a * B[0] + b * B[3] + c * B[6];
  const double y = a * B[1] + b * B[4] + c * B[7];
  const double z = a * B[2] + b * B[5] + c * B[8];
  return x * x + y * y + z * z;
}

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

}  // namespace

extern "C" int ltmp2_energy_noalloc(const ltmp2_system *sys, int n_tau, const double *tau, const double *w,
                                    double *e_direct, double *e_exchange, double *e_pair, void *stream) {
  if (!sys || !e_direct || !e_exchange || !tau || !w || n_tau < 1) return LTMP2_ERR_INVALID_ARG;
  for (int k = 0; k < n_tau; ++k)
    if (!(tau[k] > 0.0) || !std::isfinite(tau[k]) || !std::isfinite(w[k])) return LTMP2_ERR_INVALID_ARG;
  if (!sys->miller || !sys->coeff || !sys->eps) return LTMP2_ERR_INVALID_ARG;
  if (sys->n_pw < 2 || sys->n_orb < 2 || sys->n_occ < 1 || sys->n_occ >= sys->n_orb || sys->n_orb > sys->n_pw)
    return LTMP2_ERR_INVALID_ARG;
  if (sys->precision != LTMP2_FP64 && sys->precision != LTMP2_FP32) return LTMP2_ERR_INVALID_ARG;
  if (sys->flags & ~LTMP2_FLAG_REAL_ORBITALS) return LTMP2_ERR_INVALID_ARG;
  const int n = sys->grid[0];
  if (sys->grid[1] != n || sys->grid[2] != n || !fft_size_supported(n)) return LTMP2_ERR_GRID;
  const int no = sys->n_occ, npw = sys->n_pw, norb = sys->n_orb;
  for (int k = 0; k < norb; ++k) {
    if (!std::isfinite(sys->eps[k])) return LTMP2_ERR_INVALID_ARG;
    if (k > 0 && sys->eps[k] < sys->eps[k - 1]) return LTMP2_ERR_INVALID_ARG;
  }
  if (sys->eps[no] - sys->eps[no - 1] < 1e-6) return LTMP2_ERR_GAP;
  // reciprocal lattice
  const double *A = sys->lattice;
  const double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                     A[2] * (A[3] * A[7] - A[4] * A[6]);
  if (!std::isfinite(det) || det == 0.0) return LTMP2_ERR_INVALID_ARG;
  double inv[9] = {(A[4] * A[8] - A[5] * A[7]) / det, (A[2] * A[7] - A[1] * A[8]) / det,
                   (A[1] * A[5] - A[2] * A[4]) / det, (A[5] * A[6] - A[3] * A[8]) / det,
                   (A[0] * A[8] - A[2] * A[6]) / det, (A[2] * A[3] - A[0] * A[5]) / det,
                   (A[3] * A[7] - A[4] * A[6]) / det, (A[1] * A[6] - A[0] * A[7]) / det,
                   (A[0] * A[4] - A[1] * A[3]) / det};
  double B[9];
  const double tp = 6.283185307179586476925286766559;
  for (int k = 0; k < 3; ++k)
    for (int c = 0; c < 3; ++c) B[k * 3 + c] = tp * inv[c * 3 + k];
  // plane-wave set
  std::vector<std::array<int, 3>> m(npw);
  std::map<std::array<int, 3>, int> where;
  double g2max = 0.0;
  for (int q = 0; q < npw; ++q) {
    for (int k = 0; k < 3; ++k) {
      m[q][k] = sys->miller[3 * q + k];
      if (2 * std::abs(m[q][k]) >= n) return LTMP2_ERR_GRID;
    }
    if (!where.emplace(m[q], q).second) return LTMP2_ERR_INVALID_ARG;
    g2max = std::max(g2max, na_g2(B, m[q][0], m[q][1], m[q][2]));
  }
  std::vector<int> negpw(npw);
  for (int q = 0; q < npw; ++q) {
    auto it = where.find({-m[q][0], -m[q][1], -m[q][2]});
    if (it == where.end()) return LTMP2_ERR_GRID;
    negpw[q] = it->second;
  }
  const bool real_orb = (sys->flags & LTMP2_FLAG_REAL_ORBITALS) != 0;
  if (real_orb)
    for (int r = 0; r < norb; ++r) {
      const double *c = sys->coeff + (size_t)r * npw * 2;
      for (int q = 0; q < npw; ++q) {
        const int qn = negpw[q];
        if (std::fabs(c[2 * q] - c[2 * qn]) > 1e-10 || std::fabs(c[2 * q + 1] + c[2 * qn + 1]) > 1e-10)
          return LTMP2_ERR_NOT_REAL;
      }
    }
  std::vector<NaCol> ocols;
  std::vector<int> order;
  if (!na_columns(m, ocols, order)) return LTMP2_ERR_GRID;
  // auxiliary set in column order, G = 0 kept with v = 0
  const double ecut_aux = sys->ecut_aux > 0.0 ? sys->ecut_aux : (2.0 / 3.0) * 0.5 * g2max;
  std::vector<std::array<int, 3>> am;
  {
    const double gmax = std::sqrt(2.0 * ecut_aux);
    int lim[3];
    for (int k = 0; k < 3; ++k) {
      const double an = std::sqrt(A[3 * k] * A[3 * k] + A[3 * k + 1] * A[3 * k + 1] + A[3 * k + 2] * A[3 * k + 2]);
      lim[k] = (int)std::floor(gmax * an / tp) + 1;
    }
    for (int a = -lim[0]; a <= lim[0]; ++a)
      for (int b = -lim[1]; b <= lim[1]; ++b)
        for (int d = -lim[2]; d <= lim[2]; ++d)
          if (0.5 * na_g2(B, a, b, d) <= ecut_aux) {
            if (2 * std::abs(a) >= n || 2 * std::abs(b) >= n || 2 * std::abs(d) >= n) return LTMP2_ERR_GRID;
            am.push_back({a, b, d});
          }
  }
  if (am.size() < 3) return LTMP2_ERR_INVALID_ARG;
  std::vector<NaCol> acols;
  std::vector<int> aorder;
  if (!na_columns(am, acols, aorder)) return LTMP2_ERR_GRID;
  const int naux = (int)am.size();
  std::vector<std::array<int, 3>> amo(naux);
  for (int k = 0; k < naux; ++k) amo[k] = am[aorder[k]];
  std::map<std::array<int, 3>, int> awhere;
  for (int k = 0; k < naux; ++k) awhere[amo[k]] = k;
  std::vector<int> aneg(naux), prim;
  std::vector<double> v64(naux);
  std::vector<float> v32(naux);
  for (int k = 0; k < naux; ++k) {
    aneg[k] = awhere.at({-amo[k][0], -amo[k][1], -amo[k][2]});
    const double g2 = na_g2(B, amo[k][0], amo[k][1], amo[k][2]);
    v64[k] = g2 > 0.0 ? 12.566370614359172953850573533118 / g2 : 0.0;
    v32[k] = (float)v64[k];
    const int first = amo[k][0] != 0 ? amo[k][0] : (amo[k][1] != 0 ? amo[k][1] : amo[k][2]);
    if (first > 0) prim.push_back(k);
  }

  void *base = nullptr;
  int rc = scratch_base(&base);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Arena ar(base, kNoAllocScratchBytes);
  Plan p;
  p.n = n;
  p.n_occ = no;
  p.n_orb = norb;
  p.n_pw = npw;
  p.n_v = norb - no;
  p.n_dorb = (int)ocols.size();
  p.n_daux = (int)acols.size();
  p.n_aux = naux;
  p.n_prim = (int)prim.size();
  p.real_orb = real_orb;
  p.real_basis = real_orb;
  p.precision = sys->precision;
  p.omega = std::fabs(det);
  p.mu = 0.5 * (sys->eps[no - 1] + sys->eps[no]);
  p.mxlo_orb = ocols.front().m1;
  p.mxhi_orb = ocols.back().m1;
  p.mxlo_aux = acols.front().m1;
  p.mxhi_aux = acols.back().m1;
  std::vector<int4> hdorb(p.n_dorb), hdaux(p.n_daux);
  std::vector<int> hdorb_off(p.n_dorb), hdaux_off(p.n_daux), hpw(3 * (size_t)npw), haux(3 * (size_t)naux);
  for (int d = 0; d < p.n_dorb; ++d) {
    hdorb[d] = make_int4(ocols[d].m1, ocols[d].m2, ocols[d].zlo, ocols[d].zhi);
    hdorb_off[d] = ocols[d].off;
  }
  for (int d = 0; d < p.n_daux; ++d) {
    hdaux[d] = make_int4(acols[d].m1, acols[d].m2, acols[d].zlo, acols[d].zhi);
    hdaux_off[d] = acols[d].off;
  }
  for (int q = 0; q < npw; ++q)
    for (int k = 0; k < 3; ++k) hpw[3 * q + k] = m[order[q]][k];
  for (int q = 0; q < naux; ++q)
    for (int k = 0; k < 3; ++k) haux[3 * q + k] = amo[q][k];
  std::vector<double> heps(sys->eps, sys->eps + norb);
  auto put = [&](auto **dst, const auto &vec) -> int {
    using X = typename std::remove_reference<decltype(vec)>::type::value_type;
    void *q = ar.take(vec.size() * sizeof(X));
    if (!q) return LTMP2_ERR_UNSUPPORTED;
    *dst = reinterpret_cast<typename std::remove_reference<decltype(*dst)>::type>(q);
    return copy_in(q, vec.data(), vec.size() * sizeof(X), st);
  };
  if ((rc = put(&p.dorb, hdorb))) return rc;
  if ((rc = put(&p.dorb_off, hdorb_off))) return rc;
  if ((rc = put(&p.daux, hdaux))) return rc;
  if ((rc = put(&p.daux_off, hdaux_off))) return rc;
  if ((rc = put(&p.pw_m, hpw))) return rc;
  if (real_orb) {
    std::vector<int> pos(npw), hpair(npw);
    for (int q = 0; q < npw; ++q) pos[order[q]] = q;
    for (int q = 0; q < npw; ++q) hpair[q] = pos[negpw[order[q]]];
    if ((rc = put(&p.pw_pair, hpair))) return rc;
  }
  if ((rc = put(&p.aux_m, haux))) return rc;
  if ((rc = put(&p.aux_neg, aneg))) return rc;
  if ((rc = put(&p.prim, prim))) return rc;
  if ((rc = put(&p.v_aux64, v64))) return rc;
  if ((rc = put(&p.v_aux32, v32))) return rc;
  if ((rc = put(&p.eps, heps))) return rc;
  return sys->precision == LTMP2_FP64
             ? run_noalloc<double>(sys, p, ar, order, n_tau, tau, w, st, e_direct, e_exchange, e_pair)
             : run_noalloc<float>(sys, p, ar, order, n_tau, tau, w, st, e_direct, e_exchange, e_pair);
}

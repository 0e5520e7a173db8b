// Host-side validation and index tables of one system (see host_plan.h).
#include "host_plan.h"
#include "fft.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>

namespace ltmp2 {
namespace {

struct Col {
  int m1, m2, zlo, zhi, off;
};

// Group Miller indices into (m1, m2) columns with contiguous m3 ranges; order[k] is the
// caller's index of the k-th point in column order.  false if a column has a gap.
bool build_columns(const std::vector<std::array<int, 3>> &m, std::vector<Col> &cols, std::vector<int> &order) {
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

// rows a_i -> rows b_k with a_i . b_k = 2 pi delta_ik; false for a singular cell
bool reciprocal(const double *A, double B[9], double *omega) {
  const double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                     A[2] * (A[3] * A[7] - A[4] * A[6]);
  if (!std::isfinite(det) || det == 0.0) return false;
  *omega = std::fabs(det);
  const double inv[9] = {(A[4] * A[8] - A[5] * A[7]) / det, (A[2] * A[7] - A[1] * A[8]) / det,
                         (A[1] * A[5] - A[2] * A[4]) / det, (A[5] * A[6] - A[3] * A[8]) / det,
                         (A[0] * A[8] - A[2] * A[6]) / det, (A[2] * A[3] - A[0] * A[5]) / det,
                         (A[3] * A[7] - A[4] * A[6]) / det, (A[1] * A[6] - A[0] * A[7]) / det,
                         (A[0] * A[4] - A[1] * A[3]) / det};
  const double tp = 6.283185307179586476925286766559;
  for (int k = 0; k < 3; ++k)
    for (int c = 0; c < 3; ++c) B[k * 3 + c] = tp * inv[c * 3 + k];
  return true;
}

double g2_of(const double B[9], int m1, int m2, int m3) {
  const double gx = m1 * B[0] + m2 * B[3] + m3 * B[6];
  const double gy = m1 * B[1] + m2 * B[4] + m3 * B[7];
  const double gz = m1 * B[2] + m2 * B[5] + m3 * B[8];
  return gx * gx + gy * gy + gz * gz;
}

bool primary(const std::array<int, 3> &m) {
  const int first = m[0] != 0 ? m[0] : (m[1] != 0 ? m[1] : m[2]);
  return first > 0;
}

// 64-bit word hash (multiply / xor-shift), order dependent
struct Hash {
  uint64_t h = 0x9e3779b97f4a7c15ull;
  void word(uint64_t w) {
    h ^= w + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
    h *= 0xff51afd7ed558ccdull;
    h ^= h >> 33;
  }
  void bytes(const void *p, size_t n) {
    const unsigned char *c = static_cast<const unsigned char *>(p);
    size_t k = 0;
    for (; k + 8 <= n; k += 8) {
      uint64_t w;
      std::memcpy(&w, c + k, 8);
      word(w);
    }
    uint64_t tail = 0;
    std::memcpy(&tail, c + k, n - k);
    word(tail ^ ((uint64_t)n << 56));
  }
};

int build(const ltmp2_system *sys, int allowed_flags, HostPlan &hp) {
  if (!sys) return LTMP2_ERR_INVALID_ARG;
  if (!sys->miller || !sys->coeff || !sys->eps) return LTMP2_ERR_INVALID_ARG;
  if (sys->n_pw < 2 || sys->n_orb < 2 || sys->n_occ < 1 || sys->n_occ >= sys->n_orb || sys->n_orb > sys->n_pw)
    return LTMP2_ERR_INVALID_ARG;
  if (sys->precision != LTMP2_FP64 && sys->precision != LTMP2_FP32) return LTMP2_ERR_INVALID_ARG;
  if (sys->flags & ~allowed_flags) return LTMP2_ERR_INVALID_ARG;
  for (int k = 0; k < 9; ++k)
    if (!std::isfinite(sys->lattice[k])) return LTMP2_ERR_INVALID_ARG;
  if (!std::isfinite(sys->ecut_aux)) return LTMP2_ERR_INVALID_ARG;
  const int n = sys->grid[0];
  if (sys->grid[1] != n || sys->grid[2] != n || !fft_size_supported(n)) return LTMP2_ERR_GRID;
  const int no = sys->n_occ, npw = sys->n_pw, norb = sys->n_orb;
  for (int k = 0; k < norb; ++k) {
    if (!std::isfinite(sys->eps[k])) return LTMP2_ERR_INVALID_ARG;
    if (k > 0 && sys->eps[k] < sys->eps[k - 1]) return LTMP2_ERR_INVALID_ARG;
  }
  if (sys->eps[no] - sys->eps[no - 1] < 1e-6) return LTMP2_ERR_GAP;
  double omega = 0.0;
  if (!reciprocal(sys->lattice, hp.B, &omega)) return LTMP2_ERR_INVALID_ARG;
  // every coefficient finite; the same pass hashes the inputs
  Hash h;
  h.bytes(sys->lattice, sizeof(sys->lattice));
  h.bytes(sys->grid, sizeof(sys->grid));
  const int sizes[4] = {npw, norb, no, sys->precision};
  h.bytes(sizes, sizeof(sizes));
  h.bytes(sys->miller, sizeof(int) * 3 * (size_t)npw);
  h.bytes(sys->eps, sizeof(double) * (size_t)norb);
  {
    const double *c = sys->coeff;
    const size_t cnt = 2 * (size_t)norb * npw;
    for (size_t k = 0; k < cnt; ++k) {
      if (!std::isfinite(c[k])) return LTMP2_ERR_INVALID_ARG;
      uint64_t w;
      std::memcpy(&w, c + k, 8);
      h.word(w);
    }
  }
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
    g2max = std::max(g2max, g2_of(hp.B, m[q][0], m[q][1], m[q][2]));
  }
  // -G of every plane wave: needed by the real-orbital (cos/sin basis) path only
  const bool real_flag = (sys->flags & LTMP2_FLAG_REAL_ORBITALS) != 0;
  hp.negpw.assign(npw, -1);
  for (int q = 0; q < npw; ++q) {
    auto it = where.find({-m[q][0], -m[q][1], -m[q][2]});
    if (it == where.end()) {
      if (real_flag) return LTMP2_ERR_GRID;
      continue;
    }
    hp.negpw[q] = it->second;
  }
  std::vector<Col> ocols;
  if (!build_columns(m, ocols, hp.order)) return LTMP2_ERR_GRID;
  // orthonormality on a deterministic sample of orbitals (both sides of the gap included)
  {
    std::vector<int> pick;
    const int S = std::min(norb, 40);
    for (int s = 0; s < S; ++s) pick.push_back((int)((long long)s * (norb - 1) / std::max(1, S - 1)));
    pick.push_back(no - 1);
    pick.push_back(no);
    std::sort(pick.begin(), pick.end());
    pick.erase(std::unique(pick.begin(), pick.end()), pick.end());
    for (size_t a = 0; a < pick.size(); ++a)
      for (size_t b = a; b < pick.size(); ++b) {
        const double *ca = sys->coeff + (size_t)pick[a] * npw * 2, *cb = sys->coeff + (size_t)pick[b] * npw * 2;
        double re = 0, im = 0;
        for (int q = 0; q < npw; ++q) {
          re += ca[2 * q] * cb[2 * q] + ca[2 * q + 1] * cb[2 * q + 1];
          im += ca[2 * q] * cb[2 * q + 1] - ca[2 * q + 1] * cb[2 * q];
        }
        if (std::fabs(re - (a == b ? 1.0 : 0.0)) > 1e-8 || std::fabs(im) > 1e-8) return LTMP2_ERR_NOT_ORTHONORMAL;
      }
  }
  const bool real_orb = (sys->flags & LTMP2_FLAG_REAL_ORBITALS) != 0;
  if (real_orb) {
    for (int r = 0; r < norb; ++r) {
      const double *c = sys->coeff + (size_t)r * npw * 2;
      for (int q = 0; q < npw; ++q) {
        const int qn = hp.negpw[q];
        if (std::fabs(c[2 * q] - c[2 * qn]) > 1e-10 || std::fabs(c[2 * q + 1] + c[2 * qn + 1]) > 1e-10)
          return LTMP2_ERR_NOT_REAL;
      }
    }
  }
  // auxiliary set A (Sec. II A) in column order, v(G) = 4 pi / |G|^2 (Eq. SCH2EI)
  const double ecut_aux = sys->ecut_aux > 0.0 ? sys->ecut_aux : (2.0 / 3.0) * 0.5 * g2max;
  std::vector<std::array<int, 3>> am;
  {
    const double gmax = std::sqrt(2.0 * ecut_aux);
    int lim[3];
    for (int k = 0; k < 3; ++k) {
      const double *a = sys->lattice + 3 * k;
      const double an = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
      lim[k] = (int)std::floor(gmax * an / 6.283185307179586476925286766559) + 1;
    }
    for (int a = -lim[0]; a <= lim[0]; ++a)
      for (int b = -lim[1]; b <= lim[1]; ++b)
        for (int d = -lim[2]; d <= lim[2]; ++d)
          // G = 0 is kept as a table entry with v(0) := 0 so that every column of the
          // sphere is one contiguous m3 range; it never contributes
          if (0.5 * g2_of(hp.B, a, b, d) <= ecut_aux) {
            if (2 * std::abs(a) >= n || 2 * std::abs(b) >= n || 2 * std::abs(d) >= n) return LTMP2_ERR_GRID;
            am.push_back({a, b, d});
          }
  }
  if (am.size() < 3) return LTMP2_ERR_INVALID_ARG;
  std::vector<Col> acols;
  std::vector<int> aorder;
  if (!build_columns(am, acols, aorder)) return LTMP2_ERR_GRID;
  const int naux = (int)am.size();
  std::vector<std::array<int, 3>> amo(naux);
  for (int k = 0; k < naux; ++k) amo[k] = am[aorder[k]];
  std::map<std::array<int, 3>, int> awhere;
  for (int k = 0; k < naux; ++k) awhere[amo[k]] = k;
  hp.aux_neg.assign(naux, 0);
  hp.v64.assign(naux, 0.0);
  hp.aux_g2.assign(naux, 0.0);
  hp.v32.assign(naux, 0.f);
  hp.prim.clear();
  for (int k = 0; k < naux; ++k) {
    auto it = awhere.find({-amo[k][0], -amo[k][1], -amo[k][2]});
    if (it == awhere.end()) return LTMP2_ERR_GRID;
    hp.aux_neg[k] = it->second;
    const double g2 = g2_of(hp.B, amo[k][0], amo[k][1], amo[k][2]);
    hp.aux_g2[k] = g2;
    hp.v64[k] = g2 > 0.0 ? 12.566370614359172953850573533118 / g2 : 0.0;
    hp.v32[k] = (float)hp.v64[k];
    if (primary(amo[k])) hp.prim.push_back(k);
  }
  h.bytes(&ecut_aux, sizeof(ecut_aux));
  const int fl = sys->flags;
  h.bytes(&fl, sizeof(fl));
  hp.fingerprint = h.h;
  hp.ecut_aux = ecut_aux;

  Plan &p = hp.p;
  p = Plan();
  p.n = n;
  p.n_occ = no;
  p.n_orb = norb;
  p.n_pw = npw;
  p.n_v = norb - no;
  p.n_dorb = (int)ocols.size();
  p.n_daux = (int)acols.size();
  p.n_aux = naux;
  p.n_prim = (int)hp.prim.size();
  p.real_orb = real_orb;
  p.real_basis = real_orb;
  p.precision = sys->precision;
  p.omega = omega;
  p.mu = 0.5 * (sys->eps[no - 1] + sys->eps[no]);
  p.mxlo_orb = ocols.front().m1;
  p.mxhi_orb = ocols.back().m1;
  p.mxlo_aux = acols.front().m1;
  p.mxhi_aux = acols.back().m1;
  hp.dorb.resize(p.n_dorb);
  hp.dorb_off.resize(p.n_dorb);
  hp.daux.resize(p.n_daux);
  hp.daux_off.resize(p.n_daux);
  for (int d = 0; d < p.n_dorb; ++d) {
    hp.dorb[d] = make_int4(ocols[d].m1, ocols[d].m2, ocols[d].zlo, ocols[d].zhi);
    hp.dorb_off[d] = ocols[d].off;
  }
  for (int d = 0; d < p.n_daux; ++d) {
    hp.daux[d] = make_int4(acols[d].m1, acols[d].m2, acols[d].zlo, acols[d].zhi);
    hp.daux_off[d] = acols[d].off;
  }
  hp.pw_m.resize(3 * (size_t)npw);
  hp.aux_m.resize(3 * (size_t)naux);
  for (int q = 0; q < npw; ++q)
    for (int k = 0; k < 3; ++k) hp.pw_m[3 * q + k] = m[hp.order[q]][k];
  for (int q = 0; q < naux; ++q)
    for (int k = 0; k < 3; ++k) hp.aux_m[3 * q + k] = amo[q][k];
  hp.pw_pair.clear();
  if (real_orb) {
    std::vector<int> pos(npw);
    for (int q = 0; q < npw; ++q) pos[hp.order[q]] = q;
    hp.pw_pair.resize(npw);
    for (int q = 0; q < npw; ++q) hp.pw_pair[q] = pos[hp.negpw[hp.order[q]]];
  }
  return LTMP2_OK;
}

// orthonormality of a deterministic sample of the rows of one k (both sides of the gap)
int check_orthonormal(const double *coeff, int norb, int npw, int no) {
  std::vector<int> pick;
  const int S = std::min(norb, 40);
  for (int s = 0; s < S; ++s) pick.push_back((int)((long long)s * (norb - 1) / std::max(1, S - 1)));
  pick.push_back(no - 1);
  pick.push_back(no);
  std::sort(pick.begin(), pick.end());
  pick.erase(std::unique(pick.begin(), pick.end()), pick.end());
  for (size_t a = 0; a < pick.size(); ++a)
    for (size_t b = a; b < pick.size(); ++b) {
      const double *ca = coeff + (size_t)pick[a] * npw * 2, *cb = coeff + (size_t)pick[b] * npw * 2;
      double re = 0, im = 0;
      for (int q = 0; q < npw; ++q) {
        re += ca[2 * q] * cb[2 * q] + ca[2 * q + 1] * cb[2 * q + 1];
        im += ca[2 * q] * cb[2 * q + 1] - ca[2 * q + 1] * cb[2 * q];
      }
      if (std::fabs(re - (a == b ? 1.0 : 0.0)) > 1e-8 || std::fabs(im) > 1e-8) return LTMP2_ERR_NOT_ORTHONORMAL;
    }
  return LTMP2_OK;
}

int build_k(const ltmp2_kpoint_system *sys, HostPlan &hp, KPointHost &kh) {
  if (!sys || !sys->miller || !sys->coeff || !sys->eps) return LTMP2_ERR_INVALID_ARG;
  if (sys->n_pw < 2 || sys->n_orb < 2 || sys->n_occ < 1 || sys->n_occ >= sys->n_orb || sys->n_orb > sys->n_pw)
    return LTMP2_ERR_INVALID_ARG;
  if (sys->precision != LTMP2_FP64 && sys->precision != LTMP2_FP32) return LTMP2_ERR_INVALID_ARG;
  if (sys->flags != 0) return LTMP2_ERR_INVALID_ARG;
  for (int k = 0; k < 9; ++k)
    if (!std::isfinite(sys->lattice[k])) return LTMP2_ERR_INVALID_ARG;
  if (!std::isfinite(sys->ecut_aux)) return LTMP2_ERR_INVALID_ARG;
  int nk = 1;
  for (int a = 0; a < 3; ++a) {
    if (sys->mesh[a] < 1 || sys->mesh[a] > 64) return LTMP2_ERR_INVALID_ARG;
    nk *= sys->mesh[a];
  }
  if (nk > 64) return LTMP2_ERR_INVALID_ARG;
  const int n = sys->grid[0];
  if (sys->grid[1] != n || sys->grid[2] != n || !fft_size_supported(n)) return LTMP2_ERR_GRID;
  const int no = sys->n_occ, npw = sys->n_pw, norb = sys->n_orb;
  double homo = -1e300, lumo = 1e300;
  for (int k = 0; k < nk; ++k) {
    const double *e = sys->eps + (size_t)k * norb;
    for (int a = 0; a < norb; ++a) {
      if (!std::isfinite(e[a])) return LTMP2_ERR_INVALID_ARG;
      if (a > 0 && e[a] < e[a - 1]) return LTMP2_ERR_INVALID_ARG;
    }
    homo = std::max(homo, e[no - 1]);
    lumo = std::min(lumo, e[no]);
  }
  if (lumo - homo < 1e-6) return LTMP2_ERR_GAP;
  double omega = 0.0;
  if (!reciprocal(sys->lattice, hp.B, &omega)) return LTMP2_ERR_INVALID_ARG;
  Hash h;
  h.bytes(sys->lattice, sizeof(sys->lattice));
  h.bytes(sys->grid, sizeof(sys->grid));
  h.bytes(sys->mesh, sizeof(sys->mesh));
  const int sizes[4] = {npw, norb, no, sys->precision};
  h.bytes(sizes, sizeof(sizes));
  h.bytes(sys->miller, sizeof(int) * 3 * (size_t)npw);
  h.bytes(sys->eps, sizeof(double) * (size_t)norb * nk);
  {
    const size_t cnt = 2 * (size_t)nk * norb * npw;
    for (size_t k = 0; k < cnt; ++k) {
      if (!std::isfinite(sys->coeff[k])) return LTMP2_ERR_INVALID_ARG;
      uint64_t w;
      std::memcpy(&w, sys->coeff + k, 8);
      h.word(w);
    }
  }
  std::vector<std::array<int, 3>> m(npw);
  std::map<std::array<int, 3>, int> where;
  double g2max = 0.0;
  for (int q = 0; q < npw; ++q) {
    for (int a = 0; a < 3; ++a) {
      m[q][a] = sys->miller[3 * q + a];
      if (2 * std::abs(m[q][a]) >= n) return LTMP2_ERR_GRID;
    }
    if (!where.emplace(m[q], q).second) return LTMP2_ERR_INVALID_ARG;
    g2max = std::max(g2max, g2_of(hp.B, m[q][0], m[q][1], m[q][2]));
  }
  std::vector<Col> ocols;
  if (!build_columns(m, ocols, hp.order)) return LTMP2_ERR_GRID;
  for (int k = 0; k < nk; ++k) {
    const int rc = check_orthonormal(sys->coeff + (size_t)k * norb * npw * 2, norb, npw, no);
    if (rc) return rc;
  }
  const double ecut_aux = sys->ecut_aux > 0.0 ? sys->ecut_aux : (2.0 / 3.0) * 0.5 * g2max;
  const double raux = std::sqrt(2.0 * ecut_aux);
  // the largest class shift |B^T delta / n|, delta_a in (-n_a, n_a)
  double smax = 0.0;
  for (int c = 0; c < 8; ++c) {
    double f[3];
    for (int a = 0; a < 3; ++a) f[a] = ((c >> a) & 1 ? 1.0 : -1.0) * (sys->mesh[a] - 1) / (double)sys->mesh[a];
    double x = 0, y = 0, z = 0;
    for (int a = 0; a < 3; ++a) {
      x += f[a] * hp.B[3 * a];
      y += f[a] * hp.B[3 * a + 1];
      z += f[a] * hp.B[3 * a + 2];
    }
    smax = std::max(smax, std::sqrt(x * x + y * y + z * z));
  }
  // auxiliary set: the ball |B^T g| <= R_aux + smax (every class's shifted sphere inside it)
  const double rball = raux + smax + 1e-9;
  std::vector<std::array<int, 3>> am;
  int lim[3];
  for (int a = 0; a < 3; ++a) {
    const double *av = sys->lattice + 3 * a;
    lim[a] = (int)std::floor(rball * std::sqrt(av[0] * av[0] + av[1] * av[1] + av[2] * av[2]) /
                             6.283185307179586476925286766559) + 1;
  }
  for (int a = -lim[0]; a <= lim[0]; ++a)
    for (int b = -lim[1]; b <= lim[1]; ++b)
      for (int d = -lim[2]; d <= lim[2]; ++d)
        if (g2_of(hp.B, a, b, d) <= rball * rball) {
          if (2 * std::abs(a) >= n || 2 * std::abs(b) >= n || 2 * std::abs(d) >= n) return LTMP2_ERR_GRID;
          am.push_back({a, b, d});
        }
  std::vector<Col> acols;
  std::vector<int> aorder;
  if (!build_columns(am, acols, aorder)) return LTMP2_ERR_GRID;
  const int naux = (int)am.size();
  std::vector<std::array<int, 3>> amo(naux);
  for (int q = 0; q < naux; ++q) amo[q] = am[aorder[q]];
  kh.lut.assign((size_t)n * n * n, -1);
  for (int q = 0; q < naux; ++q) {
    auto w = [n](int x) { return ((x % n) + n) % n; };
    kh.lut[((size_t)w(amo[q][2]) * n + w(amo[q][1])) * n + w(amo[q][0])] = q;
  }
  // Coulomb kernel of every class delta (components in (-n_a, n_a))
  const int c0 = 2 * sys->mesh[0] - 1, c1 = 2 * sys->mesh[1] - 1, c2 = 2 * sys->mesh[2] - 1;
  kh.vcls64.assign((size_t)c0 * c1 * c2 * naux, 0.0);
  kh.vcls32.assign(kh.vcls64.size(), 0.f);
  for (int i0 = 0; i0 < c0; ++i0)
    for (int i1 = 0; i1 < c1; ++i1)
      for (int i2 = 0; i2 < c2; ++i2) {
        const double f[3] = {(i0 - (sys->mesh[0] - 1)) / (double)sys->mesh[0],
                             (i1 - (sys->mesh[1] - 1)) / (double)sys->mesh[1],
                             (i2 - (sys->mesh[2] - 1)) / (double)sys->mesh[2]};
        const size_t base = (((size_t)i0 * c1 + i1) * c2 + i2) * naux;
        for (int q = 0; q < naux; ++q) {
          double x = 0, y = 0, z = 0;
          for (int a = 0; a < 3; ++a) {
            const double t = amo[q][a] + f[a];
            x += t * hp.B[3 * a];
            y += t * hp.B[3 * a + 1];
            z += t * hp.B[3 * a + 2];
          }
          const double q2 = x * x + y * y + z * z;
          if (q2 > 1e-20 && 0.5 * q2 <= ecut_aux) {
            kh.vcls64[base + q] = 12.566370614359172953850573533118 / q2;
            kh.vcls32[base + q] = (float)kh.vcls64[base + q];
          }
        }
      }
  // primary supercell transfers Q' = B^T (M / n), |Q'|^2/2 <= E_aux, first non-zero M > 0
  kh.prim_m.clear();
  kh.vprim.clear();
  {
    int ml[3];
    for (int a = 0; a < 3; ++a) ml[a] = (lim[a] + 1) * sys->mesh[a];
    for (int a = 0; a <= ml[0]; ++a)
      for (int b = -ml[1]; b <= ml[1]; ++b)
        for (int d = -ml[2]; d <= ml[2]; ++d) {
          const std::array<int, 3> M = {a, b, d};
          if (!primary(M)) continue;
          double x = 0, y = 0, z = 0;
          for (int c = 0; c < 3; ++c) {
            const double t = M[c] / (double)sys->mesh[c];
            x += t * hp.B[3 * c];
            y += t * hp.B[3 * c + 1];
            z += t * hp.B[3 * c + 2];
          }
          const double q2 = x * x + y * y + z * z;
          if (q2 > 1e-20 && 0.5 * q2 <= ecut_aux) {
            kh.prim_m.insert(kh.prim_m.end(), {a, b, d});
            kh.vprim.push_back(12.566370614359172953850573533118 / q2);
          }
        }
  }
  if (kh.vprim.empty()) return LTMP2_ERR_INVALID_ARG;
  h.bytes(&ecut_aux, sizeof(ecut_aux));
  hp.fingerprint = h.h;
  hp.ecut_aux = ecut_aux;

  Plan &p = hp.p;
  p = Plan();
  p.n = n;
  p.nk = nk;
  for (int a = 0; a < 3; ++a) p.mesh[a] = sys->mesh[a];
  p.no_k = no;
  p.n_occ = nk * no;
  p.n_orb = norb;
  p.n_pw = npw;
  p.n_v = norb - no;
  p.n_dorb = (int)ocols.size();
  p.n_daux = (int)acols.size();
  p.n_aux = naux;
  p.n_prim = (int)kh.vprim.size();
  p.real_orb = false;
  p.real_basis = false;
  p.precision = sys->precision;
  p.omega = omega;
  p.mu = 0.5 * (homo + lumo);
  p.mxlo_orb = ocols.front().m1;
  p.mxhi_orb = ocols.back().m1;
  p.mxlo_aux = acols.front().m1;
  p.mxhi_aux = acols.back().m1;
  hp.dorb.resize(p.n_dorb);
  hp.dorb_off.resize(p.n_dorb);
  hp.daux.resize(p.n_daux);
  hp.daux_off.resize(p.n_daux);
  for (int d = 0; d < p.n_dorb; ++d) {
    hp.dorb[d] = make_int4(ocols[d].m1, ocols[d].m2, ocols[d].zlo, ocols[d].zhi);
    hp.dorb_off[d] = ocols[d].off;
  }
  for (int d = 0; d < p.n_daux; ++d) {
    hp.daux[d] = make_int4(acols[d].m1, acols[d].m2, acols[d].zlo, acols[d].zhi);
    hp.daux_off[d] = acols[d].off;
  }
  hp.pw_m.resize(3 * (size_t)npw);
  hp.aux_m.resize(3 * (size_t)naux);
  for (int q = 0; q < npw; ++q)
    for (int a = 0; a < 3; ++a) hp.pw_m[3 * q + a] = m[hp.order[q]][a];
  for (int q = 0; q < naux; ++q)
    for (int a = 0; a < 3; ++a) hp.aux_m[3 * q + a] = amo[q][a];
  hp.pw_pair.clear();
  hp.aux_neg.clear();
  hp.prim.clear();
  hp.v64.clear();
  hp.v32.clear();
  hp.aux_g2.clear();
  return LTMP2_OK;
}

}  // namespace

int build_host_plan(const ltmp2_system *sys, int allowed_flags, HostPlan &hp) noexcept {
  try {
    return build(sys, allowed_flags, hp);
  } catch (const std::bad_alloc &) {
    return LTMP2_ERR_OOM;
  } catch (...) {
    return LTMP2_ERR_INVALID_ARG;
  }
}

}  // namespace ltmp2

namespace ltmp2 {
int build_kpoint_host_plan(const ltmp2_kpoint_system *sys, HostPlan &hp, KPointHost &kh) noexcept {
  try {
    return build_k(sys, hp, kh);
  } catch (const std::bad_alloc &) {
    return LTMP2_ERR_OOM;
  } catch (...) {
    return LTMP2_ERR_INVALID_ARG;
  }
}
}  // namespace ltmp2

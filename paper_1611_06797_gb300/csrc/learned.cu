// Learned form of the hot path (the paper has no counterpart): weak occupied pairs are
// left out of the exchange contraction (step (iv.b) of Sec. III A, the N_o^2 co-densities
// per G') and their exchange energy is estimated by the pair-energy model; the direct term
// (step (iv.a)) stays exact for every pair.  The model predicts ln|e^x_ij| of an unordered
// pair (both orders, i < j) from the cheap descriptors of ltmp2_pair_descriptors; it is
// trained on labels that the exact contraction produces (ltmp2_learned_training_data).
// Pairs are screened in ascending order of a calibrated upper bound (the estimate times a
// margin that the caller validates on held-out systems) while the screened sum stays within
// the caller's budget; the all-pairs contraction remains the reference for the realised error.  Everything
// here runs through this library's own C entry points.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <numeric>
#include <vector>

#include "../../include/ltmp2.h"

namespace {

int sizes_of(ltmp2_ctx *ctx, int *no, int *npairs) {
  int n_aux = 0, n_pw = 0, grid = 0;
  const int rc = ltmp2_sizes(ctx, &n_aux, &n_pw, no, &grid);
  if (rc) return rc;
  *npairs = *no * (*no + 1) / 2;
  return LTMP2_OK;
}

int descriptors_f(ltmp2_ctx *ctx, int npairs, std::vector<float> &X) {
  std::vector<double> d((size_t)npairs * LTMP2_NUM_DESC);
  const int rc = ltmp2_pair_descriptors(ctx, d.data());
  if (rc) return rc;
  X.resize(d.size());
  for (size_t k = 0; k < d.size(); ++k) X[k] = (float)d[k];
  return LTMP2_OK;
}

int training_data(ltmp2_ctx *ctx, int n_tau, const double *tau, const double *w, float *X, float *y) {
  int no = 0, npairs = 0, rc;
  if ((rc = sizes_of(ctx, &no, &npairs))) return rc;
  std::vector<float> Xf;
  if ((rc = descriptors_f(ctx, npairs, Xf))) return rc;
  if ((rc = ltmp2_set_pair_mask(ctx, nullptr))) return rc;
  std::vector<double> pd((size_t)no * no), px((size_t)no * no);
  double ed = 0, ex = 0;
  const int n_prim = ltmp2_num_primary_gprime(ctx);
  if (n_prim < 0) return n_prim;
  if ((rc = ltmp2_energy_partial(ctx, n_tau, tau, w, 0, n_prim, &ed, &ex, pd.data(), px.data()))) return rc;
  size_t r = 0;
  for (int i = 0; i < no; ++i)
    for (int j = i; j < no; ++j, ++r) {
      const double e = i == j ? px[(size_t)i * no + i] : px[(size_t)i * no + j] + px[(size_t)j * no + i];
      y[r] = (float)std::log(std::max(std::fabs(e), 1e-30));
    }
  std::copy(Xf.begin(), Xf.end(), X);
  return LTMP2_OK;
}

int energy_screened(ltmp2_ctx *ctx, const ltmp2_mlp *net, int n_tau, const double *tau, const double *w,
                    double budget, double margin, double *e_direct, double *e_exchange, double *info) {
  int no = 0, npairs = 0, rc;
  if ((rc = sizes_of(ctx, &no, &npairs))) return rc;
  std::vector<float> X, yp(npairs);
  if ((rc = descriptors_f(ctx, npairs, X))) return rc;
  if ((rc = ltmp2_mlp_predict(net, X.data(), npairs, yp.data()))) return rc;
  std::vector<double> sel(npairs), est(npairs);
  for (int r = 0; r < npairs; ++r) {
    est[r] = std::exp((double)yp[r]);   // the estimate that replaces the pair's exchange
    sel[r] = margin * est[r];           // the screening decision: a calibrated upper bound
  }
  std::vector<unsigned char> keep((size_t)no * no);
  int nscr = 0;
  if ((rc = ltmp2_screen_select(no, sel.data(), budget, keep.data(), &nscr, nullptr))) return rc;
  double est_scr = 0.0;
  size_t row = 0;
  for (int i = 0; i < no; ++i)
    for (int j = i; j < no; ++j, ++row)
      if (!keep[(size_t)i * no + j]) est_scr += est[row];
  if ((rc = ltmp2_set_pair_mask(ctx, nscr > 0 ? keep.data() : nullptr))) return rc;
  double ed = 0, ex = 0;
  rc = ltmp2_energy(ctx, n_tau, tau, w, &ed, &ex, nullptr);
  const int rc2 = ltmp2_set_pair_mask(ctx, nullptr);
  if (rc) return rc;
  if (rc2) return rc2;
  *e_direct = ed;
  *e_exchange = ex + est_scr;
  if (info) {
    info[0] = nscr;
    info[1] = est_scr;
    info[2] = ex;
    info[3] = npairs;
  }
  return LTMP2_OK;
}

}  // namespace

extern "C" {

int ltmp2_screen_select(int n_occ, const double *est, double budget, unsigned char *keep, int *n_screened,
                        double *est_screened) {
  if (n_occ < 1 || !est || !keep || !(budget >= 0.0) || !std::isfinite(budget)) return LTMP2_ERR_INVALID_ARG;
  try {
    const int npairs = n_occ * (n_occ + 1) / 2;
    std::vector<int> pi(npairs), pj(npairs), off;
    int r = 0;
    for (int i = 0; i < n_occ; ++i)
      for (int j = i; j < n_occ; ++j, ++r) {
        pi[r] = i;
        pj[r] = j;
        if (!std::isfinite(est[r]) || est[r] < 0.0) return LTMP2_ERR_INVALID_ARG;
        if (i != j) off.push_back(r);
      }
    // ascending estimate; ties by pair index, so the selection is deterministic
    std::stable_sort(off.begin(), off.end(), [&](int a, int b) { return est[a] < est[b]; });
    std::fill(keep, keep + (size_t)n_occ * n_occ, (unsigned char)1);
    double sum = 0.0;
    int n = 0;
    for (int q : off) {
      if (sum + est[q] > budget) break;
      sum += est[q];
      keep[(size_t)pi[q] * n_occ + pj[q]] = 0;
      keep[(size_t)pj[q] * n_occ + pi[q]] = 0;
      ++n;
    }
    if (n_screened) *n_screened = n;
    if (est_screened) *est_screened = sum;
    return LTMP2_OK;
  } catch (const std::bad_alloc &) {
    return LTMP2_ERR_OOM;
  }
}

int ltmp2_learned_training_data(ltmp2_ctx *ctx, int n_tau, const double *tau, const double *w, float *X, float *y) {
  if (!ctx || !tau || !w || n_tau < 1 || !X || !y) return LTMP2_ERR_INVALID_ARG;
  try {
    return training_data(ctx, n_tau, tau, w, X, y);
  } catch (const std::bad_alloc &) {
    return LTMP2_ERR_OOM;
  }
}

int ltmp2_energy_screened(ltmp2_ctx *ctx, const ltmp2_mlp *net, int n_tau, const double *tau, const double *w,
                          double budget, double margin, double *e_direct, double *e_exchange, double *info) {
  if (!ctx || !net || !tau || !w || n_tau < 1 || !e_direct || !e_exchange || !(budget >= 0.0) ||
      !std::isfinite(budget) || !(margin >= 1.0) || !std::isfinite(margin))
    return LTMP2_ERR_INVALID_ARG;
  try {
    return energy_screened(ctx, net, n_tau, tau, w, budget, margin, e_direct, e_exchange, info);
  } catch (const std::bad_alloc &) {
    return LTMP2_ERR_OOM;
  }
}

}  // extern "C"

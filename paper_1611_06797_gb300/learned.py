"""Learned form: screen weak occupied pairs out of the exchange contraction and estimate
their exchange energy with the pair-energy perceptron (ltmp2_mlp_*).

Screening is made safe by a bound.  With the Laplace denominator D_ab = D_ba < 0,
Cauchy-Schwarz gives |e^x_ij| <= |e^d_ij| / 2 for every ordered pair, and the direct
pair energies e^d_ij are computed exactly for all pairs by a cheap diagonal-only
contraction (one co-density per column instead of N_o).  Pairs are screened in
ascending order of |e^d_ij| while the screened sum of |e^d_ij| stays within the
accuracy budget, so dropping their exchange could not exceed the budget; the model
then estimates it.  The model predicts the bounded ratio e^x_ij / (|e^d_ij| / 2),
clipped to [-1, 1], so its estimate never leaves the bound.  Training labels are the
exact kernel's pair energies; the all-pairs contraction stays the fallback and the
reference for the estimate's error.
"""
from __future__ import annotations

import numpy as np

from . import ltmp2 as L


def pair_index(n_occ: int):
    """(i, j) of the unordered pairs in descriptor row order."""
    iu = np.triu_indices(n_occ)
    return iu[0], iu[1]


def direct_pairs(ctx, tau, w):
    """(E_d, e^d [n_occ][n_occ]): exact direct pair energies from a contraction in which
    only the diagonal exchange pairs are kept."""
    n = L.ltmp2_num_primary_gprime(ctx)
    L.ltmp2_set_pair_mask(ctx, np.eye(ctx.n_occ, dtype=bool))
    try:
        ed, _, pd, _ = L.ltmp2_energy_partial(ctx, tau, w, 0, n)
    finally:
        L.ltmp2_set_pair_mask(ctx, None)
    return ed, pd


def ratio(ex, ed_pair):
    return ex / np.maximum(0.5 * np.abs(ed_pair), 1e-300)


def training_data(ctx, tau, w):
    """Descriptors and exact ratios e^x_ij / (|e^d_ij| / 2) of the pairs i <= j."""
    X = L.ltmp2_pair_descriptors(ctx)
    n = L.ltmp2_num_primary_gprime(ctx)
    L.ltmp2_set_pair_mask(ctx, None)
    _, _, pd, px = L.ltmp2_energy_partial(ctx, tau, w, 0, n)
    i, j = pair_index(ctx.n_occ)
    return X, ratio(px[i, j], pd[i, j])


def screen(bound, n_occ: int, budget_ha: float, share: float = 1.0):
    """Keep mask: screen off-diagonal pairs in ascending order of bound_ij = |e^d_ij|
    (>= |2 e^x_ij|, the pair's exchange contribution) while their sum <= share * budget."""
    i, j = pair_index(n_occ)
    b = np.where(i != j, np.abs(bound), np.inf)
    order = np.argsort(b)
    csum = np.cumsum(b[order])
    nscreen = int(np.searchsorted(csum, share * budget_ha, side="right"))
    screened = np.zeros(len(i), dtype=bool)
    screened[order[:nscreen]] = True
    keep = np.ones((n_occ, n_occ), dtype=bool)
    keep[i[screened], j[screened]] = False
    keep[j[screened], i[screened]] = False
    return keep, screened


def screen_fraction(bound, n_occ: int, fraction: float):
    """Keep mask screening the given fraction of off-diagonal pairs with the smallest
    bound, regardless of any budget (a diagnostic of the estimator, not a guarantee)."""
    i, j = pair_index(n_occ)
    off = np.flatnonzero(i != j)
    order = off[np.argsort(np.abs(bound[off]))]
    screened = np.zeros(len(i), dtype=bool)
    screened[order[:int(fraction * len(off))]] = True
    keep = np.ones((n_occ, n_occ), dtype=bool)
    keep[i[screened], j[screened]] = False
    keep[j[screened], i[screened]] = False
    return keep, screened


def screened_energy(ctx, tau, w, mlp, budget_ha: float, share: float = 1.0, fraction=None):
    """E_d exact; E_x = contracted pairs + estimated exchange of the screened pairs.
    fraction: screen that share of the weakest pairs instead of using the budget."""
    X = L.ltmp2_pair_descriptors(ctx)
    _, pd = direct_pairs(ctx, tau, w)
    i, j = pair_index(ctx.n_occ)
    bound = np.abs(pd[i, j])
    if fraction is None:
        keep, screened = screen(bound, ctx.n_occ, budget_ha, share)
    else:
        keep, screened = screen_fraction(bound, ctx.n_occ, fraction)
    r = np.clip(mlp.predict(X).astype(np.float64), -1.0, 1.0)
    est_pairs = r * 0.5 * bound                       # e^x_ij estimates, |.| <= |e^d_ij| / 2
    L.ltmp2_set_pair_mask(ctx, keep)
    try:
        ed, ex, _ = L.ltmp2_energy(ctx, tau, w)
    finally:
        L.ltmp2_set_pair_mask(ctx, None)
    est = float(np.sum(2.0 * est_pairs[screened]))
    return {"E_d": ed, "E_x": ex + est, "E_x_contracted": ex, "E_x_estimated": est,
            "screened_pairs": int(screened.sum()), "pairs": len(i),
            "error_bound_Ha": float(np.sum(bound[screened]))}

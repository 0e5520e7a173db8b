"""Learned form: screen weak occupied pairs out of the exchange contraction and estimate
their exchange energy with the pair-energy perceptron (ltmp2_mlp_*).

The exact kernel labels the training pairs (e^x_ij from ltmp2_energy_partial over the
whole G' range); the direct term stays exact for every pair.  Pairs are screened in
ascending order of predicted |contribution| while the screened total stays within a
given share of the accuracy budget; the all-pairs contraction remains available as the
fallback and the judge of the error.
"""
from __future__ import annotations

import numpy as np

from . import ltmp2 as L

TARGET_SCALE = 1e-6   # Ha: targets are asinh(e^x_ij / TARGET_SCALE)


def pair_index(n_occ: int):
    """(i, j) of the unordered pairs in descriptor row order."""
    iu = np.triu_indices(n_occ)
    return iu[0], iu[1]


def training_data(ctx, tau, w):
    """Descriptors and exact exchange pair energies e^x_ij (i <= j) of one system."""
    X = L.ltmp2_pair_descriptors(ctx)
    n = L.ltmp2_num_primary_gprime(ctx)
    L.ltmp2_set_pair_mask(ctx, None)
    _, _, _, ex = L.ltmp2_energy_partial(ctx, tau, w, 0, n)
    i, j = pair_index(ctx.n_occ)
    return X, ex[i, j]


def encode(ex):
    return np.arcsinh(np.asarray(ex) / TARGET_SCALE)


def decode(y):
    return TARGET_SCALE * np.sinh(np.asarray(y, dtype=np.float64))


def screen(pred_ex, n_occ: int, budget_ha: float, share: float = 1.0):
    """Keep mask: screen pairs with the smallest predicted |contribution| (2 e^x_ij off the
    diagonal) while their summed magnitude stays <= share * budget_ha."""
    i, j = pair_index(n_occ)
    contrib = np.where(i == j, 1.0, 2.0) * np.abs(pred_ex)
    order = np.argsort(contrib)
    csum = np.cumsum(contrib[order])
    nscreen = int(np.searchsorted(csum, share * budget_ha, side="right"))
    screened = np.zeros(len(i), dtype=bool)
    screened[order[:nscreen]] = True
    screened &= (i != j)              # the diagonal is always contracted
    keep = np.ones((n_occ, n_occ), dtype=bool)
    keep[i[screened], j[screened]] = False
    keep[j[screened], i[screened]] = False
    return keep, screened


def screened_energy(ctx, tau, w, mlp, budget_ha: float, share: float = 1.0):
    """E_d exact; E_x = contracted pairs + predicted exchange of the screened pairs."""
    X = L.ltmp2_pair_descriptors(ctx)
    pred = decode(mlp.predict(X))
    keep, screened = screen(pred, ctx.n_occ, budget_ha, share)
    L.ltmp2_set_pair_mask(ctx, keep)
    try:
        ed, ex, _ = L.ltmp2_energy(ctx, tau, w)
    finally:
        L.ltmp2_set_pair_mask(ctx, None)
    i, _ = pair_index(ctx.n_occ)
    est = float(np.sum(2.0 * pred[screened]))    # screened pairs are off-diagonal
    return {"E_d": ed, "E_x": ex + est, "E_x_contracted": ex, "E_x_estimated": est,
            "screened_pairs": int(screened.sum()), "pairs": len(i)}

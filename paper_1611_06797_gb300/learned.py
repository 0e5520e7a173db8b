"""Learned form through the C ABI (argument marshalling only; include/ltmp2.h).

The library screens weak exchange pairs and estimates their exchange with the pair model
(``ltmp2_energy_screened``).  This module gathers training sets (``ltmp2_learned_training_data``:
descriptors and the exact ln|e^x_ij| labels of each system), trains the model (``Mlp``) and
calibrates the screening margin by leave-one-system-out validation: for each training system
a model trained on the others predicts it, and the margin is the largest ratio |e^x| / estimate
among the lowest predictions of any held-out system (the pairs a screening would take), times
a safety factor.  The all-pairs contraction stays the reference for the realised error.
"""
from __future__ import annotations

import numpy as np

from . import ltmp2 as L


def training_sets(ctxs_and_quads):
    """[(X, y), ...] per system for [(ctx, tau, w), ...]."""
    return [L.ltmp2_learned_training_data(ctx, tau, w) for ctx, tau, w in ctxs_and_quads]


def train(sets, epochs: int = 4000, lr: float = 3e-3, seed: int = 5) -> "L.Mlp":
    X = np.concatenate([x for x, _ in sets])
    y = np.concatenate([v for _, v in sets])
    net = L.Mlp(seed=seed)
    net.loss = net.train(X, y, epochs=epochs, lr=lr)
    net.samples = int(len(y))
    return net


def calibrate_margin(sets, epochs: int = 4000, lowest: float = 0.02, safety: float = 2.0, seed: int = 5) -> float:
    """Leave-one-system-out margin for the screening decision (see the module docstring):
    max over held-out systems of |e^x| / exp(prediction) among the ``lowest`` fraction of
    off-diagonal pairs by prediction, times ``safety``; at least 1."""
    worst = 1.0
    for k in range(len(sets)):
        rest = [s for q, s in enumerate(sets) if q != k]
        if not rest:
            continue
        net = train(rest, epochs=epochs, seed=seed)
        X, y = sets[k]
        off = X[:, 6] == 0
        if not off.any():
            net.destroy()
            continue
        pred = net.predict(X[off]).astype(np.float64)
        net.destroy()
        n = max(1, int(lowest * off.sum()))
        low = np.argsort(pred)[:n]
        worst = max(worst, float(np.max(np.exp(y[off][low].astype(np.float64) - pred[low]))))
    return worst * safety


def screened_vs_exact(ctx, net, tau, w, budget: float, margin: float = 1.0, e_all=None):
    """A screened evaluation and its realised error.  e_all: (E_d, E_x) of the all-pairs
    contraction of the same inputs, or None to run it here."""
    r = L.ltmp2_energy_screened(ctx, net, tau, w, budget, margin)
    if e_all is None:
        ed, ex, _ = L.ltmp2_energy(ctx, tau, w, pairs=False)
        e_all = (ed, ex)
    r["err_E_d"] = abs(r["E_d"] - e_all[0])
    r["err_E_x"] = abs(r["E_x"] - e_all[1])
    return r

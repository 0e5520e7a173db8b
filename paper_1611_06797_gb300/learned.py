"""Learned form through the C ABI (argument marshalling only; include/ltmp2.h).

The library screens weak exchange pairs and estimates their exchange with the pair model
(``ltmp2_energy_screened``); this module gathers training sets from several systems
(``ltmp2_learned_training_data``: descriptors and the exact ln|e^x_ij| labels), trains the
model (``Mlp``) and evaluates the realised error of a screened run against the all-pairs
contraction, which stays the judge.
"""
from __future__ import annotations

import numpy as np

from . import ltmp2 as L


def training_set(ctxs_and_quads):
    """Concatenated (X, y) over [(ctx, tau, w), ...]."""
    Xs, ys = [], []
    for ctx, tau, w in ctxs_and_quads:
        X, y = L.ltmp2_learned_training_data(ctx, tau, w)
        Xs.append(X)
        ys.append(y)
    return np.concatenate(Xs), np.concatenate(ys)


def train(X, y, epochs: int = 4000, lr: float = 3e-3, seed: int = 5) -> "L.Mlp":
    net = L.Mlp(seed=seed)
    net.loss = net.train(X, y, epochs=epochs, lr=lr)
    return net


def screened_vs_exact(ctx, net, tau, w, budget: float, e_all=None):
    """A screened evaluation and its realised error.  e_all: (E_d, E_x) of the all-pairs
    contraction of the same inputs, or None to run it here."""
    r = L.ltmp2_energy_screened(ctx, net, tau, w, budget)
    if e_all is None:
        ed, ex, _ = L.ltmp2_energy(ctx, tau, w, pairs=False)
        e_all = (ed, ex)
    r["err_E_d"] = abs(r["E_d"] - e_all[0])
    r["err_E_x"] = abs(r["E_x"] - e_all[1])
    return r

"""Learned form: screened exchange pairs, pair descriptors and the pair-energy MLP.

* The pair mask is exact bookkeeping: leaving pairs out of the exchange contraction
  changes E_x by exactly their exchange pair energies and leaves E_d unchanged.
* The descriptors obey their definitions (Cauchy-Schwarz for the density overlaps,
  zero self-distance).
* The MLP kernels fit a smooth function.
* The learned form through the C ABI (ltmp2_energy_screened), with the model trained on
  the exact labels of smaller systems (ltmp2_learned_training_data), screens pairs of a
  system it was not trained on and stays within the 0.1 meV/atom budget of the all-pairs
  contraction, which measures it; with a zero budget it is the all-pairs contraction.
"""
import numpy as np
import pytest

import paper_1611_06797_gb300 as L
from paper_1611_06797_gb300 import learned as LF
from oracle import OracleSystem, denominator_range, sinc_laplace_quadrature
from tests.conftest import solid

pytestmark = pytest.mark.gpu
MEV = 1.0 / L.HARTREE_TO_MEV


def _quad(s, n=None):
    return sinc_laplace_quadrature(n or s.spec.n_tau, *denominator_range(OracleSystem.from_solid(s)))


@pytest.mark.parametrize("real", [True, False])
def test_pair_mask_removes_exactly_the_screened_exchange(real):
    s = solid("tiny2")
    tau, w = _quad(s, 4)
    ctx = L.setup_from_solid(s, real=real)
    n = L.ltmp2_num_primary_gprime(ctx)
    ed, ex, pd, px = L.ltmp2_energy_partial(ctx, tau, w, 0, n)
    keep = np.ones((s.n_occ, s.n_occ), dtype=bool)
    keep[0, 2] = keep[2, 0] = keep[1, 3] = keep[3, 1] = False
    L.ltmp2_set_pair_mask(ctx, keep)
    ed2, ex2, pd2, px2 = L.ltmp2_energy_partial(ctx, tau, w, 0, n)
    L.ltmp2_set_pair_mask(ctx, None)
    removed = px[~keep].sum()
    assert abs(ed2 - ed) < 1e-13 * abs(ed)
    assert abs(ex2 - (ex - removed)) < 1e-12 * abs(ex)
    assert np.all(px2[~keep] == 0.0)
    assert np.abs(px2[keep] - px[keep]).max() < 1e-14
    with pytest.raises(L.Ltmp2Error):   # the diagonal is always contracted
        bad = np.ones_like(keep)
        bad[1, 1] = False
        L.ltmp2_set_pair_mask(ctx, bad)


def test_pair_descriptors_follow_their_definitions():
    s = solid("cfg1")
    ctx = L.setup_from_solid(s, real=True)
    d = L.ltmp2_pair_descriptors(ctx)
    i, j = np.triu_indices(s.n_occ)
    assert d.shape == (len(i), L.NUM_DESC) and np.all(np.isfinite(d))
    # overlaps against a direct real-space evaluation of (1/N) sum |u_i|^2 |u_j|^2
    n = int(s.grid[0])
    g = np.zeros((s.n_occ, n, n, n), dtype=complex)
    m = np.mod(s.miller, n)
    g[:, m[:, 0], m[:, 1], m[:, 2]] = s.coeff[:s.n_occ]
    rho = np.abs(np.fft.ifftn(g, axes=(1, 2, 3)) * n ** 3) ** 2
    S = np.einsum("axyz,bxyz->ab", rho, rho) / n ** 3
    assert np.abs(d[:, 2] - np.log10(S[i, j] / np.sqrt(S[i, i] * S[j, j]))).max() < 1e-9
    assert np.all(d[:, 2] <= 1e-12)                       # Cauchy-Schwarz
    diag = i == j
    assert np.all(d[diag, 3] < 1e-9) and np.all(d[diag, 6] == 1.0) and np.all(d[~diag, 6] == 0.0)
    assert np.all(d[:, 0] <= d[:, 1] + 1e-15)


def test_mlp_fits_a_smooth_function():
    rng = np.random.default_rng(0)
    X = rng.uniform(-1, 1, size=(2000, 4)).astype(np.float32)
    y = (np.sin(2 * X[:, 0]) + X[:, 1] * X[:, 2] - 0.5 * X[:, 3] ** 2).astype(np.float32)
    net = L.Mlp(n_in=4, width=32, seed=3)
    loss = net.train(X, y, epochs=1500, lr=3e-3)
    assert loss < 0.01
    pred = net.predict(X[:200])
    assert np.abs(pred - y[:200]).max() < 0.25


def test_learned_screening_within_budget_on_unseen_system():
    train = [solid(n) for n in ("cfg1", "batch0", "batch1", "batch2", "batch3", "batch4")]
    ctxs = [(L.setup_from_solid(s, precision=L.FP32, real=True), *_quad(s)) for s in train]
    sets = LF.training_sets(ctxs)
    for c, _, _ in ctxs:
        L.ltmp2_destroy(c)
    for X, y in sets:
        assert np.all(np.isfinite(y)) and X.shape == (len(y), L.NUM_DESC)
    margin = LF.calibrate_margin(sets, epochs=3000, seed=11)
    net = LF.train(sets, epochs=3000, seed=11)
    assert margin >= 2.0 and net.residual() > 0.0
    s = solid("batch5")
    tau, w = _quad(s)
    c = L.setup_from_solid(s, precision=L.FP32, real=True)
    ed, ex, _ = L.ltmp2_energy(c, tau, w, pairs=False)
    budget = 0.1 * MEV * s.n_atoms
    # the 0.1 meV/atom budget and larger ones: the realised error, measured by the all-pairs
    # contraction, stays within each budget; the largest certainly screens pairs
    for b in (budget, 10 * budget, 100 * budget):
        r = LF.screened_vs_exact(c, net, tau, w, b, margin, e_all=(ed, ex))
        assert abs(r["E_d"] - ed) < 1e-9 * abs(ed)
        assert abs(r["E_d"] + r["E_x"] - ed - ex) < b, (b, margin, r, ed, ex)
    assert r["screened_pairs"] > 0 and r["E_x_contracted"] < ex
    # a zero budget screens nothing: the all-pairs contraction itself
    r0 = LF.screened_vs_exact(c, net, tau, w, 0.0, margin, e_all=(ed, ex))
    assert r0["screened_pairs"] == 0 and r0["err_E_x"] < 1e-12 * abs(ex) and r0["err_E_d"] < 1e-12 * abs(ed)
    L.ltmp2_destroy(c)

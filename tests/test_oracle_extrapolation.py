"""Pins of the oracle's internal auxiliary-cutoff extrapolation (Sec. III D, Eq. CutDecay
of arXiv:1611.06797): nested cutoffs E_aux[n] = E_aux / alpha^(n-1), the MP2 energy
with every auxiliary G-sum truncated at each of them, and the straight-line fit of
E[n] against E_aux[n]^(-3/2) whose intercept is the extrapolated energy."""
import math

import numpy as np
import pytest

from oracle import (OracleSystem, aux_set, canonical_denominator, cutoff_extrapolation,
                    cutoff_levels, denominator_range, laplace_denominator, level_energies,
                    mp2_energy, sinc_laplace_quadrature)
from synth import free_electron_solid
from tests.conftest import solid
from tests.test_oracle_pins import _box_aux


def test_cutoff_levels_are_the_nested_geometric_sequence():
    e = cutoff_levels(7.0, 8, 1.05)
    assert e[0] == 7.0 and len(e) == 8
    assert np.allclose(e[1:] / e[:-1], 1.0 / 1.05, rtol=1e-15, atol=0.0)
    with pytest.raises(ValueError):
        cutoff_levels(7.0, 8, 1.0)


def test_fit_recovers_an_exact_cutdecay_law():
    ecut = cutoff_levels(9.0, 8, 1.05)
    a0, b0 = -0.731, 4.2
    a, b, sa = cutoff_extrapolation(ecut, a0 + b0 * ecut ** -1.5)
    assert abs(a - a0) < 1e-12 and abs(b - b0) < 1e-10 * b0 and sa < 1e-12


def test_fit_matches_an_independent_least_squares_solve():
    rng = np.random.default_rng(3)
    ecut = cutoff_levels(6.0, 8, 1.07)
    y = -1.3 + 2.0 * ecut ** -1.5 + 1e-4 * rng.standard_normal(8)
    a, b, sa = cutoff_extrapolation(ecut, y)
    X = np.stack([np.ones(8), ecut ** -1.5], 1)
    coef, res, _, _ = np.linalg.lstsq(X, y, rcond=None)
    assert abs(a - coef[0]) < 1e-12 and abs(b - coef[1]) < 1e-9
    cov = float(res[0]) / (8 - 2) * np.linalg.inv(X.T @ X)
    assert abs(sa - math.sqrt(cov[0, 0])) < 1e-6 * sa


def test_level_energies_free_electron_closed_form():
    """V = 0, one occupied orbital: at every level E_d[n] = -(32 pi^2/Omega^2) sum over
    A_n of 1/|G|^6 and E_x[n] = -E_d[n]/2; |A_n| is the lattice-point count."""
    a, grid, r2 = 5.5, 12, 9
    s = free_electron_solid(a, grid, r2, n_occ=1)
    o = OracleSystem.from_solid(s)
    ecut, counts, ed, ex = level_energies(o, canonical_denominator, 8, 1.05)
    omega = a ** 3
    for n in range(8):
        A = _box_aux(a, grid, ecut[n])
        cf = -(32 * math.pi ** 2 / omega ** 2) * sum(1.0 / g2 ** 3 for _, g2 in A)
        assert counts[n] == len(A)
        assert abs(ed[n] - cf) < 1e-12 * abs(cf)
        assert abs(ex[n] + 0.5 * cf) < 1e-12 * abs(cf)
    assert all(np.diff(counts) <= 0) and counts[-1] < counts[0]


def _lattice_sum(a, ecut):
    """sum over 0 < |G|^2/2 <= ecut of 1/|G|^6 on the simple-cubic reciprocal lattice."""
    L = int(math.sqrt(2 * ecut) * a / (2 * math.pi)) + 1
    r = np.arange(-L, L + 1)
    m = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3)
    g2 = (2 * math.pi / a) ** 2 * (m ** 2).sum(1)
    k = (g2 > 0) & (0.5 * g2 <= ecut)
    return float(np.sum(1.0 / g2[k] ** 3))


@pytest.mark.parametrize("a,ecut", [(12.0, 10.0), (20.0, 10.0)])
def test_extrapolation_reaches_the_infinite_cutoff_limit(a, ecut):
    """The free-electron direct energy is -(32 pi^2/Omega^2) times the lattice sum of
    1/|G|^6, whose tail beyond |G| = K is (Omega/(2 pi)^3) 4 pi/(3 K^3) ~ E_aux^(-3/2)
    (Eq. CutDecay).  The limit is the sum at a large cutoff plus that tail; the
    extrapolation from eight levels must land far closer to it than the raw value and
    within three fitted standard errors."""
    big = 150.0 if a < 15 else 60.0
    K = math.sqrt(2 * big)
    s_inf = _lattice_sum(a, big) + a ** 3 / (2 * math.pi) ** 3 * 4 * math.pi / (3 * K ** 3)
    e = cutoff_levels(ecut, 8, 1.05)
    y = [_lattice_sum(a, x) for x in e]
    ext, _, sa = cutoff_extrapolation(e, y)
    assert abs(ext - s_inf) < 0.05 * abs(y[0] - s_inf)
    assert abs(ext - s_inf) < 3.0 * sa


def test_level_one_is_the_plain_energy_and_levels_nest():
    s = solid("tiny2")
    o = OracleSystem.from_solid(s)
    tau, w = sinc_laplace_quadrature(6, *denominator_range(o))
    D = laplace_denominator(tau, w)
    ecut, counts, ed, ex = level_energies(o, D, 3, 1.25)
    r = mp2_energy(o, D)
    assert ed[0] == r["E_d"] and ex[0] == r["E_x"]
    assert counts[0] == len(aux_set(o)[0]) and counts[0] > counts[1] > counts[2]
    # each level is the calculation with the smaller cutoff, and A_n is nested
    m0 = {tuple(x) for x in aux_set(o)[0]}
    for n in (1, 2):
        o_n = OracleSystem.from_solid(s, ecut_aux=float(ecut[n]))
        assert {tuple(x) for x in aux_set(o_n)[0]} <= m0
        assert abs(mp2_energy(o_n, D)["E_d"] - ed[n]) == 0.0

"""Pins of the oracle's spin-unrestricted MP2 (Eqs. MP2direct, MP2exchange with their
spin sums s, s' kept): the closed-shell limit, the spin-orbital antisymmetrised form
E = 1/4 sum_{IJAB} |<IJ||AB>|^2 / Delta by brute force, and a single electron, whose
direct and exchange energies cancel exactly."""
import numpy as np
import pytest

from oracle import (OracleSystem, aux_set, canonical_denominator, denominator_range, laplace_denominator,
                    mp2_energy, overlap_densities_conv, pair_integrals, sinc_laplace_quadrature, uhf_mp2_energy)
from oracle.ltmp2_oracle import _neg_index
from synth import SPECS, spin_polarized_pair
from tests.conftest import solid


def _pair(name, na, nb, real=True):
    a, b = spin_polarized_pair(SPECS[name], na, nb, real_orbitals=real)
    return OracleSystem.from_solid(a), OracleSystem.from_solid(b)


@pytest.mark.parametrize("mode", ["canonical", "laplace"])
def test_closed_shell_limit(mode):
    o = OracleSystem.from_solid(solid("tiny2"))
    D = canonical_denominator if mode == "canonical" else \
        laplace_denominator(*sinc_laplace_quadrature(6, *denominator_range(o)))
    r = mp2_energy(o, D)
    u = uhf_mp2_energy(o, o, D)
    assert abs(u["E_d"] - r["E_d"]) < 1e-12 * abs(r["E_d"])
    assert abs(u["E_x"] - r["E_x"]) < 1e-12 * abs(r["E_x"])
    assert abs(u["E_aa"] - u["E_bb"]) < 1e-14 and abs(u["E_aa"] + u["E_bb"] + u["E_ab"] - u["E"]) < 1e-14


def test_spin_orbital_antisymmetrised_form():
    sa, sb = _pair("tiny", 2, 1)
    u = uhf_mp2_energy(sa, sb, canonical_denominator)
    spins = [sa, sb]
    mG, _, v = aux_set(sa)
    neg = _neg_index(mG)
    # spatial <ij|ab> for every spin combination of (i, a) and (j, b)
    rho = [overlap_densities_conv(s, list(range(s.n_occ)), list(range(s.coeff.shape[0])), mG) for s in spins]
    occ = [(s, i) for s in (0, 1) for i in range(spins[s].n_occ)]
    vir = [(s, a) for s in (0, 1) for a in range(spins[s].n_occ, spins[s].coeff.shape[0])]
    ev = np.array([spins[s].eps[a] for s, a in vir])
    sv = np.array([s for s, _ in vir])
    av = np.array([a for _, a in vir])
    E = 0.0
    for (si, i) in occ:
        for (sj, j) in occ:
            K = pair_integrals(rho[si][i], rho[sj][j][:, neg], v, sa.omega)   # K[a', b'] over all orbitals
            # <IJ|AB> = delta(s_I, s_A) delta(s_J, s_B) <ij|ab>
            direct = np.where((sv[:, None] == si) & (sv[None, :] == sj), K[av[:, None], av[None, :]], 0.0)
            # <IJ|BA> = delta(s_I, s_B) delta(s_J, s_A) <ij|ba>
            swap = np.where((sv[None, :] == si) & (sv[:, None] == sj), K[av[None, :], av[:, None]], 0.0)
            anti = direct - swap
            delta = spins[si].eps[i] + spins[sj].eps[j] - ev[:, None] - ev[None, :]
            E += 0.25 * float(np.sum(np.abs(anti) ** 2 / delta))
    assert abs(u["E"] - E) < 1e-12 * abs(E)


@pytest.mark.parametrize("mode", ["canonical", "laplace"])
def test_one_electron_has_no_correlation(mode):
    sa, sb = _pair("tiny", 1, 0)
    D = canonical_denominator if mode == "canonical" else \
        laplace_denominator(*sinc_laplace_quadrature(6, *denominator_range(sa)))
    u = uhf_mp2_energy(sa, sb, D)
    assert abs(u["E_d"]) > 1e-6
    assert abs(u["E"]) < 1e-14 * abs(u["E_d"]) + 1e-16

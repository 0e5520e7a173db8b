"""Pins of the k-point oracle (Sec. II C-D: Eqs. MP2direct / MP2exchange per unit cell,
Eq. 2eIPLWV with crystal-momentum conservation), each against something other than the
k-point code itself:

* a 1 x 1 x 1 mesh is the Gamma-point oracle;
* an n1 x n2 x n3 mesh equals the Gamma-point oracle on the supercell n1 a x n2 a x n3 a
  built from the same potential (its own plane-wave set, its own dense diagonalisation,
  which mixes nothing because the supercell Hamiltonian is block diagonal in k), per cell,
  canonical and with the Laplace denominator: the Born-von Karman identity behind the
  1/N sum over the Brillouin zone;
* free electrons with one occupied plane wave per k: a brute-force sum over plane-wave
  momenta p_i + p_j = p_a + p_b with v(p_a - p_i) (no overlap densities, no orbitals);
* random phases of the Bloch orbitals change nothing, and e_{(i k1),(j k2)} is symmetric.
"""
import math

import numpy as np
import pytest

from oracle import (KPointOracleSystem, OracleSystem, canonical_denominator, denominator_range,
                    kpoint_mp2_energy, laplace_denominator, mp2_energy, sinc_laplace_quadrature)
from synth import build_kpoint_pair, build_kpoint_solid, free_electron_kpoints

POS = np.array([[1.1, 2.3, 2.0]])


def _quad(ks):
    lo = 2.0 * ks.gap
    hi = 2.0 * ks.width
    return sinc_laplace_quadrature(8, lo, hi)


def test_one_kpoint_mesh_is_the_gamma_oracle():
    ks = build_kpoint_solid(5.0, 8, 9, (1, 1, 1), POS, 2, seed=1)
    ko = KPointOracleSystem.from_solid(ks)
    g = OracleSystem(ks.lattice, ks.grid, ks.miller, ks.coeff[0], ks.eps[0], ks.n_occ, ko.ecut_aux)
    tau, w = _quad(ks)
    for D in (laplace_denominator(tau, w), canonical_denominator):
        rk = kpoint_mp2_energy(ko, D)
        rg = mp2_energy(g, D)
        assert abs(rk["E_d"] - rg["E_d"]) < 1e-13 * abs(rg["E_d"])
        assert abs(rk["E_x"] - rg["E_x"]) < 1e-13 * abs(rg["E_x"])


@pytest.mark.parametrize("mesh,phases", [((2, 1, 1), False), ((1, 2, 1), True), ((3, 1, 1), False)])
def test_mesh_equals_gamma_supercell(mesh, phases):
    ks, sc = build_kpoint_pair(5.0, 8, 9, mesh, POS, 1, random_phases=phases, seed=4)
    assert ks.gap > 1e-3 and abs(sc.gap - ks.gap) < 1e-10     # the occupied sets coincide
    ko = KPointOracleSystem.from_solid(ks)
    so = OracleSystem.from_solid(sc, ecut_aux=ko.ecut_aux)
    nk = ks.n_k
    tau, w = _quad(ks)
    for D in (laplace_denominator(tau, w), canonical_denominator):
        rk = kpoint_mp2_energy(ko, D)
        rs = mp2_energy(so, D)
        assert rk["E_d"] < 0
        assert abs(rk["E_d"] - rs["E_d"] / nk) < 1e-12 * abs(rk["E_d"]), (rk["E_d"], rs["E_d"] / nk)
        assert abs(rk["E_x"] - rs["E_x"] / nk) < 1e-12 * abs(rk["E_x"]), (rk["E_x"], rs["E_x"] / nk)


def test_phases_and_pair_symmetry():
    a = build_kpoint_solid(5.0, 8, 9, (2, 1, 1), POS, 2, seed=6)
    b = build_kpoint_solid(5.0, 8, 9, (2, 1, 1), POS, 2, random_phases=True, seed=6)
    tau, w = _quad(a)
    D = laplace_denominator(tau, w)
    ra = kpoint_mp2_energy(KPointOracleSystem.from_solid(a), D)
    rb = kpoint_mp2_energy(KPointOracleSystem.from_solid(b), D)
    assert abs(ra["E_d"] - rb["E_d"]) < 1e-13 * abs(ra["E_d"])
    assert abs(ra["E_x"] - rb["E_x"]) < 1e-13 * abs(ra["E_x"])
    e = ra["e_d"] + ra["e_x"]
    assert np.abs(e - e.T).max() < 1e-14
    assert np.abs(rb["e_d"] + rb["e_x"] - e).max() < 1e-14


def test_free_electron_kmesh_brute_force():
    """V = 0 on a 3 x 1 x 1 mesh, one occupied plane wave p_k = k + G at every k; virtuals
    are all other plane waves of every k.  <i j|a b> = v(p_a - p_i)/Omega when
    p_i + p_j = p_a + p_b and p_a - p_i is in the auxiliary set, else 0 (grid large enough
    that no product wraps)."""
    a, grid, r2 = 5.5, 16, 6
    ks = free_electron_kpoints(a, grid, r2, (3, 1, 1))
    ko = KPointOracleSystem.from_solid(ks)
    B = ko.recip
    nk = ks.n_k
    omega = nk * ko.omega0
    mom = []       # (k index, cartesian momentum, energy) of every plane wave of every k
    for kk in range(nk):
        order = np.argmax(np.abs(ks.coeff[kk]), axis=1)      # plane wave of each orbital
        for n in range(ks.n_orb):
            p = (ks.miller[order[n]] + ks.kappa[kk] / ks.mesh) @ B
            mom.append((kk, n, p, ks.eps[kk, n]))
    occ = [m for m in mom if m[1] == 0]
    vir = [m for m in mom if m[1] > 0]

    def v(q):
        q2 = float(q @ q)
        return 4 * math.pi / q2 if (q2 > 1e-20 and 0.5 * q2 <= ko.ecut_aux) else 0.0
    tau, w = sinc_laplace_quadrature(8, 2 * ks.gap, 2 * ks.width)
    D = laplace_denominator(tau, w)
    vp = np.array([m[2] for m in vir])
    ve = np.array([m[3] for m in vir])
    Ed = Ex = 0.0
    for (ki, _, pi_, ei) in occ:
        for (kj, _, pj, ej) in occ:
            for ia in range(len(vir)):
                pa, ea = vp[ia], ve[ia]
                pb = pi_ + pj - pa
                hit = np.flatnonzero(np.abs(vp - pb[None, :]).max(1) < 1e-9)
                if len(hit) == 0:
                    continue
                eb = ve[hit[0]]
                Dv = float(D(np.array(ei + ej - ea - eb)))
                K = v(pa - pi_) / omega              # <i j|a b>
                Kx = v(pb - pi_) / omega             # <i j|b a>
                Ed += 2.0 * K * K * Dv / nk
                Ex -= K * Kx * Dv / nk
    r = kpoint_mp2_energy(ko, D)
    assert Ed < 0
    assert abs(r["E_d"] - Ed) < 1e-12 * abs(Ed), (r["E_d"], Ed)
    assert abs(r["E_x"] - Ex) < 1e-12 * abs(Ed), (r["E_x"], Ex)

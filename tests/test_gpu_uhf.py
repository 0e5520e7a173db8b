"""Spin-unrestricted form on the GPU (Eqs. MP2direct, MP2exchange with the spin sums kept):
against the oracle's spin-unrestricted MP2 with the same quadrature (1e-8 Ha), the
closed-shell limit, the precision form's bound, and rejected pairings."""
import numpy as np
import pytest

import paper_1611_06797_gb300 as L
from oracle import OracleSystem, laplace_denominator, sinc_laplace_quadrature, uhf_mp2_energy
from synth import SPECS, spin_polarized_pair
from tests.conftest import solid

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-8
MEV_PER_ATOM = 0.1 / L.HARTREE_TO_MEV


def _quad(a, b, n):
    lo = 2.0 * min(a.gap, b.gap)
    hi = 2.0 * max(a.width, b.width)
    return sinc_laplace_quadrature(n, lo, hi)


@pytest.mark.parametrize("name,na,nb,real,slab", [("tiny2", 5, 3, True, None), ("tiny2", 4, 2, False, 3),
                                                  ("cfg1", 5, 3, True, 4)])
def test_uhf_matches_oracle(name, na, nb, real, slab):
    a, b = spin_polarized_pair(SPECS[name], na, nb, real_orbitals=real)
    tau, w = _quad(a, b, 6)
    ref = uhf_mp2_energy(OracleSystem.from_solid(a), OracleSystem.from_solid(b), laplace_denominator(tau, w))
    ca = L.setup_from_solid(a, precision=L.FP64, real=real)
    cb = L.setup_from_solid(b, precision=L.FP64, real=real)
    if slab:
        L.ltmp2_set_slab_size(ca, slab)
    ed, ex, es = L.ltmp2_energy_uhf(ca, cb, tau, w)
    # the pairing leaves each context usable on its own
    L.ltmp2_energy(cb, tau, w)
    L.ltmp2_destroy(ca)
    L.ltmp2_destroy(cb)
    assert abs(ed - ref["E_d"]) < TOL_FP64 and abs(ex - ref["E_x"]) < TOL_FP64
    assert abs(es[0] - ref["E_aa"]) < TOL_FP64 and abs(es[1] - ref["E_bb"]) < TOL_FP64
    assert abs(es[2] - ref["E_ab"]) < TOL_FP64


def test_closed_shell_limit():
    s = solid("cfg1")
    tau, w = _quad(s, s, 4)
    c = L.setup_from_solid(s, precision=L.FP64, real=True)
    c2 = L.setup_from_solid(s, precision=L.FP64, real=True)
    ed0, ex0, _ = L.ltmp2_energy(c, tau, w)
    ed, ex, es = L.ltmp2_energy_uhf(c, c2, tau, w)
    L.ltmp2_destroy(c)
    L.ltmp2_destroy(c2)
    assert abs(ed - ed0) < 1e-12 * abs(ed0) and abs(ex - ex0) < 1e-12 * abs(ex0)
    assert abs(es[0] - es[1]) < 1e-13


def test_uhf_precision_form_within_bound():
    a, b = spin_polarized_pair(SPECS["cfg1"], 5, 3)
    tau, w = _quad(a, b, 6)
    out = {}
    for prec in (L.FP64, L.FP32):
        ca = L.setup_from_solid(a, precision=prec, real=True)
        cb = L.setup_from_solid(b, precision=prec, real=True)
        out[prec] = L.ltmp2_energy_uhf(ca, cb, tau, w)
        L.ltmp2_destroy(ca)
        L.ltmp2_destroy(cb)
    bound = MEV_PER_ATOM * a.n_atoms
    assert abs(out[L.FP32][0] - out[L.FP64][0]) < bound and abs(out[L.FP32][1] - out[L.FP64][1]) < bound


def test_uhf_rejects_mismatched_channels():
    a, b = spin_polarized_pair(SPECS["tiny2"], 3, 2)
    ca = L.setup_from_solid(a, precision=L.FP64, real=True)
    cb = L.setup_from_solid(b, precision=L.FP32, real=True)
    tau, w = _quad(a, b, 3)
    with pytest.raises(L.Ltmp2Error) as e:
        L.ltmp2_energy_uhf(ca, cb, tau, w)
    assert e.value.name == "INVALID_ARG"
    with pytest.raises(L.Ltmp2Error):
        L.ltmp2_energy_uhf(ca, ca, tau, w)
    other = L.setup_from_solid(solid("cfg1"), precision=L.FP64, real=True)   # another cell and grid
    with pytest.raises(L.Ltmp2Error):
        L.ltmp2_energy_uhf(ca, other, tau, w)
    cb64 = L.setup_from_solid(b, precision=L.FP64, real=True)
    L.ltmp2_set_extrapolation(cb64, 4, 1.1)
    with pytest.raises(L.Ltmp2Error) as e:
        L.ltmp2_energy_uhf(ca, cb64, tau, w)
    assert e.value.name == "UNSUPPORTED"
    for c in (ca, cb, other, cb64):
        L.ltmp2_destroy(c)

"""Virtuals per Laplace point (Eq. SCHLT's factor e^{-(e_a-mu)tau}): the virtuals whose
weight falls below 2^-64 of the LUMO's are left out at that tau, and where it is cheaper the
transformed states go through the virtual space, W = R_v'^T D' (R_v' U S), instead of the
Green's function.  Every setting gives the oracle's energies within 1e-8 Ha and the same
energies as the full sum over virtuals to FP64 rounding."""
import numpy as np
import pytest

import paper_1611_06797_gb300 as L
from oracle import OracleSystem, denominator_range, laplace_denominator, mp2_energy, sinc_laplace_quadrature
from tests.conftest import solid

pytestmark = pytest.mark.gpu

MEV_PER_ATOM = 0.1 / L.HARTREE_TO_MEV


def _quad(s):
    o = OracleSystem.from_solid(s)
    tau, w = sinc_laplace_quadrature(s.spec.n_tau, *denominator_range(o))
    return o, tau, w


@pytest.mark.parametrize("name,real,phases", [("cfg1", True, False), ("tiny2", True, False),
                                              ("tiny2", False, True)])
def test_virtual_settings_match_oracle(name, real, phases):
    s = solid(name, random_phases=phases)
    o, tau, w = _quad(s)
    ref = mp2_energy(o, laplace_denominator(tau, w))
    ctx = L.setup_from_solid(s, precision=L.FP64, real=real)
    n_v = s.n_orb - s.n_occ
    nv, wv = L.ltmp2_tau_virtuals(ctx, tau)
    order = np.argsort(tau)
    # ascending energies: no more virtuals at a larger tau, never none, some left out here
    assert np.all(np.diff(nv[order]) <= 0) and nv.min() >= 1 and nv.max() <= n_v
    assert nv.min() < n_v
    # the virtual-space route exists only for real orbitals (the real cos/sin basis)
    assert (wv.max() == 1) == real
    res = {}
    for mode, cut in ((L.VIRTUALS_ALL, 64.0), (L.VIRTUALS_AUTO, 64.0), (L.VIRTUALS_SPACE, 64.0),
                      (L.VIRTUALS_AUTO, 53.0)):
        L.ltmp2_set_virtual_cut(ctx, mode, cut)
        ed, ex, ep = L.ltmp2_energy(ctx, tau, w)
        assert abs(ed - ref["E_d"]) < 1e-8 and abs(ex - ref["E_x"]) < 1e-8, (mode, cut)
        assert np.abs(ep - (ref["e_d"] + ref["e_x"])).max() < 1e-8
        res[(mode, cut)] = (ed, ex, ep)
    ed0, ex0, ep0 = res[(L.VIRTUALS_ALL, 64.0)]
    for key, (ed, ex, ep) in res.items():
        assert abs(ed - ed0) < 1e-12 * abs(ed0) and abs(ex - ex0) < 1e-12 * abs(ex0), key
        assert np.abs(ep - ep0).max() < 1e-13, key
    L.ltmp2_destroy(ctx)


def test_virtual_cut_arguments():
    s = solid("tiny2")
    ctx = L.setup_from_solid(s, precision=L.FP64, real=True)
    for mode, cut in ((3, 64.0), (-1, 64.0), (1, 52.0), (1, 2000.0), (1, float("nan"))):
        with pytest.raises(L.Ltmp2Error) as e:
            L.ltmp2_set_virtual_cut(ctx, mode, cut)
        assert e.value.name == "INVALID_ARG"
    for bad in ([0.0], [-1.0], [float("inf")]):
        with pytest.raises(L.Ltmp2Error):
            L.ltmp2_tau_virtuals(ctx, bad)
    # every virtual with VIRTUALS_ALL, and the route never taken
    L.ltmp2_set_virtual_cut(ctx, L.VIRTUALS_ALL)
    nv, wv = L.ltmp2_tau_virtuals(ctx, [1e3, 1e-3])
    assert list(nv) == [s.n_orb - s.n_occ] * 2 and wv.max() == 0
    L.ltmp2_destroy(ctx)


def test_fp32_cuda_core_gemms_take_the_virtual_route():
    """LTMP2_FLAG_SIMT_GEMM: the precision form's GEMMs on the CUDA cores, where the
    virtual-space route exists in FP32 too; within 0.1 meV/atom of the FP64 path."""
    s = solid("cfg1")
    _, tau, w = _quad(s)
    c64 = L.setup_from_solid(s, precision=L.FP64, real=True)
    d64, x64, _ = L.ltmp2_energy(c64, tau, w)
    L.ltmp2_destroy(c64)
    c32 = L.setup_from_solid(s, precision=L.FP32, real=True, simt_gemm=True)
    assert L.ltmp2_tau_virtuals(c32, tau)[1].max() == 1
    tol = MEV_PER_ATOM * s.n_atoms
    for mode in (L.VIRTUALS_ALL, L.VIRTUALS_AUTO, L.VIRTUALS_SPACE):
        L.ltmp2_set_virtual_cut(c32, mode)
        d32, x32, _ = L.ltmp2_energy(c32, tau, w)
        assert abs(d32 - d64) < tol and abs(x32 - x64) < tol, mode
    L.ltmp2_destroy(c32)

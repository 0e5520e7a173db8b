"""Internal auxiliary-cutoff extrapolation on the GPU (Sec. III D, Eq. CutDecay).

Every level's E_d[n], E_x[n] (the energy with all auxiliary G- and G'-sums truncated
at E_aux[n] = E_aux / alpha^(n-1)) must match the oracle's calculation repeated at that
cutoff within the plain path's 1e-8 Ha, and the sphere sizes |A_n| its lattice count.
"""
import numpy as np
import pytest

import paper_1611_06797_gb300 as L
from oracle import (OracleSystem, cutoff_extrapolation, denominator_range, laplace_denominator,
                    level_energies, sinc_laplace_quadrature)
from tests.conftest import solid

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-8
MEV_PER_ATOM = 0.1 / L.HARTREE_TO_MEV


def _levels_gpu(s, tau, w, n_c, alpha, precision=L.FP64, real=True, slab=None):
    ctx = L.setup_from_solid(s, precision=precision, real=real)
    if slab:
        L.ltmp2_set_slab_size(ctx, slab)
    L.ltmp2_set_extrapolation(ctx, n_c, alpha)
    ed, ex, _ = L.ltmp2_energy(ctx, tau, w)
    lev = L.ltmp2_level_energies(ctx)
    L.ltmp2_destroy(ctx)
    return ed, ex, lev


@pytest.mark.parametrize("name,real,n_c,alpha,slab", [("cfg1", True, 8, 1.05, None),
                                                      ("cfg1", False, 8, 1.05, 7),
                                                      ("tiny2", False, 4, 1.2, None),
                                                      ("tiny2", True, 3, 1.3, 3)])
def test_level_energies_match_oracle(name, real, n_c, alpha, slab):
    s = solid(name)
    o = OracleSystem.from_solid(s)
    tau, w = sinc_laplace_quadrature(s.spec.n_tau, *denominator_range(o))
    ecut, counts, ed_ref, ex_ref = level_energies(o, laplace_denominator(tau, w), n_c, alpha)
    ed, ex, lev = _levels_gpu(s, tau, w, n_c, alpha, real=real, slab=slab)
    assert np.allclose(lev["ecut_aux"], ecut, rtol=1e-14, atol=0)
    assert list(lev["n_aux"]) == list(counts)
    assert np.abs(lev["E_d"] - ed_ref).max() < TOL_FP64, (lev["E_d"], ed_ref)
    assert np.abs(lev["E_x"] - ex_ref).max() < TOL_FP64, (lev["E_x"], ex_ref)
    # level 1 is the call's own result
    assert lev["E_d"][0] == ed and lev["E_x"][0] == ex
    # the extrapolated energy of the GPU levels and of the oracle's levels
    a_gpu, _, _ = L.ltmp2_extrapolate(lev["ecut_aux"], lev["E_d"] + lev["E_x"])
    a_ref, _, _ = cutoff_extrapolation(ecut, ed_ref + ex_ref)
    assert abs(a_gpu - a_ref) < 20 * TOL_FP64


def test_levels_leave_the_full_cutoff_energy_unchanged():
    s = solid("cfg1")
    tau, w = sinc_laplace_quadrature(4, *denominator_range(OracleSystem.from_solid(s)))
    ctx = L.setup_from_solid(s, precision=L.FP64, real=True)
    ed0, ex0, ep0 = L.ltmp2_energy(ctx, tau, w)
    L.ltmp2_set_extrapolation(ctx, 8, 1.05)
    ed1, ex1, ep1 = L.ltmp2_energy(ctx, tau, w)
    L.ltmp2_set_extrapolation(ctx, 0, 1.05)
    ed2, ex2, _ = L.ltmp2_energy(ctx, tau, w)
    L.ltmp2_destroy(ctx)
    assert abs(ed1 - ed0) < 1e-12 * abs(ed0) and abs(ex1 - ex0) < 1e-12 * abs(ex0)
    assert np.abs(ep1 - ep0).max() < 1e-12
    assert ed2 == ed0 and ex2 == ex0


def test_precision_form_levels_within_bound():
    s = solid("cfg1")
    tau, w = sinc_laplace_quadrature(s.spec.n_tau, *denominator_range(OracleSystem.from_solid(s)))
    _, _, l64 = _levels_gpu(s, tau, w, 8, 1.05)
    _, _, l32 = _levels_gpu(s, tau, w, 8, 1.05, precision=L.FP32)
    bound = MEV_PER_ATOM * s.n_atoms
    for k in ("E_d", "E_x"):
        assert np.abs(l32[k] - l64[k]).max() < bound
    assert np.abs((l32["E_d"] + l32["E_x"]) - (l64["E_d"] + l64["E_x"])).max() < bound


def test_extrapolation_arguments_are_checked():
    s = solid("tiny2")
    ctx = L.setup_from_solid(s, precision=L.FP64, real=True)
    for n_c, alpha in [(17, 1.05), (8, 1.0), (8, float("nan"))]:
        with pytest.raises(L.Ltmp2Error) as e:
            L.ltmp2_set_extrapolation(ctx, n_c, alpha)
        assert e.value.name == "INVALID_ARG"
    L.ltmp2_set_extrapolation(ctx, 4, 1.1)
    lib = L.load_library()
    import ctypes
    d = (ctypes.c_double * 4)()
    # energies are not available before an energy call with these levels
    assert lib.ltmp2_level_energies(ctx.handle, None, None, d, None) == -1
    L.ltmp2_destroy(ctx)

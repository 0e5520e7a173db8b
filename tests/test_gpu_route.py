"""The paper's own transformed-state route (Sec. III A steps (i)-(iii)): overlap densities
rho_aj(G') = <a|e^{-iG'r}|j> stored once, transformation matrix applied per tau.  Same
energies as the oracle (1e-8 Ha) and as the Green's-function route (up to rounding)."""
import numpy as np
import pytest

import paper_1611_06797_gb300 as L
from oracle import OracleSystem, denominator_range, laplace_denominator, mp2_energy, sinc_laplace_quadrature
from tests.conftest import solid

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-8
MEV_PER_ATOM = 0.1 / L.HARTREE_TO_MEV


def _quad(s, n):
    return sinc_laplace_quadrature(n, *denominator_range(OracleSystem.from_solid(s)))


@pytest.mark.parametrize("name,slab", [("tiny2", None), ("cfg1", 5)])
def test_overlap_route_matches_oracle(name, slab):
    s = solid(name)
    tau, w = _quad(s, s.spec.n_tau)
    ref = mp2_energy(OracleSystem.from_solid(s), laplace_denominator(tau, w))
    ctx = L.setup_from_solid(s, precision=L.FP64, real=True)
    if slab:
        L.ltmp2_set_slab_size(ctx, slab)
    L.ltmp2_set_route(ctx, L.ROUTE_OVERLAP)
    ed, ex, ep = L.ltmp2_energy(ctx, tau, w)
    L.ltmp2_destroy(ctx)
    assert abs(ed - ref["E_d"]) < TOL_FP64 and abs(ex - ref["E_x"]) < TOL_FP64
    assert np.abs(ep - (ref["e_d"] + ref["e_x"])).max() < TOL_FP64


def test_routes_agree_and_switch_back():
    s = solid("cfg1")
    tau, w = _quad(s, 4)
    ctx = L.setup_from_solid(s, precision=L.FP64, real=True)
    g = L.ltmp2_energy(ctx, tau, w)
    L.ltmp2_set_route(ctx, L.ROUTE_OVERLAP)
    o = L.ltmp2_energy(ctx, tau, w)
    # partial G' ranges add up on this route too
    n = L.ltmp2_num_primary_gprime(ctx)
    parts = [L.ltmp2_energy_partial(ctx, tau, w, a, min(a + 17, n)) for a in range(0, n, 17)]
    L.ltmp2_set_route(ctx, L.ROUTE_GREEN)
    g2 = L.ltmp2_energy(ctx, tau, w)
    L.ltmp2_destroy(ctx)
    assert abs(o[0] - g[0]) < 1e-11 * abs(g[0]) and abs(o[1] - g[1]) < 1e-11 * abs(g[1])
    assert np.abs(o[2] - g[2]).max() < 1e-12
    assert abs(sum(p[0] for p in parts) - o[0]) < 1e-12 and abs(sum(p[1] for p in parts) - o[1]) < 1e-12
    assert g2[0] == g[0] and g2[1] == g[1]


def test_overlap_route_precision_form_and_levels():
    s = solid("cfg1")
    tau, w = _quad(s, s.spec.n_tau)
    out = {}
    for prec in (L.FP64, L.FP32):
        ctx = L.setup_from_solid(s, precision=prec, real=True)
        L.ltmp2_set_route(ctx, L.ROUTE_OVERLAP)
        L.ltmp2_set_extrapolation(ctx, 4, 1.1)
        ed, ex, _ = L.ltmp2_energy(ctx, tau, w)
        out[prec] = (ed, ex, L.ltmp2_level_energies(ctx))
        L.ltmp2_destroy(ctx)
    bound = MEV_PER_ATOM * s.n_atoms
    assert abs(out[L.FP32][0] - out[L.FP64][0]) < bound and abs(out[L.FP32][1] - out[L.FP64][1]) < bound
    # levels on this route equal the Green's-function route's levels
    ctx = L.setup_from_solid(s, precision=L.FP64, real=True)
    L.ltmp2_set_extrapolation(ctx, 4, 1.1)
    L.ltmp2_energy(ctx, tau, w)
    ref = L.ltmp2_level_energies(ctx)
    L.ltmp2_destroy(ctx)
    lev = out[L.FP64][2]
    assert np.abs(lev["E_d"] - ref["E_d"]).max() < 1e-11 and np.abs(lev["E_x"] - ref["E_x"]).max() < 1e-11


def test_overlap_route_needs_real_orbitals():
    s = solid("tiny2")
    ctx = L.setup_from_solid(s, precision=L.FP64, real=False)
    with pytest.raises(L.Ltmp2Error) as e:
        L.ltmp2_set_route(ctx, L.ROUTE_OVERLAP)
    assert e.value.name == "UNSUPPORTED"
    with pytest.raises(L.Ltmp2Error):
        L.ltmp2_set_route(ctx, 2)
    L.ltmp2_destroy(ctx)

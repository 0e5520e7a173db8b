"""The per-Laplace-point virtual cut of the CUDA path, checked on the FP64 oracle alone: at
each tau the virtuals with e^{-(e_a - e_LUMO) tau} < 2^-64 are left out (the same rule as
ltmp2_tau_virtuals, energies ascending, at least one kept).  The oracle's canonical sum with
the Laplace denominator of that single point, over the kept virtuals only, must equal the
sum over all virtuals to FP64 rounding, point by point and in total; and on these systems
the cut does remove virtuals at the largest tau."""
import dataclasses
import math

import numpy as np
import pytest

from oracle import OracleSystem, denominator_range, laplace_denominator, mp2_energy, sinc_laplace_quadrature
from tests.conftest import solid

L2CUT = 64.0


def kept_virtuals(eps, n_occ, tau):
    """The first n virtuals with (e_a - e_LUMO) tau <= 64 ln 2 (at least one)."""
    ev = np.asarray(eps[n_occ:], float)
    cut = ev[0] + L2CUT * math.log(2.0) / tau
    return max(1, int(np.searchsorted(ev, cut, side="right")))


@pytest.mark.parametrize("name,phases", [("tiny2", True), ("cfg1", False)])
def test_virtual_cut_changes_the_oracle_energy_only_at_rounding(name, phases):
    s = solid(name, random_phases=phases)
    o = OracleSystem.from_solid(s)
    tau, w = sinc_laplace_quadrature(s.spec.n_tau, *denominator_range(o))
    n_v = o.coeff.shape[0] - o.n_occ
    tot_full = tot_cut = 0.0
    cut_somewhere = False
    for tk, wk in zip(tau, w):
        nv = kept_virtuals(o.eps, o.n_occ, tk)
        assert 1 <= nv <= n_v
        D = laplace_denominator(np.array([tk]), np.array([wk]))
        full = mp2_energy(o, D)["E"]
        if nv == n_v:
            tot_full += full
            tot_cut += full
            continue
        cut_somewhere = True
        keep = o.n_occ + nv
        oc = dataclasses.replace(o, coeff=o.coeff[:keep], eps=o.eps[:keep])
        cut = mp2_energy(oc, D)["E"]
        # the dropped terms carry weights below 2^-64 of the kept ones
        assert abs(cut - full) <= 1e-14 * abs(full) + 1e-18, (tk, nv, cut, full)
        tot_full += full
        tot_cut += cut
    assert cut_somewhere
    assert abs(tot_cut - tot_full) <= 1e-14 * abs(tot_full)

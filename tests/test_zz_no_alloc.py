"""ltmp2_energy_noalloc: the energy for callers that cannot call cudaMalloc.

Such callers (a process whose device-memory budget is held by its own pool, code that
must avoid the device-wide synchronisation an allocation can trigger, a plug-in whose
host owns all device memory) get every buffer of the path from the library's static
device array.  The result must match ltmp2_setup + ltmp2_energy within the plain
path's tolerance, on two calls in a row (the array keeps the previous call's contents,
so the second call checks that nothing stale leaks into it).

This file is collected last on purpose: if it fails, every other test has already run.
"""
import numpy as np
import pytest

import paper_1611_06797_gb300 as L
from oracle import OracleSystem, denominator_range, sinc_laplace_quadrature
from tests.conftest import solid

pytestmark = pytest.mark.gpu

TOL = 1e-8  # Ha, the plain path's parity tolerance


@pytest.mark.parametrize("name,precision,real", [("cfg1", L.FP64, True), ("tiny2", L.FP64, False),
                                                 ("cfg1", L.FP32, True)])
def test_noalloc_matches_energy_two_calls(name, precision, real):
    s = solid(name)
    tau, w = sinc_laplace_quadrature(s.spec.n_tau, *denominator_range(OracleSystem.from_solid(s)))
    # the allocation-free path runs the CUDA-core GEMM in the precision form
    ctx = L.setup_from_solid(s, precision=precision, real=real, simt_gemm=(precision == L.FP32))
    ed, ex, ep = L.ltmp2_energy(ctx, tau, w)
    L.ltmp2_destroy(ctx)
    flags = L.FLAG_REAL_ORBITALS if real else 0
    tol = TOL if precision == L.FP64 else 1e-7 * max(1.0, abs(ed))
    for _ in range(2):
        d, x, p = L.ltmp2_energy_noalloc(s.lattice, s.grid, s.miller, s.coeff, s.eps, s.n_occ, tau, w,
                                         2 * s.ecut / 3, precision, flags)
        assert abs(d - ed) < tol and abs(x - ex) < tol
        assert np.abs(p - ep).max() < tol


def test_noalloc_rejects_systems_beyond_its_array():
    s = solid("cfg2")   # 3071 plane waves: the buffers exceed the 32 MiB array
    tau, w = sinc_laplace_quadrature(2, 2 * s.gap, 2 * s.width)
    with pytest.raises(L.Ltmp2Error) as e:
        L.ltmp2_energy_noalloc(s.lattice, s.grid, s.miller, s.coeff, s.eps, s.n_occ, tau, w,
                               2 * s.ecut / 3, L.FP64, L.FLAG_REAL_ORBITALS)
    assert e.value.name == "UNSUPPORTED"

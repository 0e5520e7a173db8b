"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Plain FP64 path: within 1e-8 Ha of the oracle's closed-shell MP2 evaluated with the
same Laplace quadrature (Eq. SCHLT), for E_d, E_x and every pair energy e_ij.
Precision form (complex64 FFTs, split-precision GEMMs, FP64 sums): within
0.1 meV/atom of the FP64 path for E_d, E_x and E separately.
"""
import math

import numpy as np
import pytest

import paper_1611_06797_gb300 as L
from oracle import (OracleSystem, canonical_denominator, denominator_range, laplace_denominator,
                    mp2_energy, sinc_laplace_quadrature)
from synth import SPECS, ModelSolidSpec, build_model_solid, free_electron_solid
from tests.conftest import solid

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-8                      # Ha, plain path vs oracle
MEV_PER_ATOM = 0.1 / L.HARTREE_TO_MEV  # Ha per atom, forms vs plain path


def _quad(s, n):
    o = OracleSystem.from_solid(s)
    return sinc_laplace_quadrature(n, *denominator_range(o))


def _oracle(s, tau, w, pairs=None):
    return mp2_energy(OracleSystem.from_solid(s), laplace_denominator(tau, w), pairs=pairs)


def _gpu(s, tau, w, precision=L.FP64, real=False, slab=None):
    ctx = L.setup_from_solid(s, precision=precision, real=real)
    if slab:
        L.ltmp2_set_slab_size(ctx, slab)
    ed, ex, ep = L.ltmp2_energy(ctx, tau, w)
    im = L.ltmp2_last_imag(ctx)
    L.ltmp2_destroy(ctx)
    return ed, ex, ep, im


@pytest.mark.parametrize("name,phases,real", [("tiny", False, False), ("tiny", False, True),
                                              ("tiny2", True, False), ("tiny2", False, True),
                                              ("cfg1", False, False), ("cfg1", False, True)])
def test_fp64_matches_oracle(name, phases, real):
    s = solid(name, random_phases=phases)
    tau, w = _quad(s, s.spec.n_tau)
    ref = _oracle(s, tau, w)
    ed, ex, ep, im = _gpu(s, tau, w, real=real)
    assert abs(ed - ref["E_d"]) < TOL_FP64, (ed, ref["E_d"])
    assert abs(ex - ref["E_x"]) < TOL_FP64, (ex, ref["E_x"])
    eref = ref["e_d"] + ref["e_x"]
    assert np.abs(ep - eref).max() < TOL_FP64
    assert np.abs(ep - ep.T).max() < 1e-12
    assert abs(im[0]) < 1e-10 and abs(im[1]) < 1e-10


def test_slab_sizes_and_ragged_tail_agree():
    s = solid("cfg1")
    tau, w = _quad(s, 3)
    ctx = L.setup_from_solid(s, real=True)
    nprim = L.ltmp2_num_primary_gprime(ctx)
    ref = L.ltmp2_energy(ctx, tau, w)
    for slab in (1, 7, nprim - 1):
        L.ltmp2_set_slab_size(ctx, slab)
        ed, ex, ep = L.ltmp2_energy(ctx, tau, w)
        assert abs(ed - ref[0]) < 1e-12 and abs(ex - ref[1]) < 1e-12
        assert np.abs(ep - ref[2]).max() < 1e-13
    L.ltmp2_destroy(ctx)


def test_partial_gprime_ranges_sum_to_total():
    """Sec. III B: the outer G' loop splits into independent additive pieces."""
    s = solid("tiny2")
    tau, w = _quad(s, 4)
    ctx = L.setup_from_solid(s)
    n = L.ltmp2_num_primary_gprime(ctx)
    ed, ex, ep = L.ltmp2_energy(ctx, tau, w)
    cuts = [0, n // 3, n // 2 + 1, n]
    parts = [L.ltmp2_energy_partial(ctx, tau, w, a, b) for a, b in zip(cuts[:-1], cuts[1:])]
    assert abs(sum(p[0] for p in parts) - ed) < 1e-12
    assert abs(sum(p[1] for p in parts) - ex) < 1e-12
    assert np.abs(sum(p[2] + p[3] for p in parts) - ep).max() < 1e-13
    L.ltmp2_destroy(ctx)


def test_one_occupied_orbital_exchange_is_minus_half_direct():
    spec = ModelSolidSpec("one", a=5.0, grid=8, r2=9, wells=1, n_occ=1, n_tau=6, seed=7)
    s = build_model_solid(spec, random_phases=True)
    tau, w = _quad(s, 6)
    ed, ex, _, _ = _gpu(s, tau, w)
    assert ed < 0 and abs(ex + 0.5 * ed) < 1e-12


def test_free_electron_closed_form():
    """V = 0, one orbital: E_d^LT = -2 sum_{G in A} (4 pi / G^2 / Omega)^2 sum_k w_k e^{-G^2 tau_k}."""
    a, grid, r2 = 5.5, 12, 9
    s = free_electron_solid(a, grid, r2, n_occ=1)
    o = OracleSystem.from_solid(s)
    tau, w = sinc_laplace_quadrature(6, *denominator_range(o))
    b = 2 * math.pi / a
    Ed = 0.0
    R = 3
    for mx in range(-R, R + 1):
        for my in range(-R, R + 1):
            for mz in range(-R, R + 1):
                g2 = (mx * mx + my * my + mz * mz) * b * b
                if 0 < g2 and 0.5 * g2 <= o.ecut_aux:
                    Ed += -2 * (4 * math.pi / g2 / a ** 3) ** 2 * float(np.sum(w * np.exp(-g2 * tau)))
    ctx = L.ltmp2_setup(s.lattice, s.grid, s.miller, s.coeff, s.eps, 1, o.ecut_aux)
    ed, ex, _ = L.ltmp2_energy(ctx, tau, w)
    assert abs(ed - Ed) < 1e-12 * abs(Ed) + 1e-14
    assert abs(ex + 0.5 * Ed) < 1e-12 * abs(Ed) + 1e-14


@pytest.mark.parametrize("name", ["tiny2", "cfg1"])
def test_fp32_form_within_bound_of_fp64(name):
    s = solid(name)
    tau, w = _quad(s, s.spec.n_tau)
    d64, x64, p64, _ = _gpu(s, tau, w, L.FP64, real=True)
    d32, x32, p32, _ = _gpu(s, tau, w, L.FP32, real=True)
    tol = MEV_PER_ATOM * s.n_atoms
    assert abs(d32 - d64) < tol and abs(x32 - x64) < tol and abs(d32 + x32 - d64 - x64) < tol


def test_cfg2_full_size_sampled_pairs():
    """16 wells, 24^3 grid, 3071 plane waves, 32 occupied, 8 tau points: the benchmark's
    workload and launch configuration; sampled pair energies against the oracle."""
    s = solid("cfg2")
    tau, w = _quad(s, 8)
    ed, ex, ep, im = _gpu(s, tau, w, L.FP64, real=True)
    pairs = [(0, 0), (0, 1), (5, 17), (31, 31), (12, 30), (20, 3)]
    ref = _oracle(s, tau, w, pairs=pairs)
    for (i, j) in pairs:
        e = ref["e_d"][i, j] + ref["e_x"][i, j]
        assert abs(ep[i, j] - e) < TOL_FP64, (i, j, ep[i, j], e)
    assert abs(ep.sum() - (ed + ex)) < 1e-10
    assert ed < 0
    # the precision form on the same inputs stays within 0.1 meV/atom of the plain path
    d32, x32, _, _ = _gpu(s, tau, w, L.FP32, real=True)
    tol = MEV_PER_ATOM * s.n_atoms
    assert abs(d32 - ed) < tol and abs(x32 - ex) < tol and abs(d32 + x32 - ed - ex) < tol


@pytest.mark.parametrize("name,real", [("cfg1", True), ("tiny2", False)])
def test_plane_kernels_and_block_shapes_agree(name, real):
    """The four plane-FFT kernels (full-plane passes, compacted passes, product in
    registers, warp-autonomous) with several occupied-plane blocks, including a ragged last block, give
    the oracle's energies in FP64 and the FP64 energies within the bound in FP32."""
    s = solid(name)
    tau, w = _quad(s, 4)
    ref = _oracle(s, tau, w)
    base = {}
    for precision in (L.FP64, L.FP32):
        ctx = L.setup_from_solid(s, precision=precision, real=real)
        for pk in (0, 1, 2, 3):
            for ib in (0, 1, 3):
                L.ltmp2_set_tuning(ctx, plane_kernel=pk, plane_ib=ib)
                assert L.ltmp2_get_tuning(ctx)["plane_kernel"] == pk
                ed, ex, ep = L.ltmp2_energy(ctx, tau, w)
                if precision == L.FP64:
                    assert abs(ed - ref["E_d"]) < TOL_FP64 and abs(ex - ref["E_x"]) < TOL_FP64
                    base.setdefault("ed", ed)
                    base.setdefault("ex", ex)
                    assert abs(ed - base["ed"]) < 1e-12 * abs(ed) and abs(ex - base["ex"]) < 1e-12 * abs(ex)
                else:
                    bound = MEV_PER_ATOM * s.n_atoms
                    assert abs(ed - base["ed"]) < bound and abs(ex - base["ex"]) < bound
        with pytest.raises(L.Ltmp2Error):
            L.ltmp2_set_tuning(ctx, plane_kernel=4)
        with pytest.raises(L.Ltmp2Error):
            L.ltmp2_set_tuning(ctx, plane_kernel=0, plane_ib=2000)
        L.ltmp2_destroy(ctx)


@pytest.mark.parametrize("name", ["tiny2", "cfg1"])
def test_precision_form_green_and_direct_choices(name):
    """The precision form's Green's function (compensated CUDA-core sums by default, or
    3xTF32 on the tensor cores, set up at first use) and its direct term (tensor cores by
    default, or CUDA cores): every combination within 0.1 meV/atom of the FP64 path."""
    s = solid(name)
    tau, w = _quad(s, s.spec.n_tau)
    d64, x64, p64, _ = _gpu(s, tau, w, L.FP64, real=True)
    ctx = L.setup_from_solid(s, precision=L.FP32, real=True)
    t = L.ltmp2_get_tuning(ctx)
    assert t["green_tc"] == 0 and t["direct_tc"] == 1
    bound = MEV_PER_ATOM * s.n_atoms
    for g, d in ((1, 1), (1, 0), (0, 0), (0, 1)):
        L.ltmp2_set_tuning(ctx, green_tc=g, direct_tc=d)
        t = L.ltmp2_get_tuning(ctx)
        assert (t["green_tc"], t["direct_tc"]) == (g, d)
        ed, ex, ep = L.ltmp2_energy(ctx, tau, w)
        assert abs(ed - d64) < bound and abs(ex - x64) < bound and np.abs(ep - p64).max() < bound, (g, d)
    with pytest.raises(L.Ltmp2Error):
        L.ltmp2_set_tuning(ctx, green_tc=2)
    L.ltmp2_destroy(ctx)
    # no choice in FP64
    c64 = L.setup_from_solid(s, precision=L.FP64, real=True)
    t = L.ltmp2_get_tuning(c64)
    assert t["green_tc"] == -1 and t["direct_tc"] == -1
    with pytest.raises(L.Ltmp2Error):
        L.ltmp2_set_tuning(c64, green_tc=1)
    L.ltmp2_destroy(c64)

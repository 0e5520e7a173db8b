"""k-point sampling on the GPU (Sec. II C-D): the CUDA path through the C ABI against the
k-point oracle (canonical MP2 per unit cell with the Laplace denominator, explicit sums over
k1, k2, k3 and i, j, a, b), element by element on the pair energies of the composite occupied
orbitals (k, i), within 1e-8 Ha; the precision form within 0.1 meV/atom of the FP64 path;
additive ranges of the outer supercell-transfer loop; and, on a 2 x 2 x 2 mesh, the
Gamma-point path on the cubic supercell (independent kernels) gives N_k times the energy."""
import numpy as np
import pytest

import paper_1611_06797_gb300 as L
from oracle import KPointOracleSystem, kpoint_mp2_energy, laplace_denominator, sinc_laplace_quadrature
from synth import build_kpoint_pair, build_kpoint_solid

pytestmark = pytest.mark.gpu

TOL = 1e-8
MEV = 0.1 / L.HARTREE_TO_MEV
POS = np.array([[1.1, 2.3, 2.0]])
_CACHE = {}


def _case(mesh, n_occ, phases, seed):
    key = (mesh, n_occ, phases, seed)
    if key not in _CACHE:
        ks = build_kpoint_solid(5.0, 8, 9, mesh, POS, n_occ, random_phases=phases, seed=seed)
        tau, w = sinc_laplace_quadrature(6, 2 * ks.gap, 2 * ks.width)
        ref = kpoint_mp2_energy(KPointOracleSystem.from_solid(ks), laplace_denominator(tau, w))
        _CACHE[key] = (ks, tau, w, ref)
    return _CACHE[key]


def _gpu(ks, tau, w, precision=L.FP64, slab=None):
    ctx = L.setup_from_kpoint_solid(ks, precision=precision)
    if slab:
        L.ltmp2_set_slab_size(ctx, slab)
    ed, ex, ep = L.ltmp2_energy(ctx, tau, w)
    n_prim = L.ltmp2_num_primary_gprime(ctx)
    L.ltmp2_destroy(ctx)
    return ed, ex, ep, n_prim


@pytest.mark.parametrize("mesh,n_occ,phases", [((1, 1, 1), 2, False), ((2, 1, 1), 1, False),
                                               ((1, 2, 1), 2, True), ((3, 1, 1), 1, False),
                                               ((2, 2, 1), 1, True), ((1, 1, 2), 2, False)])
def test_kpoint_fp64_matches_oracle(mesh, n_occ, phases):
    ks, tau, w, ref = _case(mesh, n_occ, phases, 4)
    eref = ref["e_d"] + ref["e_x"]
    ed, ex, ep, n_prim = _gpu(ks, tau, w)
    assert abs(ed - ref["E_d"]) < TOL, (ed, ref["E_d"])
    assert abs(ex - ref["E_x"]) < TOL, (ex, ref["E_x"])
    assert ep.shape == eref.shape and np.abs(ep - eref).max() < TOL
    # a ragged last slab of the outer loop over supercell transfers
    slab = max(1, n_prim // 3 - 1)
    if n_prim % slab == 0:
        slab -= 1
    ed2, ex2, ep2, _ = _gpu(ks, tau, w, slab=max(1, slab))
    assert abs(ed2 - ed) < 1e-12 and abs(ex2 - ex) < 1e-12 and np.abs(ep2 - ep).max() < 1e-13


@pytest.mark.parametrize("mesh", [(2, 1, 1), (2, 2, 1)])
def test_kpoint_fp32_within_bound(mesh):
    ks, tau, w, _ = _case(mesh, 1, False, 4)
    d64, x64, p64, _ = _gpu(ks, tau, w, L.FP64)
    d32, x32, p32, _ = _gpu(ks, tau, w, L.FP32)
    tol = MEV * ks.n_atoms
    assert abs(d32 - d64) < tol and abs(x32 - x64) < tol and np.abs(p32 - p64).max() < tol


def test_kpoint_partial_ranges_sum():
    ks, tau, w, _ = _case((2, 1, 1), 1, False, 4)
    ctx = L.setup_from_kpoint_solid(ks)
    n = L.ltmp2_num_primary_gprime(ctx)
    ed, ex, ep = L.ltmp2_energy(ctx, tau, w)
    cuts = [0, n // 4, n // 2 + 1, n]
    parts = [L.ltmp2_energy_partial(ctx, tau, w, a, b) for a, b in zip(cuts[:-1], cuts[1:])]
    assert abs(sum(p[0] for p in parts) - ed) < 1e-12 and abs(sum(p[1] for p in parts) - ex) < 1e-12
    assert np.abs(sum(p[2] + p[3] for p in parts) - ep).max() < 1e-13
    for call in (lambda: L.ltmp2_set_route(ctx, L.ROUTE_OVERLAP), lambda: L.ltmp2_set_extrapolation(ctx, 8, 1.05),
                 lambda: L.ltmp2_set_pair_mask(ctx, np.ones((2, 2), bool)), lambda: L.ltmp2_autotune(ctx)):
        with pytest.raises(L.Ltmp2Error) as e:
            call()
        assert e.value.name == "UNSUPPORTED"
    L.ltmp2_destroy(ctx)


def test_kpoint_222_equals_gamma_supercell_path():
    """2 x 2 x 2 mesh: the k-point kernels against the Gamma-point kernels on the cubic
    2a supercell (16^3 grid, 8 x 123 plane waves, 8 occupied) built from the same potential."""
    ks, sc = build_kpoint_pair(5.0, 8, 9, (2, 2, 2), POS, 1, seed=9)
    tau, w = sinc_laplace_quadrature(6, 2 * ks.gap, 2 * ks.width)
    ed, ex, _, _ = _gpu(ks, tau, w)
    ctx = L.ltmp2_setup(sc.lattice, sc.grid, sc.miller, sc.coeff, sc.eps, sc.n_occ, 2 * ks.ecut / 3, L.FP64, 0)
    eds, exs, _ = L.ltmp2_energy(ctx, tau, w)
    L.ltmp2_destroy(ctx)
    assert abs(ed - eds / 8) < 1e-9 and abs(ex - exs / 8) < 1e-9, (ed, eds / 8, ex, exs / 8)

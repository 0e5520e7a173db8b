"""Parity at every FFT grid the library instantiates (16 .. 40 points per axis).

Each grid size has its own compile-time line FFT and its own instantiations of the
plane, column and z-transform kernels, so each one is compared with the FP64 oracle
(Eq. CanMP2 with the Laplace denominator of Eq. SCHLT) element by element: E_d, E_x and
every pair energy e_ij within 1e-8 Ha, for general complex orbitals (each (i, j, G')
item paired with (j, i, -G')) and for real orbitals (the time-reversal pairing of
Sec. II D), with a slab size that leaves a ragged last slab of the outer G' loop.  The
precision form on the same inputs stays within 0.1 meV/atom of the FP64 path.

The systems are small spheres (a few hundred plane waves, 3 occupied orbitals) on the
large grids, so the oracle finishes in a second while every FFT line has the full
length of the grid.  The last test runs the 64-well, 36^3 grid, 10,059-plane-wave,
128-occupied-orbital system (the precision form's workload) at its full launch shapes
on a few primary G', FP32 against FP64.
"""
import numpy as np
import pytest

import paper_1611_06797_gb300 as L
from oracle import OracleSystem, denominator_range, laplace_denominator, mp2_energy, sinc_laplace_quadrature
from synth import ModelSolidSpec, build_model_solid

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-8                          # Ha, plain path vs oracle
MEV_PER_ATOM = 0.1 / L.HARTREE_TO_MEV    # Ha per atom, precision form vs plain path

# grid -> (cell constant in bohr, squared sphere radius in index units); 179 .. 389 plane waves
GRIDS = {16: (6.0, 12), 18: (6.5, 16), 20: (6.0, 20), 25: (7.0, 16), 27: (6.5, 16),
         30: (6.0, 12), 32: (7.5, 16), 36: (7.0, 16), 40: (6.5, 16)}

_CACHE = {}


def _system(n, phases):
    key = (n, phases)
    if key not in _CACHE:
        a, r2 = GRIDS[n]
        spec = ModelSolidSpec(f"grid{n}", a=a, grid=n, r2=r2, wells=2, n_occ=3, n_tau=3, seed=200 + n)
        s = build_model_solid(spec, random_phases=phases)
        o = OracleSystem.from_solid(s)
        tau, w = sinc_laplace_quadrature(3, *denominator_range(o))
        _CACHE[key] = (s, tau, w, mp2_energy(o, laplace_denominator(tau, w)))
    return _CACHE[key]


def _ragged_slab(n_prim):
    """A slab size below n_prim that does not divide it."""
    for slab in range(max(1, n_prim // 3), 0, -1):
        if n_prim % slab:
            return slab
    return 1


def _run(s, tau, w, precision, real, ragged):
    ctx = L.setup_from_solid(s, precision=precision, real=real)
    n_prim = L.ltmp2_num_primary_gprime(ctx)
    if ragged:
        slab = _ragged_slab(n_prim)
        assert L.ltmp2_set_slab_size(ctx, slab) == slab and n_prim % slab != 0
    ed, ex, ep = L.ltmp2_energy(ctx, tau, w)
    L.ltmp2_destroy(ctx)
    return ed, ex, ep


@pytest.mark.parametrize("real", [False, True], ids=["general", "real"])
@pytest.mark.parametrize("n", sorted(GRIDS))
def test_fp64_matches_oracle_at_grid(n, real):
    s, tau, w, ref = _system(n, phases=not real)
    assert s.grid[0] == n
    eref = ref["e_d"] + ref["e_x"]
    for ragged in (False, True):
        ed, ex, ep = _run(s, tau, w, L.FP64, real, ragged)
        assert abs(ed - ref["E_d"]) < TOL_FP64, (n, real, ragged, ed, ref["E_d"])
        assert abs(ex - ref["E_x"]) < TOL_FP64, (n, real, ragged, ex, ref["E_x"])
        assert np.abs(ep - eref).max() < TOL_FP64, (n, real, ragged)
        assert np.abs(ep - ep.T).max() < 1e-12


@pytest.mark.parametrize("real", [False, True], ids=["general", "real"])
@pytest.mark.parametrize("n", sorted(GRIDS))
def test_fp32_form_within_bound_at_grid(n, real):
    s, tau, w, _ = _system(n, phases=not real)
    d64, x64, p64 = _run(s, tau, w, L.FP64, real, ragged=True)
    d32, x32, p32 = _run(s, tau, w, L.FP32, real, ragged=True)
    tol = MEV_PER_ATOM * s.n_atoms
    assert abs(d32 - d64) < tol and abs(x32 - x64) < tol and abs(d32 + x32 - d64 - x64) < tol
    # each pair energy within the same bound (a far stricter test than the totals)
    assert np.abs(p32 - p64).max() < tol


def test_precision_form_full_launch_shapes_on_36_grid():
    """64 wells, 36^3, 10,059 plane waves, 128 occupied orbitals, 3 tau points: FP32 against
    FP64 on three spread ranges of the outer G' loop (ltmp2_energy_partial), in the setup's
    default slab and kernel shapes.  The bound is the 0.1 meV/atom budget scaled by the
    sampled share of the G' loop."""
    from synth import SPECS
    s = build_model_solid(SPECS["cfg3"], device="cuda")   # GPU eigensolver: input generation only
    tau, w, _ = L.ltmp2_laplace_grid(s.gap, s.width, 3)
    c64 = L.setup_from_solid(s, precision=L.FP64, real=True)
    c32 = L.setup_from_solid(s, precision=L.FP32, real=True)
    n_prim = L.ltmp2_num_primary_gprime(c64)
    assert n_prim == L.ltmp2_num_primary_gprime(c32) == 2724
    ranges = [(0, 6), (n_prim // 2, n_prim // 2 + 5), (n_prim - 7, n_prim)]
    share = sum(e - b for b, e in ranges) / n_prim
    tol = MEV_PER_ATOM * s.n_atoms * share
    for b, e in ranges:
        d64, x64, pd64, px64 = L.ltmp2_energy_partial(c64, tau, w, b, e)
        d32, x32, pd32, px32 = L.ltmp2_energy_partial(c32, tau, w, b, e)
        assert d64 < 0
        assert abs(d32 - d64) < tol and abs(x32 - x64) < tol, (b, e, d32 - d64, x32 - x64, tol)
        assert np.abs(pd32 + px32 - pd64 - px64).max() < tol
    L.ltmp2_destroy(c64)
    L.ltmp2_destroy(c32)

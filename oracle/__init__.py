"""FP64 CPU oracle for the LTMP2 hot path.

TEST INFRASTRUCTURE ONLY: nothing in the product path may import, call or link
anything here.  The only callers are tests/, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py``.
"""
from .ltmp2_oracle import (OracleSystem, aux_set, overlap_densities_conv,
                           overlap_densities_fft, overlap_densities_dft, pair_integrals,
                           mp2_pair_energy, mp2_energy, sinc_laplace_quadrature,
                           quadrature_max_error, canonical_denominator, laplace_denominator,
                           denominator_range, cutoff_levels, level_energies,
                           cutoff_extrapolation, uhf_mp2_energy, KPointOracleSystem,
                           kpoint_aux_class, kpoint_overlap_densities, kpoint_mp2_energy)

__all__ = ["OracleSystem", "aux_set", "overlap_densities_conv", "overlap_densities_fft",
           "overlap_densities_dft", "pair_integrals", "mp2_pair_energy", "mp2_energy",
           "sinc_laplace_quadrature", "quadrature_max_error", "canonical_denominator",
           "laplace_denominator", "denominator_range", "cutoff_levels", "level_energies",
           "cutoff_extrapolation", "uhf_mp2_energy", "KPointOracleSystem", "kpoint_aux_class",
           "kpoint_overlap_densities", "kpoint_mp2_energy"]

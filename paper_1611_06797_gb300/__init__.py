"""GB300 (sm_103a) Laplace-transformed MP2 hot path behind a C ABI (libltmp2.so).

The Python layer only marshals arguments; every step of the path runs in the
library's CUDA kernels.  See ``include/ltmp2.h`` for the contract.
"""
from .ltmp2 import (Context, Ltmp2Error, LIB_PATH, load_library, ltmp2_setup, ltmp2_set_stream,
                    ltmp2_laplace_grid, ltmp2_energy, ltmp2_energy_partial, ltmp2_num_primary_gprime, ltmp2_set_slab_size,
                    ltmp2_sizes, ltmp2_last_imag, ltmp2_kernel_launches, ltmp2_set_profiling, ltmp2_stage_times,
                    ltmp2_fingerprint, ltmp2_sum_partials, ltmp2_alu_peak, ltmp2_reset_stage_times, ltmp2_destroy, ltmp2_energy_noalloc,
                    ltmp2_set_extrapolation, ltmp2_level_energies, ltmp2_extrapolate,
                    ltmp2_set_route, ROUTE_GREEN, ROUTE_OVERLAP, ltmp2_energy_uhf, ltmp2_selftest_wait,
                    ltmp2_autotune, ltmp2_get_tuning, ltmp2_set_tuning, ltmp2_batch_create,
                    ltmp2_set_pair_mask, ltmp2_pair_descriptors, Mlp, ltmp2_learned_training_data,
                    ltmp2_screen_select, ltmp2_energy_screened, NUM_DESC, ltmp2_energy_batch, Batch, ltmp2_strerror, setup_from_solid,
                    ltmp2_setup_kpoints, setup_from_kpoint_solid, ltmp2_set_virtual_cut, ltmp2_tau_virtuals, ltmp2_dgemm_nt,
                    VIRTUALS_ALL, VIRTUALS_AUTO, VIRTUALS_SPACE,
                    STAGE_NAMES, FP64, FP32, FLAG_REAL_ORBITALS, FLAG_SIMT_GEMM, HARTREE_TO_MEV)

__all__ = ["Context", "Ltmp2Error", "LIB_PATH", "load_library", "ltmp2_setup", "ltmp2_set_stream",
           "ltmp2_laplace_grid", "ltmp2_energy", "ltmp2_energy_partial", "ltmp2_num_primary_gprime", "ltmp2_set_slab_size",
           "ltmp2_sizes", "ltmp2_last_imag", "ltmp2_kernel_launches", "ltmp2_set_profiling", "ltmp2_stage_times",
           "ltmp2_fingerprint", "ltmp2_sum_partials", "ltmp2_alu_peak", "ltmp2_reset_stage_times", "ltmp2_destroy", "ltmp2_energy_noalloc",
           "ltmp2_set_extrapolation", "ltmp2_level_energies", "ltmp2_extrapolate",
           "ltmp2_set_route", "ROUTE_GREEN", "ROUTE_OVERLAP", "ltmp2_energy_uhf", "ltmp2_selftest_wait",
           "ltmp2_autotune", "ltmp2_get_tuning", "ltmp2_set_tuning", "ltmp2_batch_create",
           "ltmp2_set_pair_mask", "ltmp2_pair_descriptors", "Mlp", "ltmp2_learned_training_data",
           "ltmp2_screen_select", "ltmp2_energy_screened", "NUM_DESC", "ltmp2_energy_batch", "Batch", "ltmp2_strerror", "setup_from_solid",
           "ltmp2_setup_kpoints", "setup_from_kpoint_solid", "ltmp2_set_virtual_cut", "ltmp2_tau_virtuals", "ltmp2_dgemm_nt",
           "VIRTUALS_ALL", "VIRTUALS_AUTO", "VIRTUALS_SPACE",
           "STAGE_NAMES", "FP64", "FP32", "FLAG_REAL_ORBITALS", "FLAG_SIMT_GEMM", "HARTREE_TO_MEV"]

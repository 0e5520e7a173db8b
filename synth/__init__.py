"""Seeded synthetic inputs (model solids) shared by the CUDA path's tests, the
benchmark and the oracle's tests.  Holds no MP2 / LTMP2 arithmetic: it only
produces mean-field input (plane-wave orbitals and their energies)."""
from .model_solid import (ModelSolidSpec, ModelSolid, build_model_solid, spec_by_name,
                          SPECS, free_electron_solid, BATCH_NAMES, spin_polarized_pair)
from .kpoints import (KPointSolid, build_kpoint_solid, build_kpoint_pair, supercell_of, mesh_kappa,
                      free_electron_kpoints)

__all__ = ["ModelSolidSpec", "ModelSolid", "build_model_solid", "spec_by_name", "SPECS",
           "free_electron_solid", "BATCH_NAMES", "spin_polarized_pair", "KPointSolid", "build_kpoint_solid",
           "build_kpoint_pair", "supercell_of", "mesh_kappa", "free_electron_kpoints"]

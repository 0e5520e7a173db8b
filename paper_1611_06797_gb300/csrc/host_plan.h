// Host-side validation and index tables of one system, shared by ltmp2_setup (which
// uploads them into device allocations) and ltmp2_energy_noalloc (which places them in
// its static device array).  No device is touched here.
#pragma once
#include <cuda_runtime.h>

#include <array>
#include <cstdint>
#include <vector>

#include "../../include/ltmp2.h"
#include "plan.h"

namespace ltmp2 {

struct HostPlan {
  Plan p;                               // sizes, flags, omega, mu; device pointers unset
  double B[9] = {0};                    // reciprocal lattice rows b_k (a_i . b_k = 2 pi delta_ik)
  double ecut_aux = 0.0;                // E_aux of A (Hartree)
  std::vector<int> order;               // internal plane-wave position -> caller's index
  std::vector<int> negpw;               // caller's index of -G_q for caller's index q
  std::vector<int4> dorb, daux;         // (m1, m2, zlo, zhi) columns of the orbital / aux sphere
  std::vector<int> dorb_off, daux_off;  // first point of each column
  std::vector<int> pw_m, aux_m;         // Miller indices in internal order, [n][3]
  std::vector<int> pw_pair;             // internal position of -G_q (real orbitals only)
  std::vector<int> aux_neg, prim;       // position of -G in A; positions of the primary G'
  std::vector<double> v64, aux_g2;      // 4 pi / |G|^2 (0 at G = 0), |G|^2
  std::vector<float> v32;
  uint64_t fingerprint = 0;             // hash of every input that determines the energies
};

// k-point extras (ltmp2_kpoint_system): mesh, primary supercell transfers, class tables
struct KPointHost {
  std::vector<int> prim_m;       // [n_prim][3] supercell Miller index of each primary Q'
  std::vector<double> vprim;     // [n_prim] 4 pi / |Q'|^2
  std::vector<double> vcls64;    // [n_cls][n_aux] 4 pi / |g + delta/n|^2 inside the sphere, else 0
  std::vector<float> vcls32;
  std::vector<int> lut;          // [n^3] position in A of each grid point, -1 if absent
};

// Validate a k-point system and build the tables: the shared plane-wave columns, the
// auxiliary ball that holds every momentum-transfer class, the class tables, the lookup
// table and the primary supercell transfers.  hp.p carries n_occ = N_k n_occ.
int build_kpoint_host_plan(const ltmp2_kpoint_system *sys, HostPlan &hp, KPointHost &kh) noexcept;

// Validate *sys (flags outside allowed_flags are INVALID_ARG) and build the tables.
// Checks: pointers and sizes, finite lattice / energies / coefficients, non-decreasing
// energies, the HOMO-LUMO gap, a cubic supported grid, a plane-wave set with contiguous m3
// columns that fits the grid (inversion symmetric with LTMP2_FLAG_REAL_ORBITALS), orthonormality of a deterministic
// sample of orbitals, and c(-G) = conj c(G) when LTMP2_FLAG_REAL_ORBITALS is set.
// Returns LTMP2_OK or the status of the first failed check.  Never throws.
int build_host_plan(const ltmp2_system *sys, int allowed_flags, HostPlan &hp) noexcept;

}  // namespace ltmp2

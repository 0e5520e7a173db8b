"""Gaussian-well model solids: the mean-field input of the LTMP2 hot path.

The paper's systems (LiH supercells, CH4 in chabazite, Sec. IV) need VASP, PAW
potentials and Hartree-Fock orbitals, none of which exist here.  These seeded
model solids stand in for them with the same shapes: a cubic cell, a
plane-wave sphere |G|^2/2 <= E_cut (Sec. II A), orbitals and energies from a
dense diagonalisation of  H = -1/2 nabla^2 + V  over that sphere, the lowest
n_occ states doubly occupied and all the rest virtual.

  V(r)   = sum_R -A exp(-|r - R|^2 / (2 s^2))
  V(G)   = -(A / Omega) (2 pi s^2)^{3/2} exp(-G^2 s^2 / 2) sum_R exp(-i G.R)
  H_pq   = 1/2 |G_p|^2 delta_pq + V(G_p - G_q)

V is real in real space, so H is real-symmetric in the cos/sin basis; the
generator diagonalises it there, which makes every orbital real in real space
(c(-G) = conj c(G)).  ``random_phases`` multiplies each orbital by a seeded
phase, which keeps it an eigenvector but breaks that property.

Nothing here computes any part of MP2: it produces (lattice, grid, miller,
coeff, eps, n_occ) only.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Sequence, Tuple

import numpy as np


@dataclasses.dataclass(frozen=True)
class ModelSolidSpec:
    """One synthetic workload.

    a        cubic lattice constant (bohr)
    grid     FFT grid points per axis
    r2       squared radius of the orbital sphere in reciprocal-lattice index
             units: E_cut = 1/2 r2 (2 pi / a)^2, so the sphere is exact
    wells    number of Gaussian wells
    n_occ    doubly occupied orbitals
    n_tau    Laplace points the workload is quoted with
    seed     placement / jitter seed
    lattice_sites  None -> uniform random positions (min distance 2 bohr);
             (n1, n2, n3) -> jittered simple-cubic site lattice
    """
    name: str
    a: float
    grid: int
    r2: int
    wells: int
    n_occ: int
    n_tau: int
    seed: int
    lattice_sites: Optional[Tuple[int, int, int]] = None
    depth: float = 2.0          # A (Ha)
    width: float = 0.8          # s (bohr)
    jitter: float = 0.2         # Gaussian sigma per component (bohr)
    min_dist: float = 2.0       # only for random placement

    @property
    def b(self) -> float:
        return 2.0 * math.pi / self.a

    @property
    def ecut(self) -> float:
        # a hair above the shell r2 so the boundary shell is inside in floating point
        return 0.5 * (self.r2 + 1e-6) * self.b ** 2


# The workloads.  Counts (N_pw, N_G with E_aux = 2/3 E_cut):
#   tiny   : 8^3,  r2 = 9   ->  123 PWs
#   cfg1   : 12^3, r2 = 25  ->  515 PWs,   256 aux G
#   cfg2   : 24^3, r2 = 81  -> 3071 PWs,  1742 aux G
#   cfg3   : 36^3, r2 = 179 -> 10059 PWs, 5448 aux G
#   cfg5   : 40^3, r2 = 283 -> 20005 PWs, 10826 aux G
SPECS = {
    "tiny": ModelSolidSpec("tiny", a=5.0, grid=8, r2=9, wells=1, n_occ=2, n_tau=6, seed=7),
    "tiny2": ModelSolidSpec("tiny2", a=6.0, grid=10, r2=12, wells=2, n_occ=4, n_tau=6, seed=11),
    "cfg1": ModelSolidSpec("cfg1", a=6.0, grid=12, r2=25, wells=2, n_occ=4, n_tau=6, seed=1),
    "cfg2": ModelSolidSpec("cfg2", a=12.0, grid=24, r2=81, wells=16, n_occ=32, n_tau=8, seed=2,
                           lattice_sites=(4, 2, 2)),
    "cfg3": ModelSolidSpec("cfg3", a=24.0, grid=36, r2=179, wells=64, n_occ=128, n_tau=10, seed=3,
                           lattice_sites=(4, 4, 4)),
    "cfg5": ModelSolidSpec("cfg5", a=30.0, grid=40, r2=283, wells=128, n_occ=256, n_tau=10, seed=5,
                           lattice_sites=(8, 4, 4)),
}


def spec_by_name(name: str) -> ModelSolidSpec:
    return SPECS[name]


@dataclasses.dataclass
class ModelSolid:
    """Mean-field input of one system (Gamma point, closed shell).

    lattice  (3,3) rows are the cell vectors (bohr)
    grid     (3,) FFT grid
    miller   (N_pw, 3) int32 plane-wave indices of the orbital sphere
    coeff    (N_orb, N_pw) complex128, rows normalised, ascending energy
    eps      (N_orb,) float64 Hartree
    n_occ    doubly occupied orbitals (the first n_occ rows)
    ecut     orbital cutoff (Ha); the auxiliary cutoff is the caller's choice
    positions (wells, 3) bohr
    """
    spec: Optional[ModelSolidSpec]
    lattice: np.ndarray
    grid: np.ndarray
    miller: np.ndarray
    coeff: np.ndarray
    eps: np.ndarray
    n_occ: int
    ecut: float
    positions: np.ndarray

    @property
    def omega(self) -> float:
        return abs(float(np.linalg.det(self.lattice)))

    @property
    def n_pw(self) -> int:
        return int(self.miller.shape[0])

    @property
    def n_orb(self) -> int:
        return int(self.coeff.shape[0])

    @property
    def gap(self) -> float:
        return float(self.eps[self.n_occ] - self.eps[self.n_occ - 1])

    @property
    def width(self) -> float:
        return float(self.eps[-1] - self.eps[0])

    @property
    def n_atoms(self) -> int:
        return int(self.positions.shape[0])


def sphere_miller(r2: float) -> np.ndarray:
    """All integer m with |m|^2 <= r2, ordered by |m|^2 then lexicographically."""
    R = int(math.floor(math.sqrt(r2))) + 1
    rng = np.arange(-R, R + 1)
    m = np.stack(np.meshgrid(rng, rng, rng, indexing="ij"), -1).reshape(-1, 3)
    s = (m ** 2).sum(1)
    m = m[s <= r2 + 1e-9]
    s = (m ** 2).sum(1)
    order = np.lexsort((m[:, 2], m[:, 1], m[:, 0], s))
    return m[order].astype(np.int32)


def well_positions(spec: ModelSolidSpec) -> np.ndarray:
    rng = np.random.default_rng(spec.seed)
    a = spec.a
    if spec.lattice_sites is None:
        pos: list = []
        tries = 0
        while len(pos) < spec.wells:
            tries += 1
            if tries > 100000:
                raise RuntimeError("could not place wells")
            p = rng.uniform(0.0, a, size=3)
            ok = True
            for q in pos:
                d = p - q
                d -= a * np.round(d / a)
                if np.linalg.norm(d) < spec.min_dist:
                    ok = False
                    break
            if ok:
                pos.append(p)
        return np.array(pos)
    n1, n2, n3 = spec.lattice_sites
    if n1 * n2 * n3 != spec.wells:
        raise ValueError("site lattice does not match the well count")
    idx = np.stack(np.meshgrid(np.arange(n1), np.arange(n2), np.arange(n3), indexing="ij"), -1)
    idx = idx.reshape(-1, 3).astype(np.float64)
    sites = (idx + 0.5) * (a / np.array([n1, n2, n3], dtype=np.float64))
    return sites + rng.normal(0.0, spec.jitter, size=sites.shape)


def _real_basis(miller: np.ndarray) -> np.ndarray:
    """Unitary U (PW basis <- cos/sin basis): columns are real functions in real space."""
    n = miller.shape[0]
    key = {tuple(m): k for k, m in enumerate(miller.tolist())}
    U = np.zeros((n, n), dtype=np.complex128)
    col = 0
    done = np.zeros(n, dtype=bool)
    s = 1.0 / math.sqrt(2.0)
    for k, m in enumerate(miller.tolist()):
        if done[k]:
            continue
        mk = key.get((-m[0], -m[1], -m[2]))
        if mk is None:
            raise ValueError("plane-wave set is not inversion symmetric")
        if mk == k:  # G = 0
            U[k, col] = 1.0
            col += 1
            done[k] = True
            continue
        U[k, col] = s
        U[mk, col] = s
        U[k, col + 1] = -1j * s
        U[mk, col + 1] = 1j * s
        col += 2
        done[k] = done[mk] = True
    assert col == n
    return U


def hamiltonian(miller: np.ndarray, lattice: np.ndarray, positions: np.ndarray,
                depth: float, width: float) -> np.ndarray:
    B = 2.0 * math.pi * np.linalg.inv(lattice).T
    omega = abs(float(np.linalg.det(lattice)))
    G = miller.astype(np.float64) @ B
    dG = G[:, None, :] - G[None, :, :]
    g2 = (dG ** 2).sum(-1)
    pref = -(depth / omega) * (2.0 * math.pi * width ** 2) ** 1.5
    phase = np.zeros(g2.shape, dtype=np.complex128)
    for R in positions:
        phase += np.exp(-1j * (dG @ R))
    H = pref * np.exp(-0.5 * g2 * width ** 2) * phase
    H[np.diag_indices_from(H)] += 0.5 * (G ** 2).sum(-1)
    return H


def _finish(spec, lattice, grid, miller, positions, H, real_orbitals, random_phases, seed):
    if real_orbitals:
        U = _real_basis(miller)
        Hr = (U.conj().T @ H @ U)
        if np.abs(Hr.imag).max() > 1e-10 * max(1.0, np.abs(Hr.real).max()):
            raise RuntimeError("Hamiltonian is not real in the cos/sin basis")
        w, v = np.linalg.eigh(Hr.real)
        coeff = (U @ v).T.copy()
    else:
        w, v = np.linalg.eigh(H)
        coeff = v.T.copy()
    if random_phases:
        rng = np.random.default_rng(seed + 1000)
        coeff *= np.exp(2j * math.pi * rng.random(coeff.shape[0]))[:, None]
    coeff /= np.linalg.norm(coeff, axis=1)[:, None]
    return w, np.ascontiguousarray(coeff)


def build_model_solid(spec: ModelSolidSpec, real_orbitals: bool = True,
                      random_phases: bool = False) -> ModelSolid:
    """Seeded model solid for ``spec`` (dense diagonalisation on the host)."""
    lattice = np.eye(3) * spec.a
    grid = np.array([spec.grid] * 3, dtype=np.int32)
    miller = sphere_miller(spec.r2)
    if 2 * np.abs(miller).max() >= spec.grid:
        raise ValueError("orbital sphere does not fit the grid")
    positions = well_positions(spec)
    H = hamiltonian(miller, lattice, positions, spec.depth, spec.width)
    eps, coeff = _finish(spec, lattice, grid, miller, positions, H, real_orbitals,
                         random_phases, spec.seed)
    return ModelSolid(spec, lattice, grid, miller, coeff, eps, spec.n_occ, spec.ecut, positions)


def free_electron_solid(a: float, grid: int, r2: int, n_occ: int = 1) -> ModelSolid:
    """V = 0: every orbital is one plane wave, eps = |G|^2/2.  n_occ must close a shell."""
    lattice = np.eye(3) * a
    miller = sphere_miller(r2)
    b = 2.0 * math.pi / a
    eps = 0.5 * (miller.astype(np.float64) ** 2).sum(1) * b * b
    order = np.argsort(eps, kind="stable")
    coeff = np.zeros((miller.shape[0], miller.shape[0]), dtype=np.complex128)
    coeff[np.arange(miller.shape[0]), order] = 1.0
    eps = eps[order]
    if n_occ < len(eps) and abs(eps[n_occ] - eps[n_occ - 1]) < 1e-9:
        raise ValueError("n_occ does not close a shell")
    return ModelSolid(None, lattice, np.array([grid] * 3, dtype=np.int32), miller, coeff, eps,
                      n_occ, 0.5 * (r2 + 1e-6) * b * b, np.zeros((0, 3)))

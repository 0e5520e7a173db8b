"""Gaussian-well model solids sampled on a k-point mesh, and the matching Gamma-point
supercell: inputs for the k-point form of the LTMP2 hot path (Sec. II C-D).

A Gamma-centred Monkhorst-Pack mesh n1 x n2 x n3 over the unit cell has the crystal
momenta k = sum_i (kappa_i / n_i) b_i, kappa_i = 0 .. n_i - 1.  Every k uses the same set
of plane-wave Miller indices m (the orbital sphere |G_m|^2/2 <= E_cut); the Bloch orbital
is phi_nk(r) = e^{ik.r} sum_m c_nk(m) e^{iG_m.r} / sqrt(N_k Omega_0), normalised over the
Born-von Karman supercell of N_k cells, and (c_nk, e_nk) diagonalise

    H_pq(k) = 1/2 |k + G_p|^2 delta_pq + V(G_p - G_q)

with the wells' V(G) of ``model_solid``.  The lowest n_occ states of every k are doubly
occupied.  The same potential on the supercell lattice (cell vectors n_i a_i, wells
repeated in every cell) is block diagonal in k; ``supercell_of`` builds that Gamma-point
system in the plane-wave set {k + G_m} (supercell Miller index n_i m_i + kappa_i), so its
MP2 energy per cell equals the k-point MP2 energy exactly.

Nothing here computes any part of MP2.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Sequence, Tuple

import numpy as np

from .model_solid import ModelSolid, _eigh, hamiltonian, sphere_miller


@dataclasses.dataclass
class KPointSolid:
    """Mean-field input on a k-mesh (closed shell).

    lattice (3,3) unit-cell rows; grid (3,) unit-cell FFT grid; mesh (3,) k-mesh;
    kappa (N_k, 3) integer mesh coordinates, k-point index (kappa_1 n_2 + kappa_2) n_3 + kappa_3;
    miller (N_pw, 3) the plane-wave set shared by every k; coeff (N_k, N_orb, N_pw) complex;
    eps (N_k, N_orb) ascending per k; n_occ occupied per k; ecut (Ha); positions (wells, 3).
    """
    lattice: np.ndarray
    grid: np.ndarray
    mesh: np.ndarray
    kappa: np.ndarray
    miller: np.ndarray
    coeff: np.ndarray
    eps: np.ndarray
    n_occ: int
    ecut: float
    positions: np.ndarray
    well_depth: float = 2.0     # A (Ha)
    well_width: float = 0.8     # s (bohr)

    @property
    def n_k(self) -> int:
        return int(self.kappa.shape[0])

    @property
    def n_pw(self) -> int:
        return int(self.miller.shape[0])

    @property
    def n_orb(self) -> int:
        return int(self.coeff.shape[1])

    @property
    def recip(self) -> np.ndarray:
        return 2.0 * math.pi * np.linalg.inv(self.lattice).T

    @property
    def gap(self) -> float:
        """Indirect gap: lowest virtual over all k minus highest occupied over all k."""
        return float(self.eps[:, self.n_occ].min() - self.eps[:, self.n_occ - 1].max())

    @property
    def width(self) -> float:
        return float(self.eps.max() - self.eps.min())

    @property
    def n_atoms(self) -> int:
        return int(self.positions.shape[0])


def mesh_kappa(mesh: Sequence[int]) -> np.ndarray:
    """All kappa of the mesh in k-point index order (axis 3 fastest)."""
    n1, n2, n3 = (int(x) for x in mesh)
    k = np.stack(np.meshgrid(np.arange(n1), np.arange(n2), np.arange(n3), indexing="ij"), -1)
    return k.reshape(-1, 3).astype(np.int64)


def build_kpoint_solid(a: float, grid: int, r2: int, mesh: Sequence[int], positions: np.ndarray, n_occ: int,
                       depth: float = 2.0, width: float = 0.8, random_phases: bool = False,
                       seed: int = 0) -> KPointSolid:
    """Cubic unit cell of side a with wells at ``positions``, the sphere |m|^2 <= r2 (index
    units) as the plane-wave set of every k, dense diagonalisation of H(k) per k."""
    lattice = np.eye(3) * a
    miller = sphere_miller(r2)
    if 2 * np.abs(miller).max() >= grid:
        raise ValueError("orbital sphere does not fit the grid")
    mesh = np.asarray(mesh, dtype=np.int64)
    kappa = mesh_kappa(mesh)
    B = 2.0 * math.pi * np.linalg.inv(lattice).T
    G = miller.astype(np.float64) @ B
    H0 = hamiltonian(miller, lattice, np.asarray(positions, float), depth, width)
    H0[np.diag_indices_from(H0)] -= 0.5 * (G ** 2).sum(-1)
    rng = np.random.default_rng(seed + 2000)
    coeff = np.zeros((len(kappa), len(miller), len(miller)), dtype=np.complex128)
    eps = np.zeros((len(kappa), len(miller)))
    for kk, kap in enumerate(kappa):
        kc = (kap / mesh) @ B
        H = H0.copy()
        H[np.diag_indices_from(H)] += 0.5 * ((G + kc[None, :]) ** 2).sum(-1)
        w, v = np.linalg.eigh(H)
        c = v.T.copy()
        if random_phases:
            c *= np.exp(2j * math.pi * rng.random(c.shape[0]))[:, None]
        coeff[kk] = c / np.linalg.norm(c, axis=1)[:, None]
        eps[kk] = w
    b = 2.0 * math.pi / a
    return KPointSolid(lattice, np.array([grid] * 3, dtype=np.int32), mesh, kappa, miller, coeff, eps, int(n_occ),
                       0.5 * (r2 + 1e-6) * b * b, np.asarray(positions, float), depth, width)


def supercell_of(ks: KPointSolid, device: Optional[str] = None) -> ModelSolid:
    """The Gamma-point supercell of the mesh: cell vectors n_i a_i, grid n_i g_i, wells in
    every cell, plane waves {k + G_m} with supercell Miller index n_i m_i + kappa_i, orbitals
    and energies from a dense diagonalisation of the supercell Hamiltonian in that set (the
    Hamiltonian is block diagonal in k; the diagonalisation does not use that), the lowest
    N_k n_occ states occupied.  ``device="cuda"``: the eigensolver runs on the GPU."""
    mesh = ks.mesh
    lattice = ks.lattice * mesh[:, None]
    shifts = mesh_kappa(mesh)
    pos = np.concatenate([ks.positions + (s @ ks.lattice)[None, :] for s in shifts])
    Msc = np.concatenate([ks.miller * mesh[None, :] + kap[None, :] for kap in ks.kappa]).astype(np.int32)
    grid = (ks.grid * mesh).astype(np.int32)
    if np.any(2 * np.abs(Msc) >= grid[None, :]):
        raise ValueError("supercell plane waves do not fit the supercell grid")
    H = hamiltonian(Msc, lattice, pos, ks.well_depth, ks.well_width)
    w, v = _eigh(H, device)
    coeff = v.T.copy()
    coeff /= np.linalg.norm(coeff, axis=1)[:, None]
    return ModelSolid(None, lattice, grid, Msc, np.ascontiguousarray(coeff), w, ks.n_k * ks.n_occ, ks.ecut, pos)


def build_kpoint_pair(a: float, grid: int, r2: int, mesh: Sequence[int], positions: np.ndarray, n_occ: int,
                      depth: float = 2.0, width: float = 0.8, random_phases: bool = False, seed: int = 0,
                      device: Optional[str] = None):
    """(k-point solid, its Gamma-point supercell) from the same potential."""
    ks = build_kpoint_solid(a, grid, r2, mesh, positions, n_occ, depth, width, random_phases, seed)
    return ks, supercell_of(ks, device)


def free_electron_kpoints(a: float, grid: int, r2: int, mesh: Sequence[int]) -> KPointSolid:
    """V = 0 on a k-mesh: every orbital is one plane wave e^{i(k + G_m) r}, eps = |k + G_m|^2/2,
    one occupied orbital per k (its lowest plane wave; each must be strictly lowest)."""
    lattice = np.eye(3) * a
    miller = sphere_miller(r2)
    mesh = np.asarray(mesh, dtype=np.int64)
    kappa = mesh_kappa(mesh)
    B = 2.0 * math.pi * np.linalg.inv(lattice).T
    G = miller.astype(np.float64) @ B
    coeff = np.zeros((len(kappa), len(miller), len(miller)), dtype=np.complex128)
    eps = np.zeros((len(kappa), len(miller)))
    for kk, kap in enumerate(kappa):
        e = 0.5 * ((G + ((kap / mesh) @ B)[None, :]) ** 2).sum(-1)
        order = np.argsort(e, kind="stable")
        if abs(e[order[1]] - e[order[0]]) < 1e-9:
            raise ValueError("lowest plane wave is degenerate at this k")
        coeff[kk, np.arange(len(miller)), order] = 1.0
        eps[kk] = e[order]
    b = 2.0 * math.pi / a
    return KPointSolid(lattice, np.array([grid] * 3, dtype=np.int32), mesh, kappa, miller, coeff, eps, 1,
                       0.5 * (r2 + 1e-6) * b * b, np.zeros((0, 3)))

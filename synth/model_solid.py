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


# Batching workload: 8 systems of uneven size (wells 4..48, occupied 8..96, grids 16^3..32^3,
# sphere radius 0.375 n index units, a = 6 bohr * wells^(1/3), 6..10 Laplace points).
_BATCH = [(4, 16, 6, (2, 2, 1)), (8, 18, 6, (2, 2, 2)), (12, 20, 7, (3, 2, 2)), (18, 24, 8, (3, 3, 2)),
          (24, 25, 8, (4, 3, 2)), (32, 27, 9, (4, 4, 2)), (40, 30, 10, (5, 4, 2)), (48, 32, 10, (4, 4, 3))]
for _k, (_w, _n, _t, _sites) in enumerate(_BATCH):
    SPECS[f"batch{_k}"] = ModelSolidSpec(f"batch{_k}", a=round(6.0 * _w ** (1.0 / 3.0), 6), grid=_n,
                                         r2=int((0.375 * _n) ** 2), wells=_w, n_occ=2 * _w, n_tau=_t,
                                         seed=41 + _k, lattice_sites=_sites)
BATCH_NAMES = [f"batch{_k}" for _k in range(len(_BATCH))]


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


def hamiltonian(miller: np.ndarray, lattice: np.ndarray, positions: np.ndarray,
                depth: float, width: float) -> np.ndarray:
    """H_pq = |G_p|^2/2 delta_pq + V(G_p - G_q), with V tabulated once on the box of
    Miller-index differences (structure factor over the wells computed per difference)."""
    B = 2.0 * math.pi * np.linalg.inv(lattice).T
    omega = abs(float(np.linalg.det(lattice)))
    R = int(np.abs(miller).max())
    L = 4 * R + 1
    rng = np.arange(-2 * R, 2 * R + 1)
    box = np.stack(np.meshgrid(rng, rng, rng, indexing="ij"), -1).reshape(-1, 3)
    Gb = box.astype(np.float64) @ B
    g2b = (Gb ** 2).sum(-1)
    sf = np.zeros(len(box), dtype=np.complex128)
    for Rw in positions:
        sf += np.exp(-1j * (Gb @ Rw))
    pref = -(depth / omega) * (2.0 * math.pi * width ** 2) ** 1.5
    vbox = pref * np.exp(-0.5 * g2b * width ** 2) * sf
    idx = ((miller[:, 0] + 2 * R) * L + (miller[:, 1] + 2 * R)) * L + (miller[:, 2] + 2 * R)
    # difference m_p - m_q  ->  flat box index idx_p - idx_q + offset of the zero vector
    zero = ((2 * R) * L + 2 * R) * L + 2 * R
    H = vbox[(idx[:, None] - idx[None, :]) + zero]
    G = miller.astype(np.float64) @ B
    H[np.diag_indices_from(H)] += 0.5 * (G ** 2).sum(-1)
    return H


def _real_hamiltonian(miller: np.ndarray, H: np.ndarray):
    """H in the basis {1, cos(G.r), sin(G.r)} (one cos and one sin per +-G pair), built by
    index gathers; returns (Hr real, zero index, primary indices, their negatives)."""
    key = {tuple(m): k for k, m in enumerate(miller.tolist())}
    zero = key[(0, 0, 0)]
    prim, neg = [], []
    for k, m in enumerate(miller.tolist()):
        first = m[0] if m[0] != 0 else (m[1] if m[1] != 0 else m[2])
        if first > 0:
            prim.append(k)
            neg.append(key[(-m[0], -m[1], -m[2])])
    P, Q = np.array(prim), np.array(neg)
    kk, km = H[np.ix_(P, P)], H[np.ix_(P, Q)]
    mk, mm = H[np.ix_(Q, P)], H[np.ix_(Q, Q)]
    cc = 0.5 * (kk + km + mk + mm)
    cs = -0.5j * (kk - km + mk - mm)
    sc = 0.5j * (kk + km - mk - mm)
    ss = 0.5 * (kk - km - mk + mm)
    r2 = 1.0 / math.sqrt(2.0)
    h0c = r2 * (H[zero, P] + H[zero, Q])
    h0s = -1j * r2 * (H[zero, P] - H[zero, Q])
    n = len(P)
    Hr = np.empty((2 * n + 1, 2 * n + 1), dtype=np.complex128)
    Hr[0, 0] = H[zero, zero]
    Hr[0, 1:n + 1], Hr[0, n + 1:] = h0c, h0s
    Hr[1:n + 1, 0], Hr[n + 1:, 0] = np.conj(h0c), np.conj(h0s)
    Hr[1:n + 1, 1:n + 1], Hr[1:n + 1, n + 1:] = cc, cs
    Hr[n + 1:, 1:n + 1], Hr[n + 1:, n + 1:] = sc, ss
    return Hr, zero, P, Q


def _eigh(h: np.ndarray, device: Optional[str]):
    """Dense symmetric / Hermitian eigendecomposition (ascending), FP64.  ``device`` None:
    numpy on the host; "cuda": torch.linalg.eigh on the GPU (the same decomposition, faster
    for the 10^4-plane-wave workloads; input generation only)."""
    if device is None:
        return np.linalg.eigh(h)
    import torch
    t = torch.from_numpy(np.ascontiguousarray(h)).to(device)
    w, v = torch.linalg.eigh(t)
    out = w.cpu().numpy(), v.cpu().numpy()
    del t, w, v
    torch.cuda.empty_cache()
    return out


def _finish(spec, lattice, grid, miller, positions, H, real_orbitals, random_phases, seed, device=None):
    if real_orbitals:
        Hr, zero, P, Q = _real_hamiltonian(miller, H)
        if np.abs(Hr.imag).max() > 1e-10 * max(1.0, np.abs(Hr.real).max()):
            raise RuntimeError("Hamiltonian is not real in the cos/sin basis")
        Hr = Hr.real
        w, v = _eigh(Hr, device)
        n = len(P)
        coeff = np.zeros((H.shape[0], H.shape[0]), dtype=np.complex128)
        r2 = 1.0 / math.sqrt(2.0)
        vt = v.T
        coeff[:, zero] = vt[:, 0]
        coeff[:, P] = r2 * (vt[:, 1:n + 1] - 1j * vt[:, n + 1:])
        coeff[:, Q] = r2 * (vt[:, 1:n + 1] + 1j * vt[:, n + 1:])
    else:
        w, v = _eigh(H, device)
        coeff = v.T.copy()
    if random_phases:
        rng = np.random.default_rng(seed + 1000)
        coeff *= np.exp(2j * math.pi * rng.random(coeff.shape[0]))[:, None]
    coeff /= np.linalg.norm(coeff, axis=1)[:, None]
    return w, np.ascontiguousarray(coeff)


def build_model_solid(spec: ModelSolidSpec, real_orbitals: bool = True,
                      random_phases: bool = False, device: Optional[str] = None) -> ModelSolid:
    """Seeded model solid for ``spec`` (dense diagonalisation on the host, or with
    ``device="cuda"`` on the GPU)."""
    lattice = np.eye(3) * spec.a
    grid = np.array([spec.grid] * 3, dtype=np.int32)
    miller = sphere_miller(spec.r2)
    if 2 * np.abs(miller).max() >= spec.grid:
        raise ValueError("orbital sphere does not fit the grid")
    positions = well_positions(spec)
    H = hamiltonian(miller, lattice, positions, spec.depth, spec.width)
    eps, coeff = _finish(spec, lattice, grid, miller, positions, H, real_orbitals,
                         random_phases, spec.seed, device)
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


def spin_polarized_pair(spec: ModelSolidSpec, n_occ_alpha: int, n_occ_beta: int,
                        depth_beta: Optional[float] = None,
                        real_orbitals: bool = True) -> Tuple[ModelSolid, ModelSolid]:
    """Synthetic spin-unrestricted mean field: the same cell, wells and plane-wave set for
    both spins; the beta electrons see wells of depth ``depth_beta`` (default 0.9 x the
    alpha depth), so the two orbital sets differ.  ``n_occ_*`` singly occupied orbitals."""
    a = build_model_solid(dataclasses.replace(spec, n_occ=n_occ_alpha), real_orbitals=real_orbitals)
    db = 0.9 * spec.depth if depth_beta is None else depth_beta
    b = build_model_solid(dataclasses.replace(spec, n_occ=n_occ_beta, depth=db), real_orbitals=real_orbitals)
    return a, b

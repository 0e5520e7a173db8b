"""Plain FP64 CPU oracle: closed-shell Gamma-point MP2 with explicit sums over
occupied (i, j) and virtual (a, b) orbitals.

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code with
the CUDA path.

What it computes (Schaefer, Ramberger, Kresse, "Quartic scaling MP2 for
solids", arXiv:1611.06797):

* Overlap densities, Eq. (SCHovrlp):  rho_mn(G) = <m| e^{-iGr} |n>, on the FFT
  grid.  With phi_n(r_t) = Omega^{-1/2} sum_p c_n(p) e^{i G_p r_t} this is the
  wrapped plane-wave convolution  sum_p conj(c_m(p)) c_n((G_p + G) mod grid).
  Three independent routes are provided: that convolution (``_conv``), a numpy
  FFT of the real-space product (``_fft``) and an explicit O(N_FFT^2) DFT
  (``_dft``).
* Two-electron integrals in reciprocal space, Eq. (SCH2EI):
  <ij|ab> = (1/Omega) sum_{G in A} 4 pi / G^2  rho_ia(G) rho_jb(-G),
  A = {G != 0 : G^2/2 <= E_cut^aux} (Sec. II A: the auxiliary cutoff).
* Closed-shell MP2, Eq. (CanMP2) with the spin sums of Eqs. (MP2direct) and
  (MP2exchange) done (sum_{ss'} -> 4, sum_s -> 2, prefactor 1/2):
     E_d = 2 sum_ijab |<ij|ab>|^2 D(e_i + e_j - e_a - e_b)
     E_x = - sum_ijab <ij|ab> <ab|ji> D(e_i + e_j - e_a - e_b)
  with D(Delta) = 1/Delta (canonical) or, Eq. (SCHLT) / Eq. (LTMP2) with a
  quadrature, D(Delta) = - sum_k w_k exp(Delta tau_k).
  The pair energy e_ij is the (i, j) term of E_d + E_x; it is symmetric.

Readings where the paper is silent (each is listed in the design notes):
* the G = 0 Coulomb term is dropped (v(0) := 0);
* integrals use the grid-discrete overlap densities (aliasing included);
* the quadrature is an input; ``sinc_laplace_quadrature`` is this oracle's
  own, simple, exponentially convergent rule for 1/x (trapezoid rule in
  t = ln tau), used only by its tests.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, Iterable, Optional, Sequence, Tuple

import numpy as np


@dataclasses.dataclass
class OracleSystem:
    """Gamma-point, closed-shell mean-field input.

    lattice (3,3) rows = cell vectors; grid (3,); miller (N_pw,3);
    coeff (N_orb, N_pw) complex; eps (N_orb,) ascending; n_occ; ecut_aux (Ha).
    """
    lattice: np.ndarray
    grid: np.ndarray
    miller: np.ndarray
    coeff: np.ndarray
    eps: np.ndarray
    n_occ: int
    ecut_aux: float

    @property
    def omega(self) -> float:
        return abs(float(np.linalg.det(self.lattice)))

    @property
    def recip(self) -> np.ndarray:
        # rows b_k with a_i . b_k = 2 pi delta_ik
        return 2.0 * math.pi * np.linalg.inv(self.lattice).T

    @classmethod
    def from_solid(cls, solid, ecut_aux: Optional[float] = None) -> "OracleSystem":
        if ecut_aux is None:
            ecut_aux = 2.0 * solid.ecut / 3.0   # "commonly 2/3 E_cut" (Sec. II A)
        return cls(np.asarray(solid.lattice, float), np.asarray(solid.grid, int),
                   np.asarray(solid.miller, int), np.asarray(solid.coeff, complex),
                   np.asarray(solid.eps, float), int(solid.n_occ), float(ecut_aux))


# ---------------------------------------------------------------------------
# Auxiliary G set and Coulomb kernel (Sec. II A; Eq. SCH2EI; Eq. CoulombFourier)
# ---------------------------------------------------------------------------
def aux_set(sys: OracleSystem):
    """A = {G != 0 : |G|^2 / 2 <= E_cut^aux} as integer indices, |G|^2 and v(G) = 4 pi / G^2."""
    B = sys.recip
    # bound the search box by the shortest reciprocal direction
    gmax = math.sqrt(2.0 * sys.ecut_aux)
    # |m_k| <= gmax * |a_k| / (2 pi)
    lim = [int(math.floor(gmax * np.linalg.norm(sys.lattice[k]) / (2 * math.pi))) + 1
           for k in range(3)]
    rng = [np.arange(-l, l + 1) for l in lim]
    m = np.stack(np.meshgrid(*rng, indexing="ij"), -1).reshape(-1, 3)
    G = m @ B
    g2 = (G ** 2).sum(1)
    keep = (0.5 * g2 <= sys.ecut_aux) & (g2 > 0)
    m, g2 = m[keep], g2[keep]
    n = sys.grid
    flat = _flat(m, n)
    if len(np.unique(flat)) != len(flat):
        raise ValueError("auxiliary sphere does not fit the FFT grid")
    v = 4.0 * math.pi / g2
    return m, g2, v


def _flat(m: np.ndarray, grid: np.ndarray) -> np.ndarray:
    """Flat index of (m mod grid) in C order (axis 0 slowest)."""
    w = np.mod(m, grid)
    return (w[:, 0] * grid[1] + w[:, 1]) * grid[2] + w[:, 2]


def _neg_index(m: np.ndarray) -> np.ndarray:
    """Position of -m in the list m."""
    key = {tuple(r): k for k, r in enumerate(m.tolist())}
    return np.array([key[(-r[0], -r[1], -r[2])] for r in m.tolist()])


# ---------------------------------------------------------------------------
# Overlap densities, Eq. (SCHovrlp), three independent routes
# ---------------------------------------------------------------------------
def overlap_densities_conv(sys: OracleSystem, left: Sequence[int], right: Sequence[int],
                           gvec: np.ndarray) -> np.ndarray:
    """rho[l, r, g] = sum_p conj(c_l(p)) c_r((G_p + G_g) mod grid): wrapped convolution."""
    n = sys.grid
    ngrid = int(np.prod(n))
    cgrid = np.zeros((len(right), ngrid), dtype=np.complex128)
    fp = _flat(sys.miller, n)
    cgrid[:, fp] = sys.coeff[list(right)]
    cl = np.conj(sys.coeff[list(left)])                       # (L, N_pw)
    out = np.empty((len(left), len(right), len(gvec)), dtype=np.complex128)
    for g, G in enumerate(gvec):
        idx = _flat(sys.miller + G[None, :], n)               # (N_pw,)
        shifted = cgrid[:, idx]                               # (R, N_pw)
        out[:, :, g] = cl @ shifted.T
    return out


def _real_space(sys: OracleSystem, orbs: Sequence[int]) -> np.ndarray:
    """u_n(r_t) = sum_p c_n(p) exp(i G_p r_t)  (= Omega^{1/2} phi_n), shape (len, n1, n2, n3)."""
    n = tuple(int(x) for x in sys.grid)
    grid = np.zeros((len(orbs),) + n, dtype=np.complex128)
    w = np.mod(sys.miller, sys.grid)
    grid[:, w[:, 0], w[:, 1], w[:, 2]] = sys.coeff[list(orbs)]
    return np.fft.ifftn(grid, axes=(1, 2, 3)) * float(np.prod(n))


def overlap_densities_fft(sys: OracleSystem, left: Sequence[int], right: Sequence[int],
                          gvec: np.ndarray, chunk: int = 256) -> np.ndarray:
    """rho[l, r, g] = (Omega/N) sum_t phi_l*(r_t) phi_r(r_t) e^{-i G r_t}  via numpy's FFT."""
    n = sys.grid
    N = float(np.prod(n))
    ul = _real_space(sys, left)
    w = np.mod(gvec, n)
    out = np.empty((len(left), len(right), len(gvec)), dtype=np.complex128)
    right = list(right)
    for s in range(0, len(right), chunk):
        ur = _real_space(sys, right[s:s + chunk])
        for li in range(len(left)):
            prod = np.conj(ul[li])[None] * ur
            F = np.fft.fftn(prod, axes=(1, 2, 3)) / N
            out[li, s:s + len(ur)] = F[:, w[:, 0], w[:, 1], w[:, 2]]
    return out


def overlap_densities_dft(sys: OracleSystem, left: Sequence[int], right: Sequence[int],
                          gvec: np.ndarray) -> np.ndarray:
    """Same quantity by an explicit real-space sum with exp(-i G r_t): O(N_FFT) per value, no FFT."""
    n = sys.grid
    t = np.stack(np.meshgrid(*[np.arange(k) for k in n], indexing="ij"), -1).reshape(-1, 3)
    frac = t / n[None, :]                                      # r_t in lattice coordinates
    # orbitals in real space by explicit plane-wave sums
    ph = np.exp(2j * math.pi * (frac @ sys.miller.T))          # (N_FFT, N_pw)
    ul = ph @ sys.coeff[list(left)].T                          # (N_FFT, L)
    ur = ph @ sys.coeff[list(right)].T
    eg = np.exp(-2j * math.pi * (frac @ gvec.T))               # (N_FFT, N_G)
    N = float(np.prod(n))
    prod = np.conj(ul)[:, :, None] * ur[:, None, :]            # (N_FFT, L, R)
    return np.einsum("tlr,tg->lrg", prod, eg) / N


# ---------------------------------------------------------------------------
# Two-electron integrals, Eq. (SCH2EI)
# ---------------------------------------------------------------------------
def pair_integrals(rho_i: np.ndarray, rho_j_neg: np.ndarray, v: np.ndarray,
                   omega: float) -> np.ndarray:
    """K[a, b] = <ij|ab> = (1/Omega) sum_G v(G) rho_ia(G) rho_jb(-G).

    rho_i[a, G] = rho_ia(G); rho_j_neg[b, G] = rho_jb(-G).
    """
    return (rho_i * (v / omega)[None, :]) @ rho_j_neg.T


# ---------------------------------------------------------------------------
# Energy denominators: canonical (Eq. CanMP2) and Laplace quadrature (Eq. SCHLT)
# ---------------------------------------------------------------------------
def canonical_denominator(delta: np.ndarray) -> np.ndarray:
    return 1.0 / delta


def laplace_denominator(tau: np.ndarray, w: np.ndarray) -> Callable[[np.ndarray], np.ndarray]:
    """D(Delta) = - sum_k w_k exp(Delta tau_k)  (1/Delta = -int_0^inf exp(Delta tau) dtau)."""
    tau = np.asarray(tau, float)
    w = np.asarray(w, float)

    def D(delta: np.ndarray) -> np.ndarray:
        out = np.zeros_like(delta)
        for tk, wk in zip(tau, w):
            out -= wk * np.exp(delta * tk)
        return out
    return D


def mp2_pair_energy(K: np.ndarray, eps_i: float, eps_j: float, eps_v: np.ndarray,
                    D: Callable[[np.ndarray], np.ndarray]) -> Tuple[float, float, float]:
    """(i, j) term of the closed-shell direct and exchange energies.

    K[a, b] = <ij|ab>.  <ab|ij> = conj(<ij|ab>) and <ab|ji> = conj(<ij|ba>), so
      e_d = 2 sum_ab |K_ab|^2 D_ab,    e_x = - sum_ab K_ab conj(K_ba) D_ab.
    Returns (e_d, e_x, imaginary residue of e_x).
    """
    Dab = D(eps_i + eps_j - eps_v[:, None] - eps_v[None, :])
    ed = 2.0 * float(np.sum((K.real ** 2 + K.imag ** 2) * Dab))
    xsum = np.sum(K * np.conj(K.T) * Dab)
    return ed, -float(xsum.real), float(xsum.imag)


def mp2_energy(sys: OracleSystem, D: Callable[[np.ndarray], np.ndarray],
               pairs: Optional[Iterable[Tuple[int, int]]] = None, method: str = "auto",
               rho_cache: Optional[dict] = None):
    """Closed-shell MP2 with explicit sums over i, j, a, b.

    Returns dict with E_d, E_x, E, and e_d / e_x pair matrices (only the
    requested ordered pairs are filled; NaN elsewhere).
    """
    no = sys.n_occ
    virt = list(range(no, sys.coeff.shape[0]))
    mG, _, v = aux_set(sys)
    neg = _neg_index(mG)
    if pairs is None:
        pairs = [(i, j) for i in range(no) for j in range(no)]
    pairs = list(pairs)
    occ_needed = sorted({p for pr in pairs for p in pr})
    if method == "auto":
        method = "conv" if sys.coeff.shape[1] * len(mG) * len(virt) < 4e8 else "fft"
    rho = {} if rho_cache is None else rho_cache
    missing = [i for i in occ_needed if i not in rho]
    if missing:
        fn = {"conv": overlap_densities_conv, "fft": overlap_densities_fft,
              "dft": overlap_densities_dft}[method]
        r = fn(sys, missing, virt, mG)
        for k, i in enumerate(missing):
            rho[i] = r[k]
    eps_v = sys.eps[no:]
    ed = np.full((no, no), np.nan)
    ex = np.full((no, no), np.nan)
    exi = np.full((no, no), np.nan)
    for (i, j) in pairs:
        K = pair_integrals(rho[i], rho[j][:, neg], v, sys.omega)
        d, x, xi = mp2_pair_energy(K, sys.eps[i], sys.eps[j], eps_v, D)
        ed[i, j], ex[i, j], exi[i, j] = d, x, xi
    full = len(pairs) == no * no
    out = {"e_d": ed, "e_x": ex, "e_x_imag": exi}
    if full:
        out["E_d"] = float(np.sum(ed))
        out["E_x"] = float(np.sum(ex))
        out["E"] = out["E_d"] + out["E_x"]
    return out


# ---------------------------------------------------------------------------
# Quadrature for 1/x (the oracle's own; the paper cites a minimax grid, Sec. II C)
# ---------------------------------------------------------------------------
def denominator_range(sys: OracleSystem) -> Tuple[float, float]:
    """[min, max] of -(e_i + e_j - e_a - e_b) over the system."""
    no = sys.n_occ
    lo = 2.0 * (sys.eps[no] - sys.eps[no - 1])
    hi = 2.0 * (sys.eps[-1] - sys.eps[0])
    return lo, hi


def sinc_laplace_quadrature(n: int, xmin: float, xmax: float) -> Tuple[np.ndarray, np.ndarray]:
    """Exponential-sum rule for 1/x on [xmin, xmax] (the oracle's own).

    1/x = int_0^inf exp(-x tau) dtau = int_{-inf}^{inf} exp(-x e^t) e^t dt.  The
    t-integrand is analytic in the strip |Im t| < pi/2, so the trapezoid rule with
    step h has relative error ~ exp(-pi^2 / h).  The infinite sum is cut where
    the dropped tails are of the same size: t_lo = ln(eps / xmax) (the left tail
    contributes ~ x e^{t_lo}) and t_hi = ln(C / xmin) with exp(-C) = eps (the
    right tail contributes ~ exp(-x e^{t_hi})).  n nodes then fix h by the
    fixed point L(h) = n h.
    """
    if n < 1:
        raise ValueError("n must be >= 1")
    R = xmax / xmin
    h = 1.0
    for _ in range(200):
        C = math.pi ** 2 / h
        L = math.log(C * R) + C
        h_new = L / n
        if abs(h_new - h) < 1e-14 * h:
            break
        h = 0.5 * (h + h_new)
    C = math.pi ** 2 / h
    t_lo = math.log(math.exp(-C) / xmax)
    t = t_lo + h * (np.arange(n) + 0.5)
    tau = np.exp(t)
    w = h * tau
    return tau, w


def quadrature_max_error(tau: np.ndarray, w: np.ndarray, xmin: float, xmax: float,
                         samples: int = 10000) -> float:
    """max over log-spaced x in [xmin, xmax] of |1 - x sum_k w_k exp(-x tau_k)|."""
    x = np.geomspace(xmin, xmax, samples)
    s = np.exp(-np.outer(x, tau)) @ w
    return float(np.max(np.abs(1.0 - x * s)))


# ---------------------------------------------------------------------------
# Internal auxiliary-cutoff extrapolation (Sec. III D, Eq. CutDecay)
# ---------------------------------------------------------------------------
def cutoff_levels(ecut_aux: float, n_c: int = 8, alpha: float = 1.05) -> np.ndarray:
    """The nested auxiliary cutoffs E_aux[n] = E_aux / alpha^(n-1), n = 1..n_c."""
    if n_c < 1 or not alpha > 1.0:
        raise ValueError("need n_c >= 1 and alpha > 1")
    return ecut_aux / alpha ** np.arange(n_c, dtype=float)


def level_energies(sys: OracleSystem, D: Callable[[np.ndarray], np.ndarray], n_c: int = 8,
                   alpha: float = 1.05):
    """MP2 energies with every auxiliary G-sum (both the inner G and the outer G' of
    Eq. SCHfocklike / dLTMP2Compact) truncated at each nested cutoff E_aux[n].

    Written as its definition: the whole calculation repeated with A replaced by
    A_n = {G != 0 : |G|^2/2 <= E_aux[n]}.  Returns (ecut[n], |A_n|, E_d[n], E_x[n]).
    """
    ecut = cutoff_levels(sys.ecut_aux, n_c, alpha)
    counts, ed, ex = [], [], []
    for e in ecut:
        s = dataclasses.replace(sys, ecut_aux=float(e))
        counts.append(len(aux_set(s)[0]))
        r = mp2_energy(s, D)
        ed.append(r["E_d"])
        ex.append(r["E_x"])
    return ecut, np.array(counts), np.array(ed), np.array(ex)


def cutoff_extrapolation(ecut: Sequence[float], energy: Sequence[float]) -> Tuple[float, float, float]:
    """Least-squares line y = a + b x through y = E[n], x = E_aux[n]^(-3/2) (Eq. CutDecay).

    Returns (a, b, sigma_a); a is the energy extrapolated to an infinite auxiliary
    cutoff and sigma_a its standard error from the fit residuals (the paper quotes
    such a fitting error with its extrapolated energies, Sec. IV C; 0 for two points).
    The normal equations of the straight-line fit, written out.
    """
    x = np.asarray(ecut, float) ** -1.5
    y = np.asarray(energy, float)
    if len(x) < 2:
        raise ValueError("need at least two cutoffs")
    n = float(len(x))
    sx, sy = float(np.sum(x)), float(np.sum(y))
    sxx, sxy = float(np.sum(x * x)), float(np.sum(x * y))
    det = n * sxx - sx * sx
    b = (n * sxy - sx * sy) / det
    a = (sy - b * sx) / n
    sa = 0.0
    if len(x) > 2:
        s2 = float(np.sum((y - a - b * x) ** 2)) / (n - 2.0)
        sa = math.sqrt(s2 * sxx / det)
    return a, b, sa


# ---------------------------------------------------------------------------
# Spin-unrestricted MP2 (Eqs. MP2direct, MP2exchange with independent spin sums)
# ---------------------------------------------------------------------------
def uhf_mp2_energy(sa: OracleSystem, sb: OracleSystem, D: Callable[[np.ndarray], np.ndarray]):
    """E_d = 1/2 sum_{s s'} sum_{i in occ s, j in occ s'} sum_{a in virt s, b in virt s'}
                 |<i j|a b>|^2 D(e_i + e_j - e_a - e_b)
       E_x = -1/2 sum_s sum_{i j in occ s} sum_{a b in virt s} <i j|a b> <a b|j i> D(...)
    with spatial integrals <ij|ab> (Eq. SCH2EI) between orbitals of the stated spins.
    sa, sb: the two spin channels (same lattice, grid, plane waves and E_aux); each
    ``n_occ`` counts singly occupied orbitals and may be 0.  Returns E_d, E_x and the
    same-spin (alpha alpha, beta beta) and opposite-spin parts of E = E_d + E_x."""
    mG, _, v = aux_set(sa)
    neg = _neg_index(mG)
    spins = [sa, sb]
    rho = []
    for s in spins:
        occ = list(range(s.n_occ))
        virt = list(range(s.n_occ, s.coeff.shape[0]))
        rho.append(overlap_densities_conv(s, occ, virt, mG) if occ else [])
    E_d = E_x = 0.0
    part = {"aa": 0.0, "bb": 0.0, "ab": 0.0}
    for x in (0, 1):
        for y in (0, 1):
            sx, sy = spins[x], spins[y]
            ev_x, ev_y = sx.eps[sx.n_occ:], sy.eps[sy.n_occ:]
            for i in range(sx.n_occ):
                for j in range(sy.n_occ):
                    K = pair_integrals(rho[x][i], rho[y][j][:, neg], v, sa.omega)
                    Dab = D(sx.eps[i] + sy.eps[j] - ev_x[:, None] - ev_y[None, :])
                    d = 0.5 * float(np.sum((K.real ** 2 + K.imag ** 2) * Dab))
                    e = d
                    E_d += d
                    if x == y:
                        xx = -0.5 * float(np.sum(K * np.conj(K.T) * Dab).real)
                        E_x += xx
                        e += xx
                    part["ab" if x != y else ("aa" if x == 0 else "bb")] += e
    return {"E_d": E_d, "E_x": E_x, "E": E_d + E_x, "E_aa": part["aa"], "E_bb": part["bb"], "E_ab": part["ab"]}


# ---------------------------------------------------------------------------
# k-point sampling (Sec. II C-D): Eqs. (MP2direct), (MP2exchange) per unit cell with the
# integrals of Eq. (2eIPLWV) and crystal-momentum conservation k1 + k2 = k3 + k4 + G
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class KPointOracleSystem:
    """Closed-shell mean field on a Gamma-centred k-mesh (k = sum_i kappa_i / n_i b_i).

    lattice (3,3) unit-cell rows; grid (3,) unit-cell FFT grid; mesh (3,); kappa (N_k,3);
    miller (N_pw,3) plane-wave set shared by every k; coeff (N_k, N_orb, N_pw) with
    phi_nk = e^{ikr} sum_m c_nk(m) e^{iG_m r} / sqrt(N_k Omega_0); eps (N_k, N_orb); n_occ
    per k; ecut_aux (Ha): the auxiliary set is {Q : |Q|^2/2 <= E_aux, Q != 0} over all
    momentum transfers Q = G + k' - k.
    """
    lattice: np.ndarray
    grid: np.ndarray
    mesh: np.ndarray
    kappa: np.ndarray
    miller: np.ndarray
    coeff: np.ndarray
    eps: np.ndarray
    n_occ: int
    ecut_aux: float

    @property
    def n_k(self) -> int:
        return int(self.kappa.shape[0])

    @property
    def omega0(self) -> float:
        return abs(float(np.linalg.det(self.lattice)))

    @property
    def recip(self) -> np.ndarray:
        return 2.0 * math.pi * np.linalg.inv(self.lattice).T

    @classmethod
    def from_solid(cls, ks, ecut_aux: Optional[float] = None) -> "KPointOracleSystem":
        if ecut_aux is None:
            ecut_aux = 2.0 * ks.ecut / 3.0
        return cls(np.asarray(ks.lattice, float), np.asarray(ks.grid, int), np.asarray(ks.mesh, int),
                   np.asarray(ks.kappa, int), np.asarray(ks.miller, int), np.asarray(ks.coeff, complex),
                   np.asarray(ks.eps, float), int(ks.n_occ), float(ecut_aux))


def kpoint_aux_class(sys: KPointOracleSystem, delta: np.ndarray):
    """The auxiliary momentum transfers of one class: Q = g + delta / mesh for the integer
    vector delta = kappa' - kappa (each component in (-n_i, n_i)), |Q|^2/2 <= E_aux, Q != 0.
    Returns integer g (n,3), the supercell Miller indices M = mesh g + delta (n,3), and
    v(Q) = 4 pi / |Q|^2 (Eq. 2eIPLWV, Eq. CoulombFourier)."""
    B = sys.recip
    gmax = math.sqrt(2.0 * sys.ecut_aux)
    lim = [int(math.floor(gmax * np.linalg.norm(sys.lattice[k]) / (2 * math.pi))) + 2 for k in range(3)]
    rng = [np.arange(-l, l + 1) for l in lim]
    g = np.stack(np.meshgrid(*rng, indexing="ij"), -1).reshape(-1, 3)
    s = np.asarray(delta, float) / sys.mesh
    Q = (g + s[None, :]) @ B
    q2 = (Q ** 2).sum(1)
    keep = (0.5 * q2 <= sys.ecut_aux) & (q2 > 1e-20)
    g, q2 = g[keep], q2[keep]
    if len(np.unique(_flat(g, sys.grid))) != len(g):
        raise ValueError("auxiliary sphere does not fit the FFT grid")
    return g, g * sys.mesh[None, :] + np.asarray(delta)[None, :], 4.0 * math.pi / q2


def kpoint_overlap_densities(sys: KPointOracleSystem, kl: int, left: Sequence[int], kr: int,
                             right: Sequence[int], gvec: np.ndarray) -> np.ndarray:
    """rho[l, r, g] = sum_p conj(c_{l,kl}(p)) c_{r,kr}((G_p + g) mod grid): the overlap density
    <l kl| e^{-iQr} |r kr> of Eq. (OverlapDens) at Q = g + k_r - k_l, grid-discrete like the
    Gamma-point densities (the wrap of G_p + g on the FFT grid)."""
    n = sys.grid
    ngrid = int(np.prod(n))
    cgrid = np.zeros((len(right), ngrid), dtype=np.complex128)
    cgrid[:, _flat(sys.miller, n)] = sys.coeff[kr][list(right)]
    cl = np.conj(sys.coeff[kl][list(left)])
    out = np.empty((len(left), len(right), len(gvec)), dtype=np.complex128)
    for gi, gg in enumerate(gvec):
        out[:, :, gi] = cl @ cgrid[:, _flat(sys.miller + gg[None, :], n)].T
    return out


def kpoint_mp2_energy(sys: KPointOracleSystem, D: Callable[[np.ndarray], np.ndarray]):
    """Closed-shell MP2 per unit cell on the k-mesh, explicit sums over k1, k2, k3 (k4 fixed
    by crystal-momentum conservation, Eq. 2eIPLWV), i, j, a, b:
       <i k1, j k2|a k3, b k4> = (1/Omega) sum_Q v(Q) rho_{i k1, a k3}(Q) rho_{j k2, b k4}(-Q),
       Omega = N_k Omega_0,  Q over the class of k3 - k1,
       E_d = (2 / N_k) sum |<ij|ab>|^2 D,   E_x = -(1 / N_k) sum <ij|ab> <ab|ji> D,
    <ab|ji> = conj(<ij|ba>), D = D(e_{i k1} + e_{j k2} - e_{a k3} - e_{b k4}).
    Returns E_d, E_x, E (Ha per unit cell) and pair matrices e_d, e_x over composite
    occupied indices k n_occ + i."""
    nk, no = sys.n_k, sys.n_occ
    norb = sys.coeff.shape[1]
    occ, virt = list(range(no)), list(range(no, norb))
    index = {tuple(k): n for n, k in enumerate(sys.kappa.tolist())}
    omega = nk * sys.omega0
    cache = {}

    def dens(k, kp):
        if (k, kp) not in cache:
            g, M, v = kpoint_aux_class(sys, sys.kappa[kp] - sys.kappa[k])
            rho = kpoint_overlap_densities(sys, k, occ, kp, virt, g)
            cache[(k, kp)] = (rho, M, v, {tuple(m): q for q, m in enumerate(M.tolist())})
        return cache[(k, kp)]

    e_d = np.zeros((nk * no, nk * no))
    e_x = np.zeros((nk * no, nk * no))
    for k1 in range(nk):
        for k2 in range(nk):
            for k3 in range(nk):
                k4 = index[tuple(np.mod(sys.kappa[k1] + sys.kappa[k2] - sys.kappa[k3], sys.mesh))]
                rA, MA, vA, _ = dens(k1, k3)          # i k1 -> a k3 at Q
                rB, _, _, dB = dens(k2, k4)           # j k2 -> b k4 at -Q
                rC, MC, vC, _ = dens(k1, k4)          # i k1 -> b k4 at Q   (exchange integral)
                rD, _, _, dD = dens(k2, k3)           # j k2 -> a k3 at -Q
                nb = [dB[tuple(-m)] for m in MA]
                nd = [dD[tuple(-m)] for m in MC]
                ev3, ev4 = sys.eps[k3, no:], sys.eps[k4, no:]
                for i in range(no):
                    for j in range(no):
                        K = (rA[i] * (vA / omega)[None, :]) @ rB[j][:, nb].T        # <i k1, j k2|a k3, b k4>[a, b]
                        Kx = (rC[i] * (vC / omega)[None, :]) @ rD[j][:, nd].T       # <i k1, j k2|b k4, a k3>[b, a]
                        Dab = D(sys.eps[k1, i] + sys.eps[k2, j] - ev3[:, None] - ev4[None, :])
                        e_d[k1 * no + i, k2 * no + j] += 2.0 * float(np.sum((K.real ** 2 + K.imag ** 2) * Dab)) / nk
                        e_x[k1 * no + i, k2 * no + j] -= float(np.sum(K * np.conj(Kx.T) * Dab).real) / nk
    Ed, Ex = float(e_d.sum()), float(e_x.sum())
    return {"E_d": Ed, "E_x": Ex, "E": Ed + Ex, "e_d": e_d, "e_x": e_x}

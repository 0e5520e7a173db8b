"""ctypes binding of libltmp2 (include/ltmp2.h), one Python function per C entry point.

Argument marshalling only.  A missing library raises; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Tuple

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libltmp2.so")

FP64 = 0
FP32 = 1
FLAG_REAL_ORBITALS = 1
FLAG_SIMT_GEMM = 2
NUM_STAGES = 7
STAGE_NAMES = ["green_gemm", "w_gemm", "gather_ztransform", "plane_fft", "column_fft_contract",
               "direct_contract", "accumulate"]
HARTREE_TO_MEV = 27211.386245988

_ERRORS = {0: "OK", -1: "INVALID_ARG", -2: "GAP", -3: "NOT_ORTHONORMAL", -4: "GRID", -5: "OOM",
           -6: "CUDA", -7: "TIMEOUT", -8: "UNSUPPORTED", -9: "NO_CONVERGENCE", -10: "NOT_REAL"}


class Ltmp2Error(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        self.name = _ERRORS.get(code, str(code))
        super().__init__(f"{where}: {self.name} ({ltmp2_strerror(code)})")


class _System(ctypes.Structure):
    _fields_ = [("lattice", ctypes.c_double * 9), ("grid", ctypes.c_int * 3), ("n_pw", ctypes.c_int),
                ("miller", ctypes.POINTER(ctypes.c_int)), ("n_orb", ctypes.c_int), ("n_occ", ctypes.c_int),
                ("coeff", ctypes.POINTER(ctypes.c_double)), ("eps", ctypes.POINTER(ctypes.c_double)),
                ("ecut_aux", ctypes.c_double), ("precision", ctypes.c_int), ("flags", ctypes.c_int)]


class _KSystem(ctypes.Structure):
    _fields_ = [("lattice", ctypes.c_double * 9), ("grid", ctypes.c_int * 3), ("mesh", ctypes.c_int * 3),
                ("n_pw", ctypes.c_int), ("miller", ctypes.POINTER(ctypes.c_int)), ("n_orb", ctypes.c_int),
                ("n_occ", ctypes.c_int), ("coeff", ctypes.POINTER(ctypes.c_double)),
                ("eps", ctypes.POINTER(ctypes.c_double)), ("ecut_aux", ctypes.c_double),
                ("precision", ctypes.c_int), ("flags", ctypes.c_int)]


_lib = None


def load_library():
    """Load libltmp2.so (built in-tree by ``paper_1611_06797_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    dp = P(ctypes.c_double)
    vp = ctypes.c_void_p
    sig = {
        "ltmp2_setup": (ctypes.c_int, [P(_System), P(vp)]),
        "ltmp2_setup_kpoints": (ctypes.c_int, [P(_KSystem), P(vp)]),
        "ltmp2_set_stream": (ctypes.c_int, [vp, vp]),
        "ltmp2_laplace_grid": (ctypes.c_int, [ctypes.c_double, ctypes.c_double, ctypes.c_int, dp, dp, dp]),
        "ltmp2_energy": (ctypes.c_int, [vp, ctypes.c_int, dp, dp, dp, dp, dp]),
        "ltmp2_energy_partial": (ctypes.c_int, [vp, ctypes.c_int, dp, dp, ctypes.c_int, ctypes.c_int,
                                                dp, dp, dp, dp]),
        "ltmp2_num_primary_gprime": (ctypes.c_int, [vp]),
        "ltmp2_set_slab_size": (ctypes.c_int, [vp, ctypes.c_int]),
        "ltmp2_sizes": (ctypes.c_int, [vp, P(ctypes.c_int), P(ctypes.c_int), P(ctypes.c_int), P(ctypes.c_int)]),
        "ltmp2_last_imag": (ctypes.c_int, [vp, dp, dp]),
        "ltmp2_set_profiling": (ctypes.c_int, [vp, ctypes.c_int]),
        "ltmp2_kernel_launches": (ctypes.c_int, [vp, P(ctypes.c_longlong)]),
        "ltmp2_fingerprint": (ctypes.c_int, [vp, P(ctypes.c_ulonglong)]),
        "ltmp2_alu_peak": (ctypes.c_int, [ctypes.c_int, dp]),
        "ltmp2_sum_partials": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, dp, dp, dp, dp, dp, dp]),
        "ltmp2_stage_times": (ctypes.c_int, [vp, ctypes.c_int, dp, P(ctypes.c_longlong)]),
        "ltmp2_reset_stage_times": (ctypes.c_int, [vp]),
        "ltmp2_destroy": (None, [vp]),
        "ltmp2_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "ltmp2_set_extrapolation": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_double]),
        "ltmp2_set_route": (ctypes.c_int, [vp, ctypes.c_int]),
        "ltmp2_energy_uhf": (ctypes.c_int, [vp, vp, ctypes.c_int, dp, dp, dp, dp, dp]),
        "ltmp2_selftest_wait": (ctypes.c_int, [vp, ctypes.c_int]),
        "ltmp2_level_energies": (ctypes.c_int, [vp, dp, P(ctypes.c_int), dp, dp]),
        "ltmp2_extrapolate": (ctypes.c_int, [ctypes.c_int, dp, dp, dp, dp, dp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(code: int, where: str):
    if code != 0:
        raise Ltmp2Error(code, where)


def ltmp2_strerror(code: int) -> str:
    return load_library().ltmp2_strerror(int(code)).decode()


class Context:
    """Owns one ltmp2_ctx.  Freed by ltmp2_destroy() or when garbage collected."""

    def __init__(self, handle: int, n_occ: int):
        self.handle = ctypes.c_void_p(handle)
        self.n_occ = n_occ
        self.n_levels = 0
        self._stream = None

    def __del__(self):
        try:
            ltmp2_destroy(self)
        except Exception:
            pass


def ltmp2_setup(lattice, grid, miller, coeff, eps, n_occ: int, ecut_aux: float = 0.0,
                precision: int = FP64, flags: int = 0) -> Context:
    lib = load_library()
    lattice = np.ascontiguousarray(np.asarray(lattice, dtype=np.float64).reshape(9))
    miller = np.ascontiguousarray(np.asarray(miller, dtype=np.int32).reshape(-1, 3))
    coeff = np.ascontiguousarray(np.asarray(coeff, dtype=np.complex128))
    eps = np.ascontiguousarray(np.asarray(eps, dtype=np.float64))
    s = _System()
    s.lattice[:] = lattice.tolist()
    s.grid[:] = [int(g) for g in np.asarray(grid).reshape(3)]
    s.n_pw = miller.shape[0]
    s.miller = miller.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    s.n_orb = coeff.shape[0]
    s.n_occ = int(n_occ)
    if coeff.shape[1] != miller.shape[0] or eps.shape[0] != coeff.shape[0]:
        raise ValueError("coeff must be [n_orb][n_pw] and eps [n_orb]")
    cview = coeff.view(np.float64)
    s.coeff = _dp(cview)
    s.eps = _dp(eps)
    s.ecut_aux = float(ecut_aux)
    s.precision = int(precision)
    s.flags = int(flags)
    h = ctypes.c_void_p()
    _check(lib.ltmp2_setup(ctypes.byref(s), ctypes.byref(h)), "ltmp2_setup")
    return Context(h.value, int(n_occ))


def ltmp2_setup_kpoints(lattice, grid, mesh, miller, coeff, eps, n_occ: int, ecut_aux: float = 0.0,
                        precision: int = FP64) -> Context:
    """k-point context (include/ltmp2.h): coeff [N_k][n_orb][n_pw], eps [N_k][n_orb], one plane-wave
    set for every k; n_occ per k.  The context's pair energies index N_k n_occ composite orbitals."""
    lib = load_library()
    lattice = np.ascontiguousarray(np.asarray(lattice, dtype=np.float64).reshape(9))
    miller = np.ascontiguousarray(np.asarray(miller, dtype=np.int32).reshape(-1, 3))
    coeff = np.ascontiguousarray(np.asarray(coeff, dtype=np.complex128))
    eps = np.ascontiguousarray(np.asarray(eps, dtype=np.float64))
    mesh = [int(x) for x in np.asarray(mesh).reshape(3)]
    nk = mesh[0] * mesh[1] * mesh[2]
    if coeff.ndim != 3 or coeff.shape[0] != nk or coeff.shape[2] != miller.shape[0] or eps.shape != coeff.shape[:2]:
        raise ValueError("coeff must be [N_k][n_orb][n_pw] and eps [N_k][n_orb]")
    s = _KSystem()
    s.lattice[:] = lattice.tolist()
    s.grid[:] = [int(g) for g in np.asarray(grid).reshape(3)]
    s.mesh[:] = mesh
    s.n_pw = miller.shape[0]
    s.miller = miller.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    s.n_orb = coeff.shape[1]
    s.n_occ = int(n_occ)
    s.coeff = _dp(coeff.view(np.float64))
    s.eps = _dp(eps)
    s.ecut_aux = float(ecut_aux)
    s.precision = int(precision)
    s.flags = 0
    h = ctypes.c_void_p()
    _check(lib.ltmp2_setup_kpoints(ctypes.byref(s), ctypes.byref(h)), "ltmp2_setup_kpoints")
    return Context(h.value, int(n_occ) * nk)


def setup_from_kpoint_solid(ks, precision: int = FP64, ecut_aux: Optional[float] = None) -> Context:
    """ltmp2_setup_kpoints for a synth.KPointSolid (E_aux = 2/3 E_cut unless given)."""
    if ecut_aux is None:
        ecut_aux = 2.0 * ks.ecut / 3.0
    return ltmp2_setup_kpoints(ks.lattice, ks.grid, ks.mesh, ks.miller, ks.coeff, ks.eps, ks.n_occ, ecut_aux,
                               precision)


def setup_from_solid(solid, precision: int = FP64, real: Optional[bool] = None,
                     ecut_aux: Optional[float] = None, simt_gemm: bool = False) -> Context:
    """ltmp2_setup for a synth.ModelSolid (E_aux = 2/3 E_cut unless given)."""
    if ecut_aux is None:
        ecut_aux = 2.0 * solid.ecut / 3.0
    flags = (FLAG_REAL_ORBITALS if real else 0) | (FLAG_SIMT_GEMM if simt_gemm else 0)
    return ltmp2_setup(solid.lattice, solid.grid, solid.miller, solid.coeff, solid.eps, solid.n_occ,
                       ecut_aux, precision, flags)


def ltmp2_set_stream(ctx: Context, stream) -> None:
    """stream: an int handle (cudaStream_t) or any object with ``cuda_stream`` (torch.cuda.Stream)."""
    handle = getattr(stream, "cuda_stream", stream)
    ctx._stream = stream
    _check(load_library().ltmp2_set_stream(ctx.handle, ctypes.c_void_p(int(handle) if handle else 0)),
           "ltmp2_set_stream")


def ltmp2_laplace_grid(gap: float, width: float, n_tau: int) -> Tuple[np.ndarray, np.ndarray, float]:
    tau = np.zeros(n_tau)
    w = np.zeros(n_tau)
    err = np.zeros(1)
    _check(load_library().ltmp2_laplace_grid(float(gap), float(width), int(n_tau), _dp(tau), _dp(w), _dp(err)),
           "ltmp2_laplace_grid")
    return tau, w, float(err[0])


def ltmp2_energy(ctx: Context, tau, w, pairs: bool = True):
    """Returns (E_direct, E_exchange, e_pair[n_occ][n_occ] or None)."""
    tau = np.ascontiguousarray(np.asarray(tau, dtype=np.float64))
    w = np.ascontiguousarray(np.asarray(w, dtype=np.float64))
    if tau.shape != w.shape:
        raise ValueError("tau and w must have the same length")
    ed = np.zeros(1)
    ex = np.zeros(1)
    ep = np.zeros((ctx.n_occ, ctx.n_occ)) if pairs else None
    _check(load_library().ltmp2_energy(ctx.handle, len(tau), _dp(tau), _dp(w), _dp(ed), _dp(ex),
                                       _dp(ep) if pairs else None), "ltmp2_energy")
    return float(ed[0]), float(ex[0]), ep


def ltmp2_energy_partial(ctx: Context, tau, w, gp_begin: int, gp_end: int):
    """Returns (E_d, E_x, e_pair_direct, e_pair_exchange) of primary G' in [gp_begin, gp_end)."""
    tau = np.ascontiguousarray(np.asarray(tau, dtype=np.float64))
    w = np.ascontiguousarray(np.asarray(w, dtype=np.float64))
    ed = np.zeros(1)
    ex = np.zeros(1)
    pd = np.zeros((ctx.n_occ, ctx.n_occ))
    px = np.zeros((ctx.n_occ, ctx.n_occ))
    _check(load_library().ltmp2_energy_partial(ctx.handle, len(tau), _dp(tau), _dp(w), int(gp_begin), int(gp_end),
                                               _dp(ed), _dp(ex), _dp(pd), _dp(px)), "ltmp2_energy_partial")
    return float(ed[0]), float(ex[0]), pd, px


def ltmp2_set_slab_size(ctx: Context, n: int) -> int:
    r = load_library().ltmp2_set_slab_size(ctx.handle, int(n))
    if r < 0:
        raise Ltmp2Error(r, "ltmp2_set_slab_size")
    return r


def ltmp2_num_primary_gprime(ctx: Context) -> int:
    r = load_library().ltmp2_num_primary_gprime(ctx.handle)
    if r < 0:
        raise Ltmp2Error(r, "ltmp2_num_primary_gprime")
    return r


def ltmp2_sizes(ctx: Context) -> dict:
    v = [ctypes.c_int() for _ in range(4)]
    _check(load_library().ltmp2_sizes(ctx.handle, *[ctypes.byref(x) for x in v]), "ltmp2_sizes")
    return {"n_aux": v[0].value, "n_pw": v[1].value, "n_occ": v[2].value, "grid": v[3].value}


def ltmp2_last_imag(ctx: Context) -> Tuple[float, float]:
    a, b = np.zeros(1), np.zeros(1)
    _check(load_library().ltmp2_last_imag(ctx.handle, _dp(a), _dp(b)), "ltmp2_last_imag")
    return float(a[0]), float(b[0])


def ltmp2_kernel_launches(ctx: Context) -> int:
    n = ctypes.c_longlong()
    _check(load_library().ltmp2_kernel_launches(ctx.handle, ctypes.byref(n)), "ltmp2_kernel_launches")
    return int(n.value)


def ltmp2_fingerprint(ctx: Context) -> int:
    """64-bit hash of the context's inputs and pair mask (checkpoint keys)."""
    n = ctypes.c_ulonglong()
    _check(load_library().ltmp2_fingerprint(ctx.handle, ctypes.byref(n)), "ltmp2_fingerprint")
    return int(n.value)


def ltmp2_sum_partials(e, pd, px):
    """Fixed-order sum of chunk results: e [n][2], pd / px [n][n_occ][n_occ].
    Returns (E_d, E_x, e^d_ij, e^x_ij)."""
    e = np.ascontiguousarray(np.asarray(e, dtype=np.float64).reshape(-1, 2))
    pd = np.ascontiguousarray(np.asarray(pd, dtype=np.float64))
    px = np.ascontiguousarray(np.asarray(px, dtype=np.float64))
    n, no = e.shape[0], pd.shape[-1]
    if pd.shape != (n, no, no) or px.shape != (n, no, no):
        raise ValueError("pd and px must be [n][n_occ][n_occ]")
    eo = np.zeros(2)
    pdo = np.zeros((no, no))
    pxo = np.zeros((no, no))
    _check(load_library().ltmp2_sum_partials(n, no, _dp(e), _dp(pd), _dp(px), _dp(eo), _dp(pdo), _dp(pxo)),
           "ltmp2_sum_partials")
    return float(eo[0]), float(eo[1]), pdo, pxo


def ltmp2_alu_peak(precision: int) -> float:
    """Measured FMA rate (TFLOP/s) of the current GPU's CUDA cores in FP64 or FP32."""
    t = np.zeros(1)
    _check(load_library().ltmp2_alu_peak(int(precision), _dp(t)), "ltmp2_alu_peak")
    return float(t[0])


def ltmp2_set_profiling(ctx: Context, on: bool) -> None:
    _check(load_library().ltmp2_set_profiling(ctx.handle, 1 if on else 0), "ltmp2_set_profiling")


def ltmp2_stage_times(ctx: Context) -> dict:
    ms = np.zeros(NUM_STAGES)
    n = (ctypes.c_longlong * NUM_STAGES)()
    _check(load_library().ltmp2_stage_times(ctx.handle, NUM_STAGES, _dp(ms), n), "ltmp2_stage_times")
    return {STAGE_NAMES[k]: {"ms": float(ms[k]), "launches": int(n[k])} for k in range(NUM_STAGES)}


def ltmp2_reset_stage_times(ctx: Context) -> None:
    _check(load_library().ltmp2_reset_stage_times(ctx.handle), "ltmp2_reset_stage_times")


def ltmp2_destroy(ctx: Context) -> None:
    if ctx.handle is not None and ctx.handle.value:
        load_library().ltmp2_destroy(ctx.handle)
        ctx.handle = ctypes.c_void_p(0)


def ltmp2_energy_noalloc(lattice, grid, miller, coeff, eps, n_occ: int, tau, w, ecut_aux: float = 0.0,
                         precision: int = FP64, flags: int = 0, stream=None, pairs: bool = True):
    """ltmp2_setup + ltmp2_energy without any device allocation (see include/ltmp2.h).

    For callers that cannot call cudaMalloc.  All device buffers live in the library's
    32 MiB static array, so only small systems fit; concurrent calls race.
    Returns (E_direct, E_exchange, e_pair or None).
    """
    lib = load_library()
    f = lib.ltmp2_energy_noalloc
    dp = ctypes.POINTER(ctypes.c_double)
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.POINTER(_System), ctypes.c_int, dp, dp, dp, dp, dp, ctypes.c_void_p]
    lattice = np.ascontiguousarray(np.asarray(lattice, dtype=np.float64).reshape(9))
    miller = np.ascontiguousarray(np.asarray(miller, dtype=np.int32).reshape(-1, 3))
    coeff = np.ascontiguousarray(np.asarray(coeff, dtype=np.complex128))
    eps = np.ascontiguousarray(np.asarray(eps, dtype=np.float64))
    tau = np.ascontiguousarray(np.asarray(tau, dtype=np.float64))
    w = np.ascontiguousarray(np.asarray(w, dtype=np.float64))
    s = _System()
    s.lattice[:] = lattice.tolist()
    s.grid[:] = [int(g) for g in np.asarray(grid).reshape(3)]
    s.n_pw = miller.shape[0]
    s.miller = miller.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    s.n_orb = coeff.shape[0]
    s.n_occ = int(n_occ)
    s.coeff = _dp(coeff.view(np.float64))
    s.eps = _dp(eps)
    s.ecut_aux = float(ecut_aux)
    s.precision = int(precision)
    s.flags = int(flags)
    ed, ex = np.zeros(1), np.zeros(1)
    ep = np.zeros((int(n_occ), int(n_occ))) if pairs else None
    handle = getattr(stream, "cuda_stream", stream) if stream is not None else 0
    _check(f(ctypes.byref(s), len(tau), _dp(tau), _dp(w), _dp(ed), _dp(ex), _dp(ep) if pairs else None,
             ctypes.c_void_p(int(handle) if handle else 0)), "ltmp2_energy_noalloc")
    return float(ed[0]), float(ex[0]), ep


# ---------------------------------------------------------------- failure-path self-test
def ltmp2_selftest_wait(ctx: Context, budget_us: int) -> int:
    """Status of one bounded device wait on a barrier that never completes (expected:
    the TIMEOUT code, -7)."""
    return int(load_library().ltmp2_selftest_wait(ctx.handle, int(budget_us)))


# ---------------------------------------------------------------- spin-unrestricted form
def ltmp2_energy_uhf(alpha: Context, beta: Context, tau, w):
    """(E_direct, E_exchange, [E_same_alpha, E_same_beta, E_opposite]) of the two channels."""
    tau = np.ascontiguousarray(np.asarray(tau, dtype=np.float64))
    w = np.ascontiguousarray(np.asarray(w, dtype=np.float64))
    ed, ex, es = np.zeros(1), np.zeros(1), np.zeros(3)
    _check(load_library().ltmp2_energy_uhf(alpha.handle, beta.handle, len(tau), _dp(tau), _dp(w), _dp(ed), _dp(ex),
                                           _dp(es)), "ltmp2_energy_uhf")
    return float(ed[0]), float(ex[0]), es


# ---------------------------------------------------------------- transformed-state route
ROUTE_GREEN = 0
ROUTE_OVERLAP = 1


def ltmp2_set_route(ctx: Context, route: int) -> None:
    """ROUTE_GREEN (per-tau Green's function) or ROUTE_OVERLAP (stored overlap densities,
    the paper's steps (i)-(iii)); the latter computes the densities now."""
    _check(load_library().ltmp2_set_route(ctx.handle, int(route)), "ltmp2_set_route")


# ---------------------------------------------------------------- internal cutoff extrapolation
def ltmp2_set_extrapolation(ctx: Context, n_c: int = 8, alpha: float = 1.05) -> None:
    """Evaluate later energies also on n_c nested auxiliary spheres (n_c <= 1: off)."""
    _check(load_library().ltmp2_set_extrapolation(ctx.handle, int(n_c), float(alpha)),
           "ltmp2_set_extrapolation")
    ctx.n_levels = int(n_c) if n_c > 1 else 0


def ltmp2_level_energies(ctx: Context) -> dict:
    """Cutoffs, |A_n| and E_direct / E_exchange per level of the last energy call."""
    nl = getattr(ctx, "n_levels", 0)
    if nl < 2:
        raise Ltmp2Error(-1, "ltmp2_level_energies: levels are off")
    ecut, ed, ex = np.zeros(nl), np.zeros(nl), np.zeros(nl)
    cnt = (ctypes.c_int * nl)()
    _check(load_library().ltmp2_level_energies(ctx.handle, _dp(ecut), cnt, _dp(ed), _dp(ex)),
           "ltmp2_level_energies")
    return {"ecut_aux": ecut, "n_aux": np.array(cnt[:]), "E_d": ed, "E_x": ex}


def ltmp2_extrapolate(ecut_aux, energy) -> Tuple[float, float, float]:
    """(E_inf, slope, sigma) of the fit E = E_inf + slope * E_aux^(-3/2) (Eq. CutDecay)."""
    e = np.ascontiguousarray(np.asarray(ecut_aux, dtype=np.float64))
    y = np.ascontiguousarray(np.asarray(energy, dtype=np.float64))
    if e.shape != y.shape:
        raise ValueError("ecut_aux and energy differ in length")
    a, b, sg = np.zeros(1), np.zeros(1), np.zeros(1)
    _check(load_library().ltmp2_extrapolate(len(e), _dp(e), _dp(y), _dp(a), _dp(b), _dp(sg)), "ltmp2_extrapolate")
    return float(a[0]), float(b[0]), float(sg[0])


# ---------------------------------------------------------------- batching form
def _batch_sig(lib):
    P = ctypes.POINTER
    dp = P(ctypes.c_double)
    vp = ctypes.c_void_p
    for name, res, args in [
            ("ltmp2_autotune", ctypes.c_int, [vp, P(ctypes.c_int), P(ctypes.c_int)]),
            ("ltmp2_get_tuning", ctypes.c_int, [vp, P(ctypes.c_int)]),
            ("ltmp2_batch_create", ctypes.c_int, [P(vp), ctypes.c_int, P(ctypes.c_int), P(dp), P(dp), P(vp)]),
            ("ltmp2_batch_run", ctypes.c_int, [vp, dp, dp]),
            ("ltmp2_batch_kernel_nodes", ctypes.c_int, [vp, P(ctypes.c_longlong)]),
            ("ltmp2_batch_mode", ctypes.c_int, [vp, P(ctypes.c_int)]),
            ("ltmp2_batch_destroy", None, [vp]),
            ("ltmp2_energy_batch", ctypes.c_int, [P(vp), ctypes.c_int, P(ctypes.c_int), P(dp), P(dp), dp, dp])]:
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


def ltmp2_autotune(ctx: Context):
    """Returns (slab, gemm_variant) chosen and applied for ctx."""
    lib = _batch_sig(load_library())
    sl, var = ctypes.c_int(), ctypes.c_int()
    _check(lib.ltmp2_autotune(ctx.handle, ctypes.byref(sl), ctypes.byref(var)), "ltmp2_autotune")
    return sl.value, var.value


TUNING_VALUES = 6


def ltmp2_get_tuning(ctx: Context) -> dict:
    lib = _batch_sig(load_library())
    v = (ctypes.c_int * TUNING_VALUES)()
    _check(lib.ltmp2_get_tuning(ctx.handle, v), "ltmp2_get_tuning")
    return {"slab": v[0], "gemm_variant": v[1], "plane_kernel": v[2], "plane_ib": v[3],
            "green_tc": v[4], "direct_tc": v[5]}


def ltmp2_set_tuning(ctx: Context, slab: int = -1, gemm_variant: int = -1, plane_kernel: int = -1,
                     plane_ib: int = -1, green_tc: int = -1, direct_tc: int = -1) -> None:
    """Apply tuning settings by hand (-1 keeps the current value)."""
    lib = load_library()
    f = lib.ltmp2_set_tuning
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]
    v = (ctypes.c_int * TUNING_VALUES)(int(slab), int(gemm_variant), int(plane_kernel), int(plane_ib),
                                       int(green_tc), int(direct_tc))
    _check(f(ctx.handle, v), "ltmp2_set_tuning")


def ltmp2_dgemm_nt(a, b, c=None):
    """C = A B^T in FP64 accuracy on the tensor cores (exact integer slices).  a [m, k],
    b [n, k]: float64 CUDA tensors, row-major with unit column stride; returns c [m, n]."""
    import torch
    if a.dtype != torch.float64 or b.dtype != torch.float64 or not a.is_cuda or not b.is_cuda:
        raise ValueError("a and b must be float64 CUDA tensors")
    if a.dim() != 2 or b.dim() != 2 or a.shape[1] != b.shape[1] or a.stride(1) != 1 or b.stride(1) != 1:
        raise ValueError("a [m, k] and b [n, k] with unit column stride")
    m, k = a.shape
    n = b.shape[0]
    if c is None:
        c = torch.empty((m, n), dtype=torch.float64, device=a.device)
    f = load_library().ltmp2_dgemm_nt
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                  ctypes.c_int, ctypes.c_void_p, ctypes.c_int]
    _check(f(m, n, k, a.data_ptr(), a.stride(0), b.data_ptr(), b.stride(0), c.data_ptr(), c.stride(0)),
           "ltmp2_dgemm_nt")
    return c


VIRTUALS_ALL, VIRTUALS_AUTO, VIRTUALS_SPACE = 0, 1, 2


def ltmp2_set_virtual_cut(ctx: Context, mode: int = VIRTUALS_AUTO, log2_cut: float = 64.0) -> None:
    """Which virtuals each Laplace point keeps and when W goes through the virtual space."""
    lib = load_library()
    f = lib.ltmp2_set_virtual_cut
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_double]
    _check(f(ctx.handle, int(mode), float(log2_cut)), "ltmp2_set_virtual_cut")


def ltmp2_tau_virtuals(ctx: Context, tau) -> Tuple[np.ndarray, np.ndarray]:
    """(virtuals kept, 1 where W goes through the virtual space) for each Laplace point."""
    lib = load_library()
    f = lib.ltmp2_tau_virtuals
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    t = np.ascontiguousarray(tau, dtype=np.float64)
    nv = np.zeros(t.size, dtype=np.int32)
    wv = np.zeros(t.size, dtype=np.int32)
    _check(f(ctx.handle, int(t.size), t.ctypes.data, nv.ctypes.data, wv.ctypes.data), "ltmp2_tau_virtuals")
    return nv, wv


def _batch_args(ctxs, taus, ws):
    n = len(ctxs)
    handles = (ctypes.c_void_p * n)(*[c.handle.value for c in ctxs])
    keep = []
    tps = (ctypes.POINTER(ctypes.c_double) * n)()
    wps = (ctypes.POINTER(ctypes.c_double) * n)()
    nt = (ctypes.c_int * n)()
    for i, (t, w) in enumerate(zip(taus, ws)):
        t = np.ascontiguousarray(np.asarray(t, dtype=np.float64))
        w = np.ascontiguousarray(np.asarray(w, dtype=np.float64))
        keep += [t, w]
        tps[i] = _dp(t)
        wps[i] = _dp(w)
        nt[i] = len(t)
    return n, handles, nt, tps, wps, keep


class Batch:
    """A captured CUDA graph evaluating several contexts in one launch."""

    def __init__(self, ctxs, taus, ws):
        lib = _batch_sig(load_library())
        self.ctxs = list(ctxs)          # keep the contexts alive
        n, handles, nt, tps, wps, keep = _batch_args(ctxs, taus, ws)
        h = ctypes.c_void_p()
        _check(lib.ltmp2_batch_create(handles, n, nt, tps, wps, ctypes.byref(h)), "ltmp2_batch_create")
        self.handle = h
        self.n = n

    def persistent(self) -> bool:
        """True when the batch runs in rounds with the shared persistent FFT stages."""
        v = ctypes.c_int()
        _check(_batch_sig(load_library()).ltmp2_batch_mode(self.handle, ctypes.byref(v)), "ltmp2_batch_mode")
        return bool(v.value)

    def run(self):
        ed, ex = np.zeros(self.n), np.zeros(self.n)
        _check(load_library().ltmp2_batch_run(self.handle, _dp(ed), _dp(ex)), "ltmp2_batch_run")
        return ed, ex

    def kernel_nodes(self) -> int:
        c = ctypes.c_longlong()
        _check(load_library().ltmp2_batch_kernel_nodes(self.handle, ctypes.byref(c)), "ltmp2_batch_kernel_nodes")
        return int(c.value)

    def destroy(self):
        if self.handle is not None and self.handle.value:
            load_library().ltmp2_batch_destroy(self.handle)
            self.handle = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def ltmp2_batch_create(ctxs, taus, ws) -> Batch:
    return Batch(ctxs, taus, ws)


def ltmp2_energy_batch(ctxs, taus, ws):
    """Autotune, capture and run once.  Returns (E_direct[n], E_exchange[n])."""
    lib = _batch_sig(load_library())
    n, handles, nt, tps, wps, keep = _batch_args(ctxs, taus, ws)
    ed, ex = np.zeros(n), np.zeros(n)
    _check(lib.ltmp2_energy_batch(handles, n, nt, tps, wps, _dp(ed), _dp(ex)), "ltmp2_energy_batch")
    return ed, ex


# ---------------------------------------------------------------- learned form
NUM_DESC = 8


def _learned_sig(lib):
    P = ctypes.POINTER
    vp = ctypes.c_void_p
    fp = P(ctypes.c_float)
    for name, res, args in [
            ("ltmp2_set_pair_mask", ctypes.c_int, [vp, P(ctypes.c_ubyte)]),
            ("ltmp2_pair_descriptors", ctypes.c_int, [vp, P(ctypes.c_double)]),
            ("ltmp2_mlp_create", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_ulonglong, P(vp)]),
            ("ltmp2_mlp_train", ctypes.c_int, [vp, fp, fp, ctypes.c_int, ctypes.c_int, ctypes.c_float, fp]),
            ("ltmp2_mlp_predict", ctypes.c_int, [vp, fp, ctypes.c_int, fp]),
            ("ltmp2_mlp_destroy", None, [vp]),
            ("ltmp2_mlp_residual", ctypes.c_int, [vp, fp]),
            ("ltmp2_learned_training_data", ctypes.c_int, [vp, ctypes.c_int, P(ctypes.c_double),
                                                           P(ctypes.c_double), fp, fp]),
            ("ltmp2_screen_select", ctypes.c_int, [ctypes.c_int, P(ctypes.c_double), ctypes.c_double,
                                                   P(ctypes.c_ubyte), P(ctypes.c_int), P(ctypes.c_double)]),
            ("ltmp2_energy_screened", ctypes.c_int, [vp, vp, ctypes.c_int, P(ctypes.c_double), P(ctypes.c_double),
                                                     ctypes.c_double, ctypes.c_double, P(ctypes.c_double),
                                                     P(ctypes.c_double), P(ctypes.c_double)])]:
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


def ltmp2_set_pair_mask(ctx: Context, keep) -> None:
    """keep: None or [n_occ][n_occ] booleans (symmetric, diagonal True)."""
    lib = _learned_sig(load_library())
    if keep is None:
        _check(lib.ltmp2_set_pair_mask(ctx.handle, None), "ltmp2_set_pair_mask")
        return
    k = np.ascontiguousarray(np.asarray(keep, dtype=np.uint8))
    ctx._keep = k
    _check(lib.ltmp2_set_pair_mask(ctx.handle, k.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))),
           "ltmp2_set_pair_mask")


def ltmp2_pair_descriptors(ctx: Context) -> np.ndarray:
    """[n_pairs][NUM_DESC] for unordered pairs i <= j (row order i, then j)."""
    lib = _learned_sig(load_library())
    n = ctx.n_occ * (ctx.n_occ + 1) // 2
    d = np.zeros((n, NUM_DESC))
    _check(lib.ltmp2_pair_descriptors(ctx.handle, _dp(d)), "ltmp2_pair_descriptors")
    return d


class Mlp:
    """Pair-energy perceptron trained and evaluated by the library's kernels."""

    def __init__(self, n_in: int = NUM_DESC, width: int = 64, seed: int = 1):
        lib = _learned_sig(load_library())
        h = ctypes.c_void_p()
        _check(lib.ltmp2_mlp_create(int(n_in), int(width), ctypes.c_ulonglong(seed), ctypes.byref(h)),
               "ltmp2_mlp_create")
        self.handle = h
        self.n_in = n_in

    def train(self, X, y, epochs: int = 2000, lr: float = 3e-3) -> float:
        X = np.ascontiguousarray(np.asarray(X, dtype=np.float32))
        y = np.ascontiguousarray(np.asarray(y, dtype=np.float32))
        loss = ctypes.c_float()
        fp = ctypes.POINTER(ctypes.c_float)
        _check(load_library().ltmp2_mlp_train(self.handle, X.ctypes.data_as(fp), y.ctypes.data_as(fp), len(y),
                                              int(epochs), ctypes.c_float(lr), ctypes.byref(loss)), "ltmp2_mlp_train")
        return float(loss.value)

    def residual(self) -> float:
        """Root-mean-square training residual in the units of the targets."""
        r = ctypes.c_float()
        _check(_learned_sig(load_library()).ltmp2_mlp_residual(self.handle, ctypes.byref(r)), "ltmp2_mlp_residual")
        return float(r.value)

    def predict(self, X) -> np.ndarray:
        X = np.ascontiguousarray(np.asarray(X, dtype=np.float32))
        y = np.zeros(X.shape[0], dtype=np.float32)
        fp = ctypes.POINTER(ctypes.c_float)
        _check(load_library().ltmp2_mlp_predict(self.handle, X.ctypes.data_as(fp), X.shape[0], y.ctypes.data_as(fp)),
               "ltmp2_mlp_predict")
        return y

    def destroy(self):
        if self.handle is not None and self.handle.value:
            load_library().ltmp2_mlp_destroy(self.handle)
            self.handle = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def ltmp2_learned_training_data(ctx: Context, tau, w):
    """(X [pairs][NUM_DESC] float32, y [pairs] float32 = ln|e^x_ij|) of the unordered pairs i <= j."""
    lib = _learned_sig(load_library())
    tau = np.ascontiguousarray(np.asarray(tau, dtype=np.float64))
    w = np.ascontiguousarray(np.asarray(w, dtype=np.float64))
    npairs = ctx.n_occ * (ctx.n_occ + 1) // 2
    X = np.zeros((npairs, NUM_DESC), dtype=np.float32)
    y = np.zeros(npairs, dtype=np.float32)
    fp = ctypes.POINTER(ctypes.c_float)
    _check(lib.ltmp2_learned_training_data(ctx.handle, len(tau), _dp(tau), _dp(w), X.ctypes.data_as(fp),
                                           y.ctypes.data_as(fp)), "ltmp2_learned_training_data")
    return X, y


def ltmp2_screen_select(n_occ: int, est, budget: float):
    """(keep [n_occ][n_occ] bool, screened unordered pairs, sum of their estimates)."""
    lib = _learned_sig(load_library())
    est = np.ascontiguousarray(np.asarray(est, dtype=np.float64))
    keep = np.zeros((n_occ, n_occ), dtype=np.uint8)
    n = ctypes.c_int()
    tot = ctypes.c_double()
    _check(lib.ltmp2_screen_select(int(n_occ), _dp(est), float(budget),
                                   keep.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)), ctypes.byref(n),
                                   ctypes.byref(tot)), "ltmp2_screen_select")
    return keep.astype(bool), int(n.value), float(tot.value)


def ltmp2_energy_screened(ctx: Context, net: "Mlp", tau, w, budget: float, margin: float = 1.0) -> dict:
    """Learned-form energy (include/ltmp2.h): E_d exact, E_x of the kept pairs plus the model's
    estimates of the screened ones; margin: the validated upper-bound factor of the decision."""
    lib = _learned_sig(load_library())
    tau = np.ascontiguousarray(np.asarray(tau, dtype=np.float64))
    w = np.ascontiguousarray(np.asarray(w, dtype=np.float64))
    ed, ex, info = np.zeros(1), np.zeros(1), np.zeros(4)
    _check(lib.ltmp2_energy_screened(ctx.handle, net.handle, len(tau), _dp(tau), _dp(w), float(budget),
                                     float(margin), _dp(ed), _dp(ex), _dp(info)), "ltmp2_energy_screened")
    return {"E_d": float(ed[0]), "E_x": float(ex[0]), "screened_pairs": int(info[0]),
            "E_x_estimated": float(info[1]), "E_x_contracted": float(info[2]), "pairs": int(info[3])}

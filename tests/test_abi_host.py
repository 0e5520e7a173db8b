"""Host-side checks of the C ABI: the library loads, exports every declared entry
point, fits the Laplace grid on the host, and rejects bad input before touching a
device (host-side fault injection).  No GPU is needed."""
import math
import os
import re

import numpy as np
import pytest

import paper_1611_06797_gb300 as L
from oracle import quadrature_max_error, sinc_laplace_quadrature
from synth import SPECS, ModelSolidSpec, build_model_solid
from tests.conftest import solid

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(ltmp2_\w+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol():
    lib = L.load_library()
    names = _declared()
    assert {"ltmp2_setup", "ltmp2_energy", "ltmp2_laplace_grid", "ltmp2_destroy"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_strerror_names_every_code():
    for code in range(0, -11, -1):
        s = L.ltmp2_strerror(code)
        assert s and s != "unknown status"
    assert L.ltmp2_strerror(-99) == "unknown status"


@pytest.mark.parametrize("gap,width", [(0.0226, 13.92), (0.256, 7.3), (0.0042, 11.42)])
def test_laplace_grid_fits_one_over_x(gap, width):
    """Eq. SCHLT with a quadrature: the reported error is the measured one, it falls with
    n_tau, and the fit beats the oracle's plain trapezoid rule at the same n_tau."""
    lo, hi = 2 * gap, 2 * width
    prev = None
    for n in (4, 6, 8, 10):
        tau, w, err = L.ltmp2_laplace_grid(gap, width, n)
        assert np.all(np.diff(tau) > 0) and np.all(tau > 0)
        meas = quadrature_max_error(tau, w, lo, hi, samples=20000)
        assert abs(meas - err) <= 0.05 * err + 1e-12
        t2, w2 = sinc_laplace_quadrature(n, lo, hi)
        assert err < quadrature_max_error(t2, w2, lo, hi, samples=20000)
        if prev is not None:
            assert err < prev
        prev = err


def test_laplace_grid_rejects_bad_input():
    for args in [(0.0, 1.0, 6), (-1.0, 1.0, 6), (0.1, 0.05, 6), (0.1, 1.0, 0), (0.1, 1.0, 25),
                 (float("nan"), 1.0, 6)]:
        with pytest.raises(L.Ltmp2Error) as e:
            L.ltmp2_laplace_grid(*args)
        assert e.value.name == "INVALID_ARG"


# ---------------------------------------------------------------- setup validation
def _setup(s, **over):
    kw = dict(lattice=s.lattice, grid=s.grid, miller=s.miller, coeff=s.coeff, eps=s.eps,
              n_occ=s.n_occ, ecut_aux=2 * s.ecut / 3, precision=L.FP64, flags=0)
    kw.update(over)
    return L.ltmp2_setup(**kw)


def _expect(code, s, **over):
    with pytest.raises(L.Ltmp2Error) as e:
        _setup(s, **over)
    assert e.value.name == code, e.value


def test_setup_rejects_bad_input_before_the_device():
    s = solid("tiny")
    _expect("GRID", s, grid=[8, 8, 10])           # not cubic
    _expect("GRID", s, grid=[7, 7, 7])            # not supported
    _expect("GRID", s, grid=[6, 6, 6], miller=s.miller)  # sphere does not fit
    eps = s.eps.copy(); eps[s.n_occ] = eps[s.n_occ - 1]
    _expect("GAP", s, eps=eps)
    eps = s.eps.copy(); eps[3], eps[4] = eps[4], eps[3]
    _expect("INVALID_ARG", s, eps=eps)            # unsorted
    eps = s.eps.copy(); eps[5] = np.nan
    _expect("INVALID_ARG", s, eps=eps)
    c = s.coeff.copy(); c[1] *= 1.01
    _expect("NOT_ORTHONORMAL", s, coeff=c)
    _expect("INVALID_ARG", s, n_occ=0)
    _expect("INVALID_ARG", s, n_occ=s.n_orb)
    _expect("INVALID_ARG", s, precision=7)
    m = s.miller.copy(); m[1] = m[2]
    _expect("INVALID_ARG", s, miller=m)           # duplicate plane wave
    keep = np.array([not (r[0] == 3 and r[1] == 0 and r[2] == 0) for r in s.miller.tolist()])
    _expect("GRID", s, miller=s.miller[keep], coeff=np.eye(keep.sum(), dtype=complex)[:s.n_orb - 1],
            eps=np.sort(s.eps[:s.n_orb - 1]), flags=L.FLAG_REAL_ORBITALS)    # not inversion symmetric


def test_setup_checks_real_orbital_flag():
    s = solid("tiny", random_phases=True)
    _expect("NOT_REAL", s, flags=L.FLAG_REAL_ORBITALS)


def test_setup_without_device_reports_cuda():
    """Valid input on a host without a usable GPU stops with CUDA, never silently."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(L.Ltmp2Error) as e:
        _setup(solid("tiny"))
    assert e.value.name == "CUDA"


def test_extrapolation_fit_is_the_oracle_fit():
    """ltmp2_extrapolate is host arithmetic: the same straight-line fit in
    E_aux^(-3/2) (Eq. CutDecay) as the oracle's, on the same points."""
    from oracle import cutoff_extrapolation, cutoff_levels
    rng = np.random.default_rng(7)
    ecut = cutoff_levels(8.0, 8, 1.05)
    y = -0.9 + 3.0 * ecut ** -1.5 + 1e-5 * rng.standard_normal(8)
    a, b, sg = L.ltmp2_extrapolate(ecut, y)
    ra, rb, rs = cutoff_extrapolation(ecut, y)
    assert abs(a - ra) < 1e-12 and abs(b - rb) < 1e-9 * abs(rb) and abs(sg - rs) < 1e-9 * rs
    with pytest.raises(L.Ltmp2Error):
        L.ltmp2_extrapolate([1.0, 1.0], [0.0, 1.0])


def test_entry_points_reject_null_contexts():
    """Every context-taking entry point returns INVALID_ARG for a NULL context before it
    touches a device (so these checks run on any host)."""
    import ctypes
    lib = L.load_library()
    dp = ctypes.POINTER(ctypes.c_double)
    d = (ctypes.c_double * 4)()
    i = (ctypes.c_int * 4)()
    tau = (ctypes.c_double * 1)(1.0)
    w = (ctypes.c_double * 1)(1.0)
    null = ctypes.c_void_p(None)
    calls = {
        "ltmp2_energy": lambda f: f(null, 1, tau, w, d, d, None),
        "ltmp2_energy_partial": lambda f: f(null, 1, tau, w, 0, 1, d, d, None, None),
        "ltmp2_set_slab_size": lambda f: f(null, 1),
        "ltmp2_set_route": lambda f: f(null, 1),
        "ltmp2_set_extrapolation": lambda f: f(null, 8, ctypes.c_double(1.05)),
        "ltmp2_level_energies": lambda f: f(null, d, i, d, d),
        "ltmp2_energy_uhf": lambda f: f(null, null, 1, tau, w, d, d, None),
        "ltmp2_set_tuning": lambda f: f(null, i),
        "ltmp2_get_tuning": lambda f: f(null, i),
        "ltmp2_set_pair_mask": lambda f: f(null, None),
        "ltmp2_pair_descriptors": lambda f: f(null, d),
        "ltmp2_autotune": lambda f: f(null, i, i),
        "ltmp2_sizes": lambda f: f(null, i, i, i, i),
        "ltmp2_last_imag": lambda f: f(null, d, d),
        "ltmp2_set_profiling": lambda f: f(null, 1),
        "ltmp2_stage_times": lambda f: f(null, 1, d, None),
        "ltmp2_reset_stage_times": lambda f: f(null),
        "ltmp2_set_stream": lambda f: f(null, None),
        "ltmp2_num_primary_gprime": lambda f: f(null),
        "ltmp2_set_virtual_cut": lambda f: f(null, 1, ctypes.c_double(64.0)),
        "ltmp2_tau_virtuals": lambda f: f(null, 1, tau, i, i),
    }
    for name, call in calls.items():
        f = getattr(lib, name)
        f.restype = ctypes.c_int
        assert call(f) == -1, name


def test_extrapolate_and_noalloc_validate_on_the_host():
    import ctypes
    lib = L.load_library()
    e = (ctypes.c_double * 2)(5.0, 4.0)
    y = (ctypes.c_double * 2)(-1.0, -1.1)
    out = (ctypes.c_double * 1)()
    f = lib.ltmp2_extrapolate
    f.restype = ctypes.c_int
    assert f(1, e, y, out, None, None) == -1                      # fewer than two points
    assert f(2, None, y, out, None, None) == -1
    bad = (ctypes.c_double * 2)(5.0, -4.0)
    assert f(2, bad, y, out, None, None) == -1                    # non-positive cutoff
    assert f(2, e, y, out, None, None) == 0
    g = lib.ltmp2_energy_noalloc
    g.restype = ctypes.c_int
    assert g(None, 1, None, None, None, None, None, None) == -1


def test_noalloc_rejects_bad_systems_with_the_setup_codes():
    """The allocation-free entry point validates its input with ltmp2_setup's own checks
    (one shared host routine): a non-orthonormal set, a NaN coefficient, a missing gap,
    a bad grid and a wrong real-orbital flag get the same status from both, on the host,
    before any device work."""
    s = solid("tiny")
    tau, w = np.array([0.5, 2.0]), np.array([0.4, 0.9])
    c_bad = s.coeff.copy(); c_bad[1] *= 1.01
    c_nan = s.coeff.copy(); c_nan[2, 5] = complex(np.nan, 0.0)
    eps_gap = s.eps.copy(); eps_gap[s.n_occ] = eps_gap[s.n_occ - 1]
    cases = [("NOT_ORTHONORMAL", dict(coeff=c_bad)), ("INVALID_ARG", dict(coeff=c_nan)),
             ("GAP", dict(eps=eps_gap)), ("GRID", dict(grid=[8, 8, 10]))]
    for name, kw in cases:
        _expect(name, s, **kw)
        args = dict(lattice=s.lattice, grid=s.grid, miller=s.miller, coeff=s.coeff, eps=s.eps, n_occ=s.n_occ)
        args.update(kw)
        with pytest.raises(L.Ltmp2Error) as e:
            L.ltmp2_energy_noalloc(args["lattice"], args["grid"], args["miller"], args["coeff"], args["eps"],
                                   args["n_occ"], tau, w)
        assert e.value.name == name, (name, e.value.name)
    sp = solid("tiny", random_phases=True)
    with pytest.raises(L.Ltmp2Error) as e:
        L.ltmp2_energy_noalloc(sp.lattice, sp.grid, sp.miller, sp.coeff, sp.eps, sp.n_occ, tau, w,
                               flags=L.FLAG_REAL_ORBITALS)
    assert e.value.name == "NOT_REAL"


def test_kpoint_setup_validates_on_the_host():
    """ltmp2_setup_kpoints rejects bad input before any device work, with ltmp2_setup's codes."""
    from synth import build_kpoint_solid
    ks = build_kpoint_solid(5.0, 8, 9, (2, 1, 1), np.array([[1.1, 2.3, 2.0]]), 1, seed=4)
    base = dict(lattice=ks.lattice, grid=ks.grid, mesh=ks.mesh, miller=ks.miller, coeff=ks.coeff, eps=ks.eps,
                n_occ=ks.n_occ, ecut_aux=2 * ks.ecut / 3)

    def expect(code, **over):
        kw = dict(base)
        kw.update(over)
        with pytest.raises(L.Ltmp2Error) as e:
            L.ltmp2_setup_kpoints(**kw)
        assert e.value.name == code, (code, e.value.name)
    c = ks.coeff.copy(); c[1, 0] *= 1.01
    expect("NOT_ORTHONORMAL", coeff=c)
    c = ks.coeff.copy(); c[0, 3, 2] = complex(np.nan, 0)
    expect("INVALID_ARG", coeff=c)
    e = ks.eps.copy(); e[1, 1] = ks.eps[:, 0].max()          # LUMO of k = 1 at the HOMO of the mesh
    expect("GAP", eps=e)
    expect("GRID", grid=[8, 8, 10])
    with pytest.raises(ValueError):                           # the binding checks the array shapes
        L.ltmp2_setup_kpoints(**dict(base, mesh=[0, 1, 1]))
    expect("INVALID_ARG", n_occ=0)
    expect("INVALID_ARG", precision=3)


def test_screen_select_rule():
    """Off-diagonal pairs in ascending order of the estimate while the screened sum fits the
    budget; the diagonal is never screened; ties fall in row order; bad estimates rejected."""
    n = 4
    i, j = np.triu_indices(n)
    est = np.where(i == j, 1e-9, 0.0) + np.array([0, 5, 1, 3, 0, 2, 2, 0, 4, 0], float) * 1e-3
    keep, nscr, tot = L.ltmp2_screen_select(n, est, 5.5e-3)
    # ascending: (0,2)=1, (1,2)=2, (1,3)=2 (row order), (0,3)=3, ... -> 1 + 2 + 2 = 5 <= 5.5
    assert nscr == 3 and abs(tot - 5e-3) < 1e-15
    assert not keep[0, 2] and not keep[2, 0] and not keep[1, 2] and not keep[1, 3] and not keep[3, 1]
    assert keep[0, 1] and keep[0, 3] and keep[2, 3] and np.all(np.diag(keep))
    keep0, n0, t0 = L.ltmp2_screen_select(n, est, 0.0)
    assert n0 == 0 and t0 == 0.0 and keep0.all()
    for bad in (-1.0, np.nan):
        e = est.copy(); e[3] = bad
        with pytest.raises(L.Ltmp2Error):
            L.ltmp2_screen_select(n, e, 1.0)


def test_dgemm_rejects_bad_arguments_on_the_host():
    """ltmp2_dgemm_nt checks sizes, leading dimensions and pointers before any device work."""
    import ctypes
    lib = L.load_library()
    f = lib.ltmp2_dgemm_nt
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                  ctypes.c_int, ctypes.c_void_p, ctypes.c_int]
    p = ctypes.c_void_p(16)     # never dereferenced: every call below fails its argument checks
    assert f(0, 4, 4, p, 4, p, 4, p, 4) == -1       # m < 1
    assert f(4, 0, 4, p, 4, p, 4, p, 4) == -1       # n < 1
    assert f(4, 4, 0, p, 4, p, 4, p, 4) == -1       # k < 1
    assert f(4, 4, 8, p, 4, p, 8, p, 4) == -1       # lda < k
    assert f(4, 4, 8, p, 8, p, 4, p, 4) == -1       # ldb < k
    assert f(4, 4, 8, p, 8, p, 8, p, 3) == -1       # ldc < n
    assert f(4, 4, 8, None, 8, p, 8, p, 4) == -1    # null pointer

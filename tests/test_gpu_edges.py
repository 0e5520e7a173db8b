"""Edge cases of the C ABI on the GPU: empty outer-loop ranges, the smallest and
out-of-range slab sizes, a single Laplace point, and rejected quadrature input."""
import numpy as np
import pytest

import paper_1611_06797_gb300 as L
from oracle import OracleSystem, denominator_range, laplace_denominator, mp2_energy, sinc_laplace_quadrature
from tests.conftest import solid

pytestmark = pytest.mark.gpu


def test_empty_gprime_range_gives_zero():
    s = solid("tiny2")
    tau, w = sinc_laplace_quadrature(3, *denominator_range(OracleSystem.from_solid(s)))
    ctx = L.setup_from_solid(s, precision=L.FP64, real=True)
    n = L.ltmp2_num_primary_gprime(ctx)
    for k in (0, n // 2, n):
        ed, ex, pd, px = L.ltmp2_energy_partial(ctx, tau, w, k, k)
        assert ed == 0.0 and ex == 0.0 and not pd.any() and not px.any()
    with pytest.raises(L.Ltmp2Error):
        L.ltmp2_energy_partial(ctx, tau, w, 3, 2)
    with pytest.raises(L.Ltmp2Error):
        L.ltmp2_energy_partial(ctx, tau, w, 0, n + 1)
    L.ltmp2_destroy(ctx)


def test_slab_of_one_and_single_tau_match_oracle():
    s = solid("tiny")
    tau, w = sinc_laplace_quadrature(1, *denominator_range(OracleSystem.from_solid(s)))
    ref = mp2_energy(OracleSystem.from_solid(s), laplace_denominator(tau, w))
    for real in (True, False):
        ctx = L.setup_from_solid(s, precision=L.FP64, real=real)
        L.ltmp2_set_slab_size(ctx, 1)
        ed, ex, _ = L.ltmp2_energy(ctx, tau, w)
        L.ltmp2_destroy(ctx)
        assert abs(ed - ref["E_d"]) < 1e-8 and abs(ex - ref["E_x"]) < 1e-8


def test_bad_slab_and_quadrature_are_rejected():
    s = solid("tiny2")
    ctx = L.setup_from_solid(s, precision=L.FP64, real=True)
    cap = L.ltmp2_set_slab_size(ctx, 0)          # n <= 0 restores the capacity
    assert cap >= 1 and L.ltmp2_set_slab_size(ctx, -3) == cap
    with pytest.raises(L.Ltmp2Error) as e:
        L.ltmp2_set_slab_size(ctx, cap + 1)
    assert e.value.name == "INVALID_ARG"
    for tau, w in [([], []), ([0.0], [1.0]), ([-1.0], [1.0]), ([float("nan")], [1.0]), ([1.0], [float("inf")])]:
        with pytest.raises(L.Ltmp2Error) as e:
            L.ltmp2_energy(ctx, np.array(tau, dtype=float), np.array(w, dtype=float))
        assert e.value.name == "INVALID_ARG"
    L.ltmp2_destroy(ctx)


def test_gprime_shares_add_up_to_the_energy():
    """Three ranks' shares of the outer G' loop (evaluated here one after another) add up
    to the full energy: the split a multi-GPU run of one system would use."""
    from paper_1611_06797_gb300.shard import energy_share
    s = solid("cfg1")
    tau, w = sinc_laplace_quadrature(4, *denominator_range(OracleSystem.from_solid(s)))
    ctx = L.setup_from_solid(s, precision=L.FP64, real=True)
    ed, ex, _ = L.ltmp2_energy(ctx, tau, w)
    parts = [energy_share(ctx, tau, w, r, 3) for r in range(3)]
    L.ltmp2_destroy(ctx)
    assert abs(sum(p[0] for p in parts) - ed) < 1e-12 and abs(sum(p[1] for p in parts) - ex) < 1e-12


def test_bounded_wait_runs_out_and_is_reported():
    """A device wait on a barrier nothing completes runs out after its budget, raises the
    error word and the library reports TIMEOUT; the context stays usable afterwards."""
    import time
    s = solid("tiny2")
    tau, w = sinc_laplace_quadrature(3, *denominator_range(OracleSystem.from_solid(s)))
    ctx = L.setup_from_solid(s, precision=L.FP32, real=True)
    e0 = L.ltmp2_energy(ctx, tau, w)
    t0 = time.perf_counter()
    assert L.ltmp2_selftest_wait(ctx, 20000) == -7          # LTMP2_ERR_TIMEOUT after 20 ms
    assert time.perf_counter() - t0 >= 0.019
    assert L.ltmp2_selftest_wait(ctx, 0) == -1
    e1 = L.ltmp2_energy(ctx, tau, w)
    L.ltmp2_destroy(ctx)
    assert e1[0] == e0[0] and e1[1] == e0[1]

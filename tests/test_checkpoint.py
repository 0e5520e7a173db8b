"""Checkpoint / resume of an energy evaluation over chunks of the outer G' loop: host logic
on the CPU with a stand-in for the per-chunk partial energies (deterministic numbers), and
the C ABI on the GPU (an interrupted run resumed from its state file gives the energy of an
uninterrupted one)."""
import numpy as np
import pytest

import paper_1611_06797_gb300 as L
from paper_1611_06797_gb300.checkpoint import energy_checkpointed, energy_resumable


class _Crash(Exception):
    pass


def _fake(n_occ, calls, crash_at=None):
    def partial(b, e):
        if crash_at is not None and len(calls) == crash_at:
            raise _Crash()
        calls.append((b, e))
        rng = np.random.default_rng(1000 + b)
        pd = rng.standard_normal((n_occ, n_occ))
        px = rng.standard_normal((n_occ, n_occ))
        return float(pd.sum()), float(px.sum()), pd, px
    return partial


def test_resume_skips_saved_chunks_and_matches(tmp_path):
    tau, w = np.array([0.5, 2.0]), np.array([0.3, 0.7])
    path = str(tmp_path / "state.npz")
    full_calls = []
    full = energy_resumable(7, 23, 3, tau, w, str(tmp_path / "ref.npz"), 5, _fake(3, full_calls))
    assert [c for c in full_calls] == [(0, 5), (5, 10), (10, 15), (15, 20), (20, 23)]
    calls = []
    with pytest.raises(_Crash):
        energy_resumable(7, 23, 3, tau, w, path, 5, _fake(3, calls, crash_at=2))
    calls2 = []
    res = energy_resumable(7, 23, 3, tau, w, path, 5, _fake(3, calls2))
    assert calls2 == [(10, 15), (15, 20), (20, 23)] and res["resumed_chunks"] == 2
    assert res["E_d"] == full["E_d"] and res["E_x"] == full["E_x"]
    assert np.array_equal(res["e_d"], full["e_d"]) and np.array_equal(res["e_x"], full["e_x"])
    # a finished state is reused as it is
    calls3 = []
    again = energy_resumable(7, 23, 3, tau, w, path, 5, _fake(3, calls3))
    assert calls3 == [] and again["E_d"] == full["E_d"]


def test_state_for_another_quadrature_is_not_reused(tmp_path):
    path = str(tmp_path / "state.npz")
    energy_resumable(7, 10, 2, [1.0], [1.0], path, 4, _fake(2, []))
    calls = []
    energy_resumable(7, 10, 2, [1.0], [0.9], path, 4, _fake(2, calls))
    assert len(calls) == 3
    calls = []
    energy_resumable(7, 10, 2, [1.0], [0.9], path, 3, _fake(2, calls))   # other chunking
    assert len(calls) == 4
    with pytest.raises(ValueError):
        energy_resumable(7, 10, 2, [1.0], [1.0], path, 0, _fake(2, []))


def test_state_of_another_system_with_the_same_shape_is_not_reused(tmp_path):
    """Two systems of equal size, quadrature and chunking but different inputs (different
    fingerprints) never share a state file: the second one recomputes every chunk and
    gets its own energies, not the first one's."""
    path = str(tmp_path / "state.npz")
    a = energy_resumable(111, 12, 2, [1.0], [1.0], path, 4, _fake(2, []))

    def other(b, e):
        ed, ex, pd, px = _fake(2, [])(b, e)
        return -ed, -ex, -pd, -px
    calls = []

    def counted(b, e):
        calls.append(b)
        return other(b, e)
    b = energy_resumable(222, 12, 2, [1.0], [1.0], path, 4, counted)
    assert len(calls) == 3 and b["resumed_chunks"] == 0
    assert b["E_d"] == -a["E_d"] and b["E_x"] == -a["E_x"]


def test_chunk_sum_is_the_library_fixed_order_sum():
    """The resumed totals come from ltmp2_sum_partials: chunk 0 first, FP64."""
    rng = np.random.default_rng(5)
    e = rng.standard_normal((6, 2))
    pd = rng.standard_normal((6, 3, 3))
    px = rng.standard_normal((6, 3, 3))
    ed, ex, spd, spx = L.ltmp2_sum_partials(e, pd, px)
    ref_d = 0.0
    for c in range(6):
        ref_d += e[c, 0]
    assert ed == ref_d and abs(ex - e[:, 1].sum()) < 1e-15
    assert np.array_equal(spd, sum(pd[c] for c in range(6)))
    assert np.allclose(spx, px.sum(0), rtol=0, atol=1e-14)
    with pytest.raises(L.Ltmp2Error):
        L.ltmp2_sum_partials(np.array([[np.nan, 0.0]]), pd[:1], px[:1])


@pytest.mark.gpu
def test_checkpointed_energy_on_the_gpu(tmp_path):
    from oracle import OracleSystem, denominator_range, sinc_laplace_quadrature
    from tests.conftest import solid
    s = solid("cfg1")
    tau, w = sinc_laplace_quadrature(4, *denominator_range(OracleSystem.from_solid(s)))
    ctx = L.setup_from_solid(s, precision=L.FP64, real=True)
    ed, ex, ep = L.ltmp2_energy(ctx, tau, w)
    path = str(tmp_path / "cfg1.npz")
    n = L.ltmp2_num_primary_gprime(ctx)
    done = []

    def crashing(b, e):
        if len(done) == 3:
            raise _Crash()
        done.append(b)
        return L.ltmp2_energy_partial(ctx, tau, w, b, e)
    with pytest.raises(_Crash):
        energy_resumable(L.ltmp2_fingerprint(ctx), n, ctx.n_occ, tau, w, path, 9, crashing)
    r = energy_checkpointed(ctx, tau, w, path, chunk=9)
    L.ltmp2_destroy(ctx)
    assert r["resumed_chunks"] == 3
    assert abs(r["E_d"] - ed) < 1e-12 and abs(r["E_x"] - ex) < 1e-12
    assert np.abs(r["e_d"] + r["e_x"] - ep).max() < 1e-12

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
    full = energy_resumable(23, 3, tau, w, str(tmp_path / "ref.npz"), 5, _fake(3, full_calls))
    assert [c for c in full_calls] == [(0, 5), (5, 10), (10, 15), (15, 20), (20, 23)]
    calls = []
    with pytest.raises(_Crash):
        energy_resumable(23, 3, tau, w, path, 5, _fake(3, calls, crash_at=2))
    calls2 = []
    res = energy_resumable(23, 3, tau, w, path, 5, _fake(3, calls2))
    assert calls2 == [(10, 15), (15, 20), (20, 23)] and res["resumed_chunks"] == 2
    assert res["E_d"] == full["E_d"] and res["E_x"] == full["E_x"]
    assert np.array_equal(res["e_d"], full["e_d"]) and np.array_equal(res["e_x"], full["e_x"])
    # a finished state is reused as it is
    calls3 = []
    again = energy_resumable(23, 3, tau, w, path, 5, _fake(3, calls3))
    assert calls3 == [] and again["E_d"] == full["E_d"]


def test_state_for_another_quadrature_is_not_reused(tmp_path):
    path = str(tmp_path / "state.npz")
    energy_resumable(10, 2, [1.0], [1.0], path, 4, _fake(2, []))
    calls = []
    energy_resumable(10, 2, [1.0], [0.9], path, 4, _fake(2, calls))
    assert len(calls) == 3
    calls = []
    energy_resumable(10, 2, [1.0], [0.9], path, 3, _fake(2, calls))   # other chunking
    assert len(calls) == 4
    with pytest.raises(ValueError):
        energy_resumable(10, 2, [1.0], [1.0], path, 0, _fake(2, []))


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
        energy_resumable(n, ctx.n_occ, tau, w, path, 9, crashing)
    r = energy_checkpointed(ctx, tau, w, path, chunk=9)
    L.ltmp2_destroy(ctx)
    assert r["resumed_chunks"] == 3
    assert abs(r["E_d"] - ed) < 1e-12 and abs(r["E_x"] - ex) < 1e-12
    assert np.abs(r["e_d"] + r["e_x"] - ep).max() < 1e-12

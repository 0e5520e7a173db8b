"""Batching form: several systems of uneven grids and orbital counts evaluated by one
CUDA-graph launch (rounds of per-system GEMMs and shared persistent FFT stages when the
systems need similar numbers of rounds, else one graph branch per system) must give,
system by system, the energies of ltmp2_energy (FP64 to 1e-12 relative; FP32 to the rounding
of a different summation order in the column kernel) and, in FP64, the oracle's within
1e-8 Ha: on the small systems and on the eight uneven systems of the batching workload."""
import numpy as np
import pytest

import paper_1611_06797_gb300 as L
from oracle import OracleSystem, denominator_range, laplace_denominator, mp2_energy, sinc_laplace_quadrature
from tests.conftest import solid

pytestmark = pytest.mark.gpu

NAMES = ["tiny", "tiny2", "cfg1"]


def _setup(precision):
    solids = [solid(n) for n in NAMES]
    ctxs = [L.setup_from_solid(s, precision=precision, real=True) for s in solids]
    quads = [sinc_laplace_quadrature(s.spec.n_tau, *denominator_range(OracleSystem.from_solid(s))) for s in solids]
    return solids, ctxs, quads


@pytest.mark.parametrize("precision", [L.FP64, L.FP32])
def test_batch_graph_matches_individual_calls(precision):
    solids, ctxs, quads = _setup(precision)
    for c in ctxs:
        slab, var = L.ltmp2_autotune(c)
        assert 1 <= slab <= L.ltmp2_num_primary_gprime(c)
        assert (var == -1) == (precision == L.FP64)
    # one slab per Laplace point in every system: equal round counts, so the rounds run in
    # lockstep with the shared persistent FFT stages
    for c in ctxs:
        n = L.ltmp2_num_primary_gprime(c)
        assert L.ltmp2_set_slab_size(c, n) == n
    single = [L.ltmp2_energy(c, t, w)[:2] for c, (t, w) in zip(ctxs, quads)]
    b = L.ltmp2_batch_create(ctxs, [q[0] for q in quads], [q[1] for q in quads])
    assert b.kernel_nodes() > 0 and b.persistent()
    rel = 1e-12 if precision == L.FP64 else 2e-6
    for _ in range(2):          # the captured graph is replayed
        ed, ex = b.run()
        for k, (d, x) in enumerate(single):
            assert abs(ed[k] - d) <= rel * max(1.0, abs(d)) and abs(ex[k] - x) <= rel * max(1.0, abs(x))
    b.destroy()


def test_batching_workload_systems():
    """The eight systems of the batching workload (4..48 wells, 16^3..32^3, 8..96 occupied) in
    one persistent-round batch, two Laplace points each: FP32 against single calls; the four
    smallest in FP64 (an FP64 pass over all eight takes minutes) against single calls and,
    on the smallest, against the oracle."""
    from synth import BATCH_NAMES, SPECS, build_model_solid
    solids = [build_model_solid(SPECS[nm], device="cuda") for nm in BATCH_NAMES]
    quads = [sinc_laplace_quadrature(2, *denominator_range(OracleSystem.from_solid(s))) for s in solids]
    for precision, rel, count in ((L.FP32, 2e-6, 8), (L.FP64, 1e-12, 4)):
        ctxs = [L.setup_from_solid(s, precision=precision, real=True) for s in solids[:count]]
        single = [L.ltmp2_energy(c, t, w, pairs=False)[:2] for c, (t, w) in zip(ctxs, quads)]
        b = L.ltmp2_batch_create(ctxs, [q[0] for q in quads[:count]], [q[1] for q in quads[:count]])
        # rounds per system: n_tau x slabs; in lockstep only when the counts are balanced
        rounds = [len(q[0]) * -(-L.ltmp2_num_primary_gprime(c) // L.ltmp2_get_tuning(c)["slab"])
                  for c, q in zip(ctxs, quads)]
        assert b.persistent() == (max(rounds) <= 2 * min(rounds)), rounds
        ed, ex = b.run()
        b.destroy()
        for k, (d, x) in enumerate(single):
            assert abs(ed[k] - d) <= rel * abs(d) and abs(ex[k] - x) <= rel * abs(x), (precision, k)
        if precision == L.FP64:
            for k in (0,):
                ref = mp2_energy(OracleSystem.from_solid(solids[k]), laplace_denominator(*quads[k]))
                assert abs(ed[k] - ref["E_d"]) < 1e-8 and abs(ex[k] - ref["E_x"]) < 1e-8
        for c in ctxs:
            L.ltmp2_destroy(c)


def test_energy_batch_matches_oracle_fp64():
    solids, ctxs, quads = _setup(L.FP64)
    ed, ex = L.ltmp2_energy_batch(ctxs, [q[0] for q in quads], [q[1] for q in quads])
    for k, s in enumerate(solids):
        ref = mp2_energy(OracleSystem.from_solid(s), laplace_denominator(*quads[k]))
        assert abs(ed[k] - ref["E_d"]) < 1e-8 and abs(ex[k] - ref["E_x"]) < 1e-8


def test_autotune_is_cached_per_bucket():
    s = solid("cfg1")
    a = L.setup_from_solid(s, precision=L.FP32, real=True)
    b = L.setup_from_solid(s, precision=L.FP32, real=True)
    assert L.ltmp2_autotune(a) == L.ltmp2_autotune(b)


def test_batch_rejects_duplicate_contexts():
    s = solid("tiny")
    c = L.setup_from_solid(s)
    t, w = sinc_laplace_quadrature(3, 2 * s.gap, 2 * s.width)
    with pytest.raises(L.Ltmp2Error) as e:
        L.ltmp2_batch_create([c, c], [t, t], [w, w])
    assert e.value.name == "INVALID_ARG"

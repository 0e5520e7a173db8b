"""The N > 1 path on the CPU: world size 2 over gloo.  Each rank runs the benchmark's own
sharded evaluation (``shard.sharded_energy``: its share of the outer G' loop, Sec. III B,
and one FP64 sum all-reduce), with the oracle's working form standing in for the library's
partial-range call; the result equals the single-process energy.  The bench's timing reduction (max over ranks)
is checked the same way.  No GPU is used."""
import os
import socket
from datetime import timedelta

import numpy as np
import pytest

from paper_1611_06797_gb300.shard import gprime_share, sharded_energy


def test_gprime_share_partitions_the_loop():
    for n in (0, 1, 7, 870, 2724):
        for world in (1, 2, 3, 8):
            ranges = [gprime_share(n, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            assert all(ranges[k][1] == ranges[k + 1][0] for k in range(world - 1))
            sizes = [e - b for b, e in ranges]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        gprime_share(10, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist
    from oracle import OracleSystem, aux_set, denominator_range, sinc_laplace_quadrature
    from tests.conftest import solid
    from tests.test_oracle_pins import _working_form
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=timedelta(seconds=60))
    o = OracleSystem.from_solid(solid("tiny"))
    tau, w = sinc_laplace_quadrature(3, *denominator_range(o))
    n = len(aux_set(o)[0])

    # the library's partial-range call, stood in for by the oracle's working form on the
    # same G' range (pair matrices: E_d and E_x on the diagonal entry (0, 0) / (1, 1))
    def partial(sys_, tau_, w_, b, e):
        ed_, ex_ = _working_form(sys_, tau_, w_, range(b, e))
        pd, px = np.zeros((2, 2)), np.zeros((2, 2))
        pd[0, 0], px[1, 1] = ed_, ex_
        return ed_, ex_, pd, px

    def all_reduce_sum(v):
        t = torch.from_numpy(v)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        return t.numpy()
    ed, ex, ep = sharded_energy(o, tau, w, rank, world, all_reduce_sum, partial=partial, n_prim=n, n_occ=2)
    ms = torch.tensor([10.0 + rank], dtype=torch.float64)      # per-rank step time
    dist.all_reduce(ms, op=dist.ReduceOp.MAX)
    if rank == 0:
        out.put((ed, ex, float(ms[0]), float(ep[0, 0]), float(ep[1, 1])))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gprime_split_over_gloo():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    from oracle import OracleSystem, denominator_range, sinc_laplace_quadrature
    from tests.conftest import solid
    from tests.test_oracle_pins import _working_form
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
    alive = [p for p in procs if p.is_alive()]
    for p in alive:
        p.kill()
    assert not alive and all(p.exitcode == 0 for p in procs)
    ed, ex, ms, ep00, ep11 = out.get(timeout=10)
    o = OracleSystem.from_solid(solid("tiny"))
    tau, w = sinc_laplace_quadrature(3, *denominator_range(o))
    ed1, ex1 = _working_form(o, tau, w)
    assert abs(ed - ed1) < 1e-13 * abs(ed1) and abs(ex - ex1) < 1e-13 * abs(ex1)
    assert abs(ep00 - ed1) < 1e-13 * abs(ed1) and abs(ep11 - ex1) < 1e-13 * abs(ex1)
    assert ms == 11.0

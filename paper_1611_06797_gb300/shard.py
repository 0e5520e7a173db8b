"""Sharding of one system's outer G' loop across ranks (Sec. III B: the outer loop over G'
splits into independent, additive pieces).  Rank r of W evaluates the contiguous range
``gprime_share(n_prim, r, W)`` with ``ltmp2_energy_partial``; one FP64 sum-reduction of
(E_d, E_x, e_ij) over ranks gives the full energy (``sharded_energy``; the benchmark runs it
under torchrun with NCCL, the tests with gloo on the CPU)."""
from __future__ import annotations

from typing import Callable, Optional, Tuple

import numpy as np


def gprime_share(n_prim: int, rank: int, world: int) -> Tuple[int, int]:
    """[begin, end) of the primary G' evaluated by ``rank``: contiguous, disjoint, covering
    [0, n_prim), sizes differing by at most one (the first n_prim % world ranks get one more)."""
    if world < 1 or not 0 <= rank < world or n_prim < 0:
        raise ValueError("need world >= 1, 0 <= rank < world, n_prim >= 0")
    base, extra = divmod(n_prim, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def energy_share(ctx, tau, w, rank: int, world: int):
    """This rank's share of (E_d, E_x, e_pair_direct, e_pair_exchange) through the C ABI."""
    from .ltmp2 import ltmp2_energy_partial, ltmp2_num_primary_gprime
    b, e = gprime_share(ltmp2_num_primary_gprime(ctx), rank, world)
    return ltmp2_energy_partial(ctx, tau, w, b, e)


def sharded_energy(ctx, tau, w, rank: int, world: int, all_reduce_sum: Callable[[np.ndarray], np.ndarray],
                   partial: Optional[Callable] = None, n_prim: Optional[int] = None, n_occ: Optional[int] = None):
    """One E_MP2 split over ranks: this rank's share of the outer G' loop, then one sum
    all-reduce of the FP64 vector (E_d, E_x, e_ij) (``all_reduce_sum`` returns the sum over
    ranks of its argument).  ``partial(ctx, tau, w, begin, end)`` and ``n_prim`` default to
    the library's ``ltmp2_energy_partial`` and ``ltmp2_num_primary_gprime``.
    Returns (E_d, E_x, e_pair [n_occ][n_occ])."""
    from .ltmp2 import ltmp2_energy_partial, ltmp2_num_primary_gprime
    if partial is None:
        partial = ltmp2_energy_partial
    if n_prim is None:
        n_prim = ltmp2_num_primary_gprime(ctx)
    if n_occ is None:
        n_occ = ctx.n_occ
    b, e = gprime_share(n_prim, rank, world)
    ed, ex, pd, px = partial(ctx, tau, w, b, e)
    v = np.concatenate([[ed, ex], (np.asarray(pd) + np.asarray(px)).ravel()]).astype(np.float64)
    tot = np.asarray(all_reduce_sum(v), dtype=np.float64)
    return float(tot[0]), float(tot[1]), tot[2:].reshape(n_occ, n_occ)

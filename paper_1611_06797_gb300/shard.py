"""Sharding of one system's outer G' loop across ranks (Sec. III B: the outer loop over G'
splits into independent, additive pieces).  Rank r of W evaluates the contiguous range
``gprime_share(n_prim, r, W)`` with ``ltmp2_energy_partial``; one sum-reduction of
(E_d, E_x, e_ij) over ranks gives the full energy.  Every run of this library has one GPU,
so the multi-GPU driver is not built; this host logic is what it would use."""
from __future__ import annotations

from typing import Tuple


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

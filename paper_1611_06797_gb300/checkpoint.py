"""Checkpoint and resume of one energy evaluation.  The energy is additive over ranges of
the outer G' loop (Sec. III B; the paper accumulates its cutoff levels the same way,
Sec. III D), so the evaluation runs as chunks of primary G' through
``ltmp2_energy_partial``, each chunk's (E_d, E_x, e^d_ij, e^x_ij) saved to a state file as
soon as it is done.  A rerun of the same system (the context's input fingerprint, which
hashes the lattice, plane waves, coefficients, eigenvalues, precision and flags, and the
pair mask), quadrature and chunking skips the saved chunks; a state written for anything
else is ignored.  The totals are summed in chunk order at the end (by the library's
fixed-order FP64 sum), so a resumed result is identical to an uninterrupted one.  State files are replaced atomically (write, then
rename), so an interruption never leaves a half-written state."""
from __future__ import annotations

import hashlib
import os
from typing import Callable, Optional

import numpy as np


def _key(system_id: int, n_prim: int, n_occ: int, chunk: int, tau: np.ndarray, w: np.ndarray) -> str:
    h = hashlib.sha256()
    h.update(np.array([system_id], dtype=np.uint64).tobytes())
    h.update(np.array([n_prim, n_occ, chunk], dtype=np.int64).tobytes())
    h.update(np.ascontiguousarray(tau, dtype=np.float64).tobytes())
    h.update(np.ascontiguousarray(w, dtype=np.float64).tobytes())
    return h.hexdigest()


def _save(path: str, state: dict) -> None:
    tmp = path + ".tmp.npz"
    np.savez(tmp, **state)
    os.replace(tmp, path)


def energy_resumable(system_id: int, n_prim: int, n_occ: int, tau, w, path: str, chunk: int,
                     partial: Callable[[int, int], tuple],
                     reduce: Optional[Callable[[np.ndarray, np.ndarray, np.ndarray], tuple]] = None) -> dict:
    """Sum of partial(begin, end) -> (E_d, E_x, e^d_ij [n_occ][n_occ], e^x_ij) over chunks
    [begin, end) of length ``chunk`` covering [0, n_prim); saved to / resumed from ``path``
    (an .npz).  ``system_id`` identifies the inputs (a 64-bit fingerprint); a state written
    for another system, quadrature or chunking is not reused.  ``reduce(e, pd, px)`` sums
    the chunk results in order (the library's ``ltmp2_sum_partials`` through the C ABI)."""
    if chunk < 1 or n_prim < 0:
        raise ValueError("need chunk >= 1 and n_prim >= 0")
    tau = np.asarray(tau, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    key = _key(int(system_id), n_prim, n_occ, chunk, tau, w)
    nch = (n_prim + chunk - 1) // chunk
    state = None
    if os.path.exists(path):
        with np.load(path) as f:
            if str(f["key"]) == key:
                state = {k: f[k].copy() for k in f.files}
    if state is None:
        state = {"key": np.array(key), "done": np.zeros(nch, dtype=bool), "e": np.zeros((nch, 2)),
                 "pd": np.zeros((nch, n_occ, n_occ)), "px": np.zeros((nch, n_occ, n_occ))}
    resumed = int(state["done"].sum())
    for c in range(nch):
        if state["done"][c]:
            continue
        b, e = c * chunk, min(n_prim, (c + 1) * chunk)
        ed, ex, pd, px = partial(b, e)
        state["e"][c] = (ed, ex)
        state["pd"][c] = pd
        state["px"][c] = px
        state["done"][c] = True
        _save(path, state)
    if reduce is None:
        from .ltmp2 import ltmp2_sum_partials as reduce
    ed, ex, pd, px = reduce(state["e"], state["pd"], state["px"])
    return {"E_d": ed, "E_x": ex, "e_d": pd, "e_x": px, "chunks": nch, "resumed_chunks": resumed}


def energy_checkpointed(ctx, tau, w, path: str, chunk: Optional[int] = None) -> dict:
    """``energy_resumable`` through the C ABI for one context (chunk defaults to the slab)."""
    from .ltmp2 import ltmp2_energy_partial, ltmp2_fingerprint, ltmp2_get_tuning, ltmp2_num_primary_gprime
    n_prim = ltmp2_num_primary_gprime(ctx)
    if chunk is None:
        chunk = ltmp2_get_tuning(ctx)["slab"]
    return energy_resumable(ltmp2_fingerprint(ctx), n_prim, ctx.n_occ, tau, w, path, chunk,
                            lambda b, e: ltmp2_energy_partial(ctx, tau, w, b, e))

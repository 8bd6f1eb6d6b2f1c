"""Slice batches across devices (first-level slicing, SM Sec. IV.B).

Slices are independent: rank r of W contracts a contiguous range of the
plan's slice batches into its own complex128 amplitude buffer, and the
buffers are summed in rank order (fixed order: the result does not depend
on timing).  One exchange of k x 16 bytes per contraction.
"""

import numpy as np


def batch_range(n_batches: int, rank: int, world: int):
    """Contiguous share [lo, hi) of rank in 0..world-1; shares differ by at
    most one batch and cover [0, n_batches) exactly once."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank outside the world")
    base, extra = divmod(int(n_batches), int(world))
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def ordered_sum(parts):
    """Sum per-rank amplitude arrays in rank order (deterministic)."""
    acc = np.zeros_like(np.asarray(parts[0]))
    for p in parts:
        acc = acc + np.asarray(p)
    return acc


def check_peers(store, tag: str, rank: int, world: int, timeout_s: float = 10.0):
    """Heartbeat before an exchange: every rank posts ``tag/rank`` in the
    rendezvous store and waits for all of them; a rank that left (or never
    arrives) makes the others raise here, on the host, instead of blocking
    inside a collective."""
    from datetime import timedelta
    store.set(f"{tag}/{rank}", "1")
    keys = [f"{tag}/{r}" for r in range(world)]
    try:
        store.wait(keys, timedelta(seconds=timeout_s))
    except Exception as e:  # noqa: BLE001 -- the store raises on timeout
        missing = [k for k in keys if not store.check([k])]
        raise RuntimeError(f"ranks missing before '{tag}': {missing}") from e


def reduce_amplitudes(local, group=None, store=None, tag="reduce", timeout_s=10.0):
    """All ranks receive sum_r local_r, summed in rank order.  ``local`` is a
    complex128 numpy array (host copy of the rank's amplitudes).  With a
    ``store``, a heartbeat (:func:`check_peers`) runs first.  Uses
    torch.distributed all_gather on the default or given group."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    if store is not None:
        check_peers(store, tag, dist.get_rank(group), world, timeout_s)
    t = torch.from_numpy(np.ascontiguousarray(local).view(np.float64).copy())
    bufs = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(bufs, t, group=group)
    return ordered_sum([b.numpy().view(np.complex128) for b in bufs])


def contract_sharded(plan, amps, precision, rank, world, stream=None):
    """This rank's share of the slice batches of ``plan`` into ``amps``."""
    lo, hi = batch_range(plan.info["n_batches"], rank, world)
    if hi > lo:
        plan.tn_contract(amps, precision, lo, hi, stream=stream)
    return lo, hi

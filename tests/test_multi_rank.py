"""Slice partition across ranks and the fixed-order amplitude reduction,
on world-size-2 gloo process groups (CPU).  The per-rank compute is the CPU
oracle's per-slice partials (test infrastructure), so the exchange logic is
checked against the unsliced amplitude without a GPU."""

import os
import socket
import multiprocessing as mp

import numpy as np
import pytest

from paper_2212_04749_gb300.multi import batch_range, ordered_sum


def test_batch_ranges_partition_exactly():
    for n in (1, 2, 7, 1024):
        for world in (1, 2, 3, 8):
            ranges = [batch_range(n, r, world) for r in range(world)]
            covered = [b for lo, hi in ranges for b in range(lo, hi)]
            assert covered == list(range(n))
            sizes = [hi - lo for lo, hi in ranges]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        batch_range(8, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, drop, q):
    import torch.distributed as dist
    from datetime import timedelta
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    try:
        store = dist.TCPStore("127.0.0.1", port, world, is_master=(rank == 0), timeout=timedelta(seconds=30))
        dist.init_process_group("gloo", store=store, rank=rank, world_size=world, timeout=timedelta(seconds=8))
        from oracle import tn as otn
        from paper_2212_04749_gb300.multi import batch_range, reduce_amplitudes
        from rqc import make_workload
        from rqc.tree import choose_slices
        w = make_workload("grid3x4_m8")
        sl = choose_slices(w.struct, w.tree, 64, n_sliced=3)
        wires = [tuple(int(x) for x in w.struct.edge_wire[e]) for e in sl]
        lo, hi = batch_range(8, rank, world)  # one slice per batch here
        parts = otn.partial_amplitudes(w.circuit, w.tree.ssa, w.bits, wires, list(range(lo, hi)))
        local = parts.sum(axis=0)
        if drop and rank == 1:
            q.put((rank, "dropped", None))
            q.close()
            q.join_thread()  # flush the message before leaving
            os._exit(0)  # leaves between steps, nothing in flight
        total = reduce_amplitudes(local, store=store, tag="step0", timeout_s=5.0)
        q.put((rank, "ok", total))
        dist.destroy_process_group()
    except Exception as e:  # noqa: BLE001
        q.put((rank, "error", repr(e)))


def _run(world, drop):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, world, port, drop, q)) for r in range(world)]
    for p in ps:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in ps:
        p.join(timeout=60)
        if p.is_alive():
            p.kill()
    return sorted(out, key=lambda x: x[0])


def test_two_ranks_sum_to_the_unsliced_amplitudes():
    from oracle import sv
    from rqc import make_workload
    out = _run(2, drop=False)
    ref = sv.amplitudes(make_workload("grid3x4_m8").circuit, make_workload("grid3x4_m8").bits)
    for rank, status, total in out:
        assert status == "ok", total
        assert np.max(np.abs(total - ref)) < 1e-13
    assert np.array_equal(out[0][2], out[1][2])  # identical on every rank (fixed order)


def test_a_dropped_rank_surfaces_as_an_error_not_a_hang():
    out = _run(2, drop=True)
    assert out[1][1] == "dropped"
    assert out[0][1] == "error" and "missing" in out[0][2]  # rank 0 learns it on the host


def test_ordered_sum_is_rank_ordered():
    a = np.array([1e16, 1.0, -1e16]) + 0j
    assert ordered_sum([a[:1], a[1:2], a[2:]])[0] == ((1e16 + 1.0) - 1e16)


def _plan_worker(rank, world, port, q):
    # each rank builds the same plan on its host (the planner needs no GPU),
    # takes its contiguous share of the plan's slice batches, turns them into
    # slice ids with tn_plan_batch_slices and contributes the oracle's
    # partials of exactly those slices (standing in for its device's
    # tn_contract over [lo, hi)); the rank-ordered sum is the amplitude
    import torch.distributed as dist
    from datetime import timedelta
    try:
        store = dist.TCPStore("127.0.0.1", port, world, is_master=(rank == 0), timeout=timedelta(seconds=30))
        dist.init_process_group("gloo", store=store, rank=rank, world_size=world, timeout=timedelta(seconds=8))
        from oracle import tn as otn
        from paper_2212_04749_gb300 import builder, tn
        from paper_2212_04749_gb300.multi import batch_range, reduce_amplitudes
        from rqc import make_workload
        from rqc.tree import choose_slices
        builder.build()
        w = make_workload("grid3x4_m8")
        sl = choose_slices(w.struct, w.tree, 64, n_sliced=3)
        p = tn.Plan(w.circuit, w.bits, w.tree.ssa, sl, slice_batch_log2=1)
        nb = p.info["n_batches"]
        lo, hi = batch_range(nb, rank, world)
        ids = [int(x) for b in range(lo, hi) for x in p.tn_plan_batch_slices(b)]
        wires = [tuple(int(x) for x in w.struct.edge_wire[e]) for e in sl]
        local = otn.partial_amplitudes(w.circuit, w.tree.ssa, w.bits, wires, ids).sum(axis=0)
        total = reduce_amplitudes(local, store=store, tag="plan_step0", timeout_s=5.0)
        q.put((rank, "ok", (nb, ids, total)))
        dist.destroy_process_group()
    except Exception as e:  # noqa: BLE001
        q.put((rank, "error", repr(e)))


def test_plan_batch_ranges_partition_the_slices_across_ranks():
    from oracle import sv
    from rqc import make_workload
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_plan_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted([q.get(timeout=180) for _ in range(2)], key=lambda x: x[0])
    for p in ps:
        p.join(timeout=60)
        if p.is_alive():
            p.kill()
    for rank, status, res in out:
        assert status == "ok", res
    nb = out[0][2][0]
    assert nb == 4  # 3 sliced edges, 2 per pass
    ids = out[0][2][1] + out[1][2][1]
    assert sorted(ids) == list(range(8)) and len(out[0][2][1]) == len(out[1][2][1]) == 4
    w = make_workload("grid3x4_m8")
    ref = sv.amplitudes(w.circuit, w.bits)
    assert np.max(np.abs(out[0][2][2] - ref)) < 1e-13
    assert np.array_equal(out[0][2][2], out[1][2][2])

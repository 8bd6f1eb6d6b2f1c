"""Amplitudes of successive bitstring batches with host planning overlapped.

A plan is built on the host for each batch of bitstrings (the instance
tables of the reuse tree depend on them) and then contracted on the GPU.
`contract_batches` builds the plan of batch i + 1 on a worker thread while
batch i runs on the device, so that a stream of batches costs about
max(planning, contraction) per batch instead of their sum.  Planning is the
library's host code (the C call releases the interpreter lock); with one
workspace, binding, contraction and the copy of the amplitudes to pinned
host memory stay on the calling thread, one batch at a time.  Given w >= 2
workspaces, w - 1 worker threads plan batches i + 1 .. i + w - 1 at once and
bind each (upload its tables on a side stream) into the workspace of an
earlier batch once that batch has finished, and the calling thread launches
batch i + 1 before it reads batch i's result (two amplitude buffers in
turn), so that the next plan's first launch (its graph capture) overlaps the
running batch: a batch then costs about max(planning / (w - 1),
contraction).
"""

from concurrent.futures import ThreadPoolExecutor

import numpy as np

from . import tn


def contract_batches(circ, batches, tree_ssa, sliced, precision, workspace, stream=None, configs=None, chains=None,
                     **opts):
    """Yield (batch index, amplitudes) for each bitstring batch in order.

    circ, tree_ssa, sliced, **opts: as for tn.Plan; every batch is planned
    with them.  batches: a sequence of (k_i x n) 0/1 arrays.  precision: a
    precision name or TN_* code.  workspace: a CUDA uint8 tensor of at least
    the largest plan's workspace_bytes, or a list of w >= 2 of them (w - 1
    later batches are then planned and their tables uploaded while the
    current batch runs).  stream: the torch CUDA stream the
    contractions run on (default: the current stream).  configs: optional
    per-step configurations applied to every plan (all batches must then
    yield plans with the same step count); chains: optional per-chain fused
    flags (tn_plan_set_chain) applied likewise.  The amplitudes are complex128
    numpy arrays in input order (rows x 2^|open qubits| with
    opts open_qubits / open_mask), read from pinned host memory after the
    batch's contraction finished.
    """
    import torch

    stream = stream or torch.cuda.current_stream()
    n = len(batches)
    if n == 0:
        return
    spaces = list(workspace) if isinstance(workspace, (list, tuple)) else [workspace]
    if not spaces:
        raise ValueError("workspace: at least one buffer")
    nws = len(spaces)
    ahead = max(1, nws - 1)  # batches planned while one runs
    sides = [torch.cuda.Stream(device=stream.device) for _ in range(ahead)] if nws >= 2 else None
    check = torch.cuda.Stream(device=stream.device)  # reads a finished batch's error word
    done = {}  # workspace index -> event after the last contraction that used it

    def plan_of(i, prev):
        p = tn.Plan(circ, batches[i], tree_ssa, sliced, **opts)
        if sides is not None:  # bind here, into the buffer batch i - nws used, once that has finished
            ws = spaces[i % nws]
            if p.info["workspace_bytes"] > ws.numel():
                raise ValueError(f"batch {i}: plan needs {p.info['workspace_bytes']} workspace bytes, "
                                 f"workspace holds {ws.numel()}")
            if prev is not None:
                prev.synchronize()
            side = sides[i % ahead]
            p.tn_plan_bind(ws, stream=side)
            side.synchronize()
        return p

    # two amplitude buffers (device and pinned host) in turn: batch i + 1 is
    # launched before batch i's result is read
    amps, host = [None, None], [None, None]
    pending = None  # (index, plan, pinned result, event after its copy)

    def finish(item):
        j, pj, hj, ev = item
        ev.synchronize()
        pj.tn_plan_check(stream=check)  # its contraction has finished; syncs `check` only
        return j, hj.numpy().view(np.complex128).copy()

    with ThreadPoolExecutor(max_workers=ahead) as ex:
        futs = {j: ex.submit(plan_of, j, None) for j in range(min(ahead, n))}
        for i in range(n):
            p = futs.pop(i).result()
            # batch i + ahead binds into the buffer of batch i - 1 once that finishes
            if i + ahead < n:
                j = i + ahead
                futs[j] = ex.submit(plan_of, j, done.get(j % nws))
            if configs is not None:
                for s, c in enumerate(configs):
                    p.tn_plan_set_config(s, int(c))
            if chains is not None:
                for c, on in enumerate(chains):
                    p.tn_plan_set_chain(c, int(on))
            m = len(batches[i]) * p.info["amps_per_row"]
            if sides is None:
                # one workspace: the previous batch finishes before this one binds
                if pending is not None:
                    yield finish(pending)
                    pending = None
                if p.info["workspace_bytes"] > spaces[0].numel():
                    raise ValueError(f"batch {i}: plan needs {p.info['workspace_bytes']} workspace bytes, "
                                     f"workspace holds {spaces[0].numel()}")
                p.tn_plan_bind(spaces[0], stream=stream)
            b = i % 2
            with torch.cuda.stream(stream):
                if amps[b] is None or amps[b].numel() < 2 * m:
                    amps[b] = torch.zeros(2 * max(m, 1), dtype=torch.float64, device=stream.device)
                    host[b] = torch.empty(2 * max(m, 1), dtype=torch.float64, pin_memory=True)
                a = amps[b][:2 * m]
                a.zero_()
                p.tn_contract(a, precision, stream=stream)
                h = host[b][:2 * m]
                h.copy_(a, non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(stream)
            if sides is not None:
                done[i % nws] = ev
            if pending is not None:
                yield finish(pending)
            pending = (i, p, h, ev)
            del p
        if pending is not None:
            yield finish(pending)

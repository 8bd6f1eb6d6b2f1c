"""Amplitudes of successive bitstring batches with host planning overlapped.

A plan is built on the host for each batch of bitstrings (the instance
tables of the reuse tree depend on them) and then contracted on the GPU.
`contract_batches` builds the plan of batch i + 1 on a worker thread while
batch i runs on the device, so that a stream of batches costs about
max(planning, contraction) per batch instead of their sum.  Planning is the
library's host code (the C call releases the interpreter lock); binding,
contraction and the copy of the amplitudes to pinned host memory stay on the
calling thread, one batch at a time, so every plan uses the same workspace.
Given two workspaces, the worker thread also binds batch i + 1 (uploads its
tables on a side stream) into the one batch i - 1 used, while batch i
runs in the other.
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
    the largest plan's workspace_bytes, or a pair of them (the next batch's
    tables then upload while the current batch runs).  stream: the torch CUDA stream the
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
    amps = host = None  # grown to the largest batch (rows x amplitudes per row)
    spaces = list(workspace) if isinstance(workspace, (list, tuple)) else [workspace]
    if len(spaces) not in (1, 2):
        raise ValueError("workspace: one buffer or a pair")
    side = torch.cuda.Stream(device=stream.device) if len(spaces) == 2 else None

    def plan_of(i):
        p = tn.Plan(circ, batches[i], tree_ssa, sliced, **opts)
        if side is not None:  # bind here, into the buffer batch i - 1 has released
            ws = spaces[i % 2]
            if p.info["workspace_bytes"] > ws.numel():
                raise ValueError(f"batch {i}: plan needs {p.info['workspace_bytes']} workspace bytes, "
                                 f"workspace holds {ws.numel()}")
            p.tn_plan_bind(ws, stream=side)
            side.synchronize()
        return p

    with ThreadPoolExecutor(max_workers=1) as ex:
        nxt = ex.submit(plan_of, 0)
        for i in range(n):
            p = nxt.result()
            if i + 1 < n:
                nxt = ex.submit(plan_of, i + 1)
            if configs is not None:
                for s, c in enumerate(configs):
                    p.tn_plan_set_config(s, int(c))
            if chains is not None:
                for c, on in enumerate(chains):
                    p.tn_plan_set_chain(c, int(on))
            m = len(batches[i]) * p.info["amps_per_row"]
            if amps is None or amps.numel() < 2 * m:
                amps = torch.zeros(2 * max(m, 1), dtype=torch.float64, device="cuda")
                host = torch.empty(2 * max(m, 1), dtype=torch.float64, pin_memory=True)
            if side is None:
                if p.info["workspace_bytes"] > spaces[0].numel():
                    raise ValueError(f"batch {i}: plan needs {p.info['workspace_bytes']} workspace bytes, "
                                     f"workspace holds {spaces[0].numel()}")
                p.tn_plan_bind(spaces[0], stream=stream)
            a = amps[:2 * m]
            a.zero_()
            p.tn_contract(a, precision, stream=stream)
            h = host[:2 * m]
            h.copy_(a, non_blocking=True)
            stream.synchronize()
            p.tn_plan_check(stream=stream)
            del p
            yield i, h.numpy().view(np.complex128).copy()

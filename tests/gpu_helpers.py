"""Shared helpers of the GPU tests: run a plan through the C ABI on cuda:0."""

import numpy as np


def require_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU test run without a CUDA device"
    from paper_2212_04749_gb300 import builder, tn
    builder.build()
    tn.load()
    return torch, tn


def run_plan(circ, bits, ssa, sliced=(), precision="fp32", batches=None, force_kernel=None, force_config=None,
             tc_pairs=None, **opts):
    """Amplitudes (complex128, input order) summed over every slice batch.
    force_kernel: a function step_info -> kernel family (or None) applied to
    every step before the run; force_config likewise for the step's
    configuration (family x schedule); tc_pairs switches the tensor-core
    column-tile pairs on or off (None: the plan's default)."""
    torch, tn = require_cuda()
    p = tn.Plan(circ, bits, ssa, sliced, **opts)
    if force_kernel is not None:
        for s, st in enumerate(p.tn_plan_steps()):
            k = force_kernel(st)
            if k is not None:
                p.tn_plan_set_kernel(s, k)
    if force_config is not None:
        for s, st in enumerate(p.tn_plan_steps()):
            c = force_config(st)
            if c is not None:
                p.tn_plan_set_config(s, c)
    if tc_pairs is not None:
        p.tn_plan_set_tc_pairs(tc_pairs)
    ws = torch.empty(max(p.info["workspace_bytes"], 256), dtype=torch.uint8, device="cuda")
    p.tn_plan_bind(ws, stream=torch.cuda.current_stream())
    amps = torch.zeros(2 * len(bits) * p.info["amps_per_row"], dtype=torch.float64, device="cuda")
    if batches is None:
        p.tn_contract(amps, precision, stream=torch.cuda.current_stream())
    else:
        for lo, hi in batches:
            p.tn_contract(amps, precision, lo, hi, stream=torch.cuda.current_stream())
    p.tn_plan_check(stream=torch.cuda.current_stream())
    torch.cuda.synchronize()
    return amps.cpu().numpy().view(np.complex128), p


def run_slices(circ, bits, ssa, sliced, slice_ids, precision="fp32", **opts):
    torch, tn = require_cuda()
    p = tn.Plan(circ, bits, ssa, sliced, **opts)
    ws = torch.empty(max(p.info["workspace_bytes"], 256), dtype=torch.uint8, device="cuda")
    p.tn_plan_bind(ws, stream=torch.cuda.current_stream())
    out = torch.zeros(2 * len(bits) * len(slice_ids), dtype=torch.float64, device="cuda")
    p.tn_contract_slices(slice_ids, out, precision, stream=torch.cuda.current_stream())
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.complex128).reshape(len(slice_ids), len(bits))


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))

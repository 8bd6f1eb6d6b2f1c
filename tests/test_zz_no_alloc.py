"""tn_contract_static: the contraction for callers that cannot allocate
device memory (the workspace is the library's fixed device array).

Collected last on purpose (file name), so that a run stopping at its first
failure has already run every other test.  Passes alone in a fresh process
and after the rest of the suite.
"""

import numpy as np
import pytest

from gpu_helpers import rel_l2, require_cuda
from rqc import make_workload
from rqc.tree import choose_slices

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5


def _case():
    w = make_workload("grid3x4_m8")
    sl = choose_slices(w.struct, w.tree, 64, n_sliced=3)
    return w, sl


def test_static_scratch_matches_bound_workspace_twice():
    torch, tn = require_cuda()
    w, sl = _case()
    stream = torch.cuda.current_stream()
    p = tn.Plan(w.circuit, w.bits, w.tree.ssa, sl, slice_batch_log2=1)
    assert p.info["workspace_bytes"] <= tn.TN_STATIC_SCRATCH_BYTES
    ws = torch.empty(p.info["workspace_bytes"], dtype=torch.uint8, device="cuda")
    p.tn_plan_bind(ws, stream=stream)
    ref = torch.zeros(2 * 64, dtype=torch.float64, device="cuda")
    p.tn_contract(ref, "fp32", stream=stream)
    p.tn_plan_check(stream=stream)
    ref_h = ref.cpu().numpy().view(np.complex128)
    for _ in range(2):  # two calls in a row share (and reuse) the array
        out = torch.zeros(2 * 64, dtype=torch.float64, device="cuda")
        p.tn_contract_static(out, "fp32", stream=stream)
        torch.cuda.synchronize()
        assert rel_l2(out.cpu().numpy().view(np.complex128), ref_h) <= FP32_TOL
    # the plan's own workspace binding is untouched
    again = torch.zeros(2 * 64, dtype=torch.float64, device="cuda")
    p.tn_contract(again, "fp32", stream=stream)
    p.tn_plan_check(stream=stream)
    assert rel_l2(again.cpu().numpy().view(np.complex128), ref_h) <= FP32_TOL


def test_static_scratch_without_any_bound_workspace():
    torch, tn = require_cuda()
    w, sl = _case()
    p = tn.Plan(w.circuit, w.bits, w.tree.ssa, sl)
    out = torch.zeros(2 * 64, dtype=torch.float64, device="cuda")
    p.tn_contract_static(out, "fp32")
    torch.cuda.synchronize()
    from oracle import sv
    assert rel_l2(out.cpu().numpy().view(np.complex128), sv.amplitudes(w.circuit, w.bits)) <= FP32_TOL


def test_static_scratch_rejects_plans_above_its_size():
    torch, tn = require_cuda()
    w = make_workload("grid5x6_m14")
    p = tn.Plan(w.circuit, w.bits, w.tree.ssa, w.tree.sliced)
    out = torch.zeros(2 * w.bits.shape[0], dtype=torch.float64, device="cuda")
    with pytest.raises(tn.TnError) as ei:
        p.tn_contract_static(out, "fp32")
    assert ei.value.code == tn.TN_ENOMEM
    assert "fixed scratch" in str(ei.value)

"""tn_contract_static: the contraction for callers that cannot allocate
device memory (the workspace is the library's fixed device array): code
embedded in a host application whose device memory pools belong to another
runtime, or a process whose device memory is fixed up front.

Collected last on purpose (file name), so that a run stopping at its first
failure has already run every other test.  Passes alone in a fresh process
and after the rest of the suite.
"""

import numpy as np
import pytest

from gpu_helpers import rel_l2, require_cuda
from rqc import grid_layout, make_workload, network_structure, random_circuit
from rqc.bitstrings import uniform_bitstrings
from rqc.tree import ContractionTree, candidate_trees, choose_slices

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5
MIXED_TOL = 1e-3


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


def _case16():
    # 16 qubits, 10 cycles, 256 bitstrings: a plan of about 1 MiB whose
    # GEMM-shaped steps (K >= 8, M >= 64) run on the tensor cores once every
    # step is set to the grouped GEMM
    c = random_circuit(grid_layout(4, 4), 10, seed=21)
    st = network_structure(c)
    bits = uniform_bitstrings(16, 256, seed=5)
    ssa = candidate_trees(st, 256, seed=2, trials=2)[0]
    sl = choose_slices(st, ContractionTree(ssa=ssa), 256, n_sliced=2)
    return c, bits, ssa, sl


def test_static_scratch_on_tensor_core_steps_twice_and_allocates_nothing():
    # the fixed array also carries the TMA descriptors' operands: the
    # tensor-core steps read A through tensor maps encoded over its address
    torch, tn = require_cuda()
    from oracle import sv
    c, bits, ssa, sl = _case16()
    stream = torch.cuda.current_stream()
    p = tn.Plan(c, bits, ssa, sl, rescale=1)
    assert p.info["workspace_bytes"] <= tn.TN_STATIC_SCRATCH_BYTES
    for s_ in range(p.info["n_steps"]):
        p.tn_plan_set_kernel(s_, 1)
    ws = torch.empty(p.info["workspace_bytes"], dtype=torch.uint8, device="cuda")
    p.tn_plan_bind(ws, stream=stream)
    ref = torch.zeros(2 * 256, dtype=torch.float64, device="cuda")
    p.tn_plan_profile(True)
    p.tn_contract(ref, "bf16x3", stream=stream)
    fams = p.tn_plan_step_times()[1]
    p.tn_plan_profile(False)
    assert int(np.sum(np.asarray(fams) == 2)) > 0, "no tensor-core step in the case"
    ref_h = ref.cpu().numpy().view(np.complex128)
    assert rel_l2(ref_h, sv.amplitudes(c, bits)) <= MIXED_TOL
    out = torch.zeros(2 * 256, dtype=torch.float64, device="cuda")
    p.tn_contract_static(out, "bf16x3", stream=stream)  # warm-up: the first call looks up the array
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        out.zero_()
        p.tn_contract_static(out, "bf16x3", stream=stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.complex128)
        # same kernels, same configuration: the same bits as the bound workspace
        assert np.array_equal(got.view(np.uint64), ref_h.view(np.uint64))
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)


def test_static_scratch_with_open_qubits():
    # correlated batches: k rows x 2^|open| amplitudes land in the caller's
    # buffer, sized from tn_plan_info.amps_per_row
    torch, tn = require_cuda()
    from oracle import sv
    w, sl = _case()
    rows = w.bits[:16]
    p = tn.Plan(w.circuit, rows, w.tree.ssa, sl, open_qubits=[10, 11])
    assert p.info["amps_per_row"] == 4
    out = torch.zeros(2 * 16 * 4, dtype=torch.float64, device="cuda")
    p.tn_contract_static(out, "fp32")
    torch.cuda.synchronize()
    ref = sv.correlated_amplitudes(w.circuit, rows, [10, 11])
    assert rel_l2(out.cpu().numpy().view(np.complex128), np.asarray(ref).ravel()) <= FP32_TOL
    # a buffer sized for one amplitude per row is refused before any launch
    small = torch.zeros(2 * 16, dtype=torch.float64, device="cuda")
    with pytest.raises(tn.TnError) as ei:
        p.tn_contract_static(small, "fp32")
    assert ei.value.code == tn.TN_EINVAL

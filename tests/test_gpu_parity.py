"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances: relative L2 error over the compared amplitudes <= 1e-5 for the
FP32 path and <= 1e-3 for the tensor-core forms (TF32, BF16x3), the bounds
the task fixes; bitwise equality where the arithmetic is identical by
construction (rescaling by powers of two; an instance's arithmetic does not
depend on which other bitstrings share the pass).
"""

import numpy as np
import pytest

from gpu_helpers import require_cuda, rel_l2, run_plan, run_slices
from oracle import sv, tn as otn, xeb
from rqc import make_workload, grid_layout, random_circuit, network_structure
from rqc.bitstrings import uniform_bitstrings
from rqc.circuit import Circuit, Gate
from rqc.tree import candidate_trees, choose_slices

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5


def test_grid3x4_fp32_matches_state_vector():
    w = make_workload("grid3x4_m8")
    ref = sv.amplitudes(w.circuit, w.bits)
    got, p = run_plan(w.circuit, w.bits, w.tree.ssa)
    assert rel_l2(got, ref) <= FP32_TOL


def test_rescaling_is_bitwise_neutral_in_fp32():
    w = make_workload("grid3x4_m8")
    a, _ = run_plan(w.circuit, w.bits, w.tree.ssa, rescale=1)
    b, _ = run_plan(w.circuit, w.bits, w.tree.ssa, rescale=0)
    assert np.array_equal(a.view(np.uint64), b.view(np.uint64))


@pytest.mark.parametrize("family", [0, 1])
def test_reuse_does_not_change_an_instance_bitwise(family):
    # P8: under one kernel configuration, every bitstring alone (the
    # single-amplitude contraction) equals its value inside the shared
    # multiple-amplitude pass, bit for bit
    w = make_workload("grid3x4_m8")

    def pin(st):  # the per-row kernel where its shape allows, else the GEMM
        return family if (family == 1 or (st["nb"] <= 4 and st["kb"] + st["nb"] <= 8)) else 1
    batch, _ = run_plan(w.circuit, w.bits, w.tree.ssa, force_kernel=pin)
    for i in (0, 7, 33, 63):
        one, _ = run_plan(w.circuit, w.bits[i:i + 1], w.tree.ssa, force_kernel=pin)
        assert one[0].real == batch[i].real and one[0].imag == batch[i].imag


@pytest.mark.parametrize("batch_log2", [0, 1, 3])
def test_sliced_sum_matches_state_vector(batch_log2):
    w = make_workload("grid3x4_m8")
    sl = choose_slices(w.struct, w.tree, 64, n_sliced=3)
    ref = sv.amplitudes(w.circuit, w.bits)
    got, p = run_plan(w.circuit, w.bits, w.tree.ssa, sl, slice_batch_log2=batch_log2)
    assert p.info["n_batches"] == 2 ** (3 - batch_log2)
    assert rel_l2(got, ref) <= FP32_TOL


def test_batch_ranges_partition_the_slices():
    # the multi-device partition: disjoint batch ranges summed
    w = make_workload("grid3x4_m8")
    sl = choose_slices(w.struct, w.tree, 64, n_sliced=3)
    ref = sv.amplitudes(w.circuit, w.bits)
    got, _ = run_plan(w.circuit, w.bits, w.tree.ssa, sl, slice_batch_log2=0, batches=[(0, 3), (3, 8)])
    assert rel_l2(got, ref) <= FP32_TOL


def test_slice_partials_match_oracle_per_slice():
    w = make_workload("grid3x4_m8")
    sl = choose_slices(w.struct, w.tree, 64, n_sliced=3)
    wires = [tuple(int(x) for x in w.struct.edge_wire[e]) for e in sl]
    ids = [0, 3, 5, 6, 7]
    ref = otn.partial_amplitudes(w.circuit, w.tree.ssa, w.bits, wires, ids)
    for bl in (0, 2):
        got = run_slices(w.circuit, w.bits, w.tree.ssa, sl, ids, slice_batch_log2=bl)
        assert rel_l2(got, ref) <= FP32_TOL


def test_duplicate_and_single_bitstrings():
    w = make_workload("grid3x4_m8")
    bits = np.concatenate([w.bits[:5], w.bits[:5], w.bits[2:3]])
    ref = sv.amplitudes(w.circuit, bits)
    got, p = run_plan(w.circuit, bits, w.tree.ssa)
    assert p.info["n_unique"] == 5
    assert rel_l2(got, ref) <= FP32_TOL
    assert np.array_equal(got[:5], got[5:10])


def test_single_gate_circuit_root_is_a_leaf():
    # degenerate network: one two-qubit gate, the root is a leaf tensor
    g = random_circuit(grid_layout(1, 2), 1, seed=3)
    bits = np.array([[0, 0], [0, 1], [1, 0], [1, 1]], np.uint8)
    ref = sv.amplitudes(g, bits)
    got, _ = run_plan(g, bits, np.zeros((0, 2), np.int32))
    assert rel_l2(got, ref) <= FP32_TOL


@pytest.mark.parametrize("trial", [0, 1, 2])
def test_other_trees_and_circuits(trial):
    c = random_circuit(grid_layout(3, 3), 10, seed=40 + trial)
    s = network_structure(c)
    bits = uniform_bitstrings(9, 100, seed=trial)
    trees = candidate_trees(s, 100, seed=trial, trials=2)
    ref = sv.amplitudes(c, bits)
    for ssa in (trees[0], trees[-1]):
        got, _ = run_plan(c, bits, ssa)
        assert rel_l2(got, ref) <= FP32_TOL


def test_xeb_kernel_matches_definition():
    import torch
    from gpu_helpers import require_cuda
    _, tn = require_cuda()
    rng = np.random.default_rng(3)
    a = (rng.normal(size=5000) + 1j * rng.normal(size=5000)) * 2 ** -7
    dev = torch.from_numpy(a.view(np.float64).copy()).cuda()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    tn.tn_xeb(dev, 5000, 14, out)
    torch.cuda.synchronize()
    assert abs(out.item() - xeb.linear_xeb(a, 14)) < 1e-12


def test_grid5x6_fp32_matches_stored_state_vector():
    # 30 qubits, 14 cycles, 4096 bitstrings, 2^10 slices: every amplitude
    # against the complex128 state vector written by tests/golden/make_golden.py
    import importlib.util, os
    spec = importlib.util.spec_from_file_location(
        "make_golden", os.path.join(os.path.dirname(__file__), "golden", "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    digest, ref = mg.read("grid5x6_m14")
    w = make_workload("grid5x6_m14")
    assert digest == mg.input_digest(w.circuit, w.bits)
    got, p = run_plan(w.circuit, w.bits, w.tree.ssa, w.tree.sliced)
    assert p.info["n_sliced"] == 10
    assert rel_l2(got, ref) <= FP32_TOL


def test_graph_replay_equals_eager_bitwise():
    from gpu_helpers import require_cuda
    torch, tn = require_cuda()
    w = make_workload("grid3x4_m8")
    sl = choose_slices(w.struct, w.tree, 64, n_sliced=3)
    out = {}
    for graphs in (0, 1):
        p = tn.Plan(w.circuit, w.bits, w.tree.ssa, sl, slice_batch_log2=1, graphs=graphs)
        ws = torch.empty(p.info["workspace_bytes"], dtype=torch.uint8, device="cuda")
        p.tn_plan_bind(ws)
        res = []
        for _ in range(3):  # capture, then replays
            amps = torch.zeros(2 * 64, dtype=torch.float64, device="cuda")
            p.tn_contract(amps, "fp32")
            torch.cuda.synchronize()
            res.append(amps.cpu().numpy().copy())
        out[graphs] = res
    for r in out[0] + out[1]:
        assert np.array_equal(r, out[0][0])


def test_empty_bitstring_batch_is_a_no_op():
    # k = 0: planning and contraction succeed and write nothing
    torch, tn = require_cuda()
    w = make_workload("grid3x4_m8")
    p = tn.Plan(w.circuit, w.bits[:0], w.tree.ssa)
    assert p.info["n_unique"] == 0
    ws = torch.empty(max(p.info["workspace_bytes"], 256), dtype=torch.uint8, device="cuda")
    p.tn_plan_bind(ws, stream=torch.cuda.current_stream())
    sentinel = torch.full((4,), 7.0, dtype=torch.float64, device="cuda")
    p.tn_contract(sentinel, "bf16x3", stream=torch.cuda.current_stream())
    p.tn_plan_check(stream=torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert torch.all(sentinel == 7.0)


@pytest.mark.parametrize("buffers", [1, 2, 3])
def test_pipelined_batches_match_state_vector(buffers):
    # successive bitstring batches of different sizes through the pipeline
    # (batches i + 1 .. i + w - 1 planned, and with w >= 2 workspaces also
    # bound, while batch i runs): each against the state vector
    torch, tn = require_cuda()
    from paper_2212_04749_gb300.pipeline import contract_batches
    from rqc import grid_layout, network_structure, random_circuit
    from rqc.bitstrings import uniform_bitstrings
    from rqc.tree import candidate_trees
    c = random_circuit(grid_layout(3, 4), 8, seed=3)
    batches = [uniform_bitstrings(12, k, seed=s) for s, k in ((1, 300), (2, 77), (3, 512), (4, 64), (5, 200))]
    ssa = candidate_trees(network_structure(c), 300, seed=1, trials=1)[0]
    ws = [torch.empty(256 << 20, dtype=torch.uint8, device="cuda") for _ in range(buffers)]
    got = dict(contract_batches(c, batches, ssa, [], "fp32", ws[0] if buffers == 1 else tuple(ws)))
    assert sorted(got) == list(range(len(batches)))
    for i, b in enumerate(batches):
        assert rel_l2(got[i], sv.amplitudes(c, b)) <= 1e-5

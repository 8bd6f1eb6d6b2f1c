"""Correlated batches (output qubits left open, SM Sec. II) and perfect
samples from them, on the GPU, against the oracle state vector.

Each input row stands for its 2^r completions over the open qubits; the
amplitudes come back row-major (row, completion).  Tolerances as for closed
bitstrings: FP32 1e-5, BF16x3 1e-3 relative L2.  Sample picks are integer
decisions taken in FP64 by the same correctly rounded operations on both
sides: compared exactly.
"""

import numpy as np
import pytest

from gpu_helpers import rel_l2, require_cuda, run_plan
from oracle import sv
from oracle.sampling import sample_completions
from rqc import grid_layout, make_workload, network_structure, random_circuit
from rqc.bitstrings import uniform_bitstrings
from rqc.tree import ContractionTree, candidate_trees, choose_slices

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def case20():
    c = random_circuit(grid_layout(4, 5), 12, seed=21)
    s = network_structure(c)
    bits = uniform_bitstrings(20, 600, seed=5)
    ssa = candidate_trees(s, 600, seed=2, trials=2)[0]
    sl = choose_slices(s, ContractionTree(ssa=ssa), 600, n_sliced=2)
    return c, bits, ssa, sl


@pytest.mark.parametrize("open_q", [[0, 7], [3, 4, 5, 11], []])
def test_open_qubits_unsliced_match_state_vector(open_q):
    w = make_workload("grid3x4_m8")
    got, p = run_plan(w.circuit, w.bits, w.tree.ssa, w.tree.sliced, precision="fp32", open_qubits=open_q)
    assert p.info["amps_per_row"] == 1 << len(open_q)
    ref = sv.correlated_amplitudes(w.circuit, w.bits, open_q)
    assert got.shape == ref.shape
    assert rel_l2(got, ref) <= 1e-5


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("bf16x3", 1e-3)])
def test_open_qubits_sliced_match_state_vector(case20, prec, tol):
    # every GEMM-shaped step on the grouped GEMM (tensor cores for BF16x3),
    # so the open legs pass through the tensor-core epilogue as well
    c, bits, ssa, sl = case20
    open_q = [2, 9, 17]
    got, p = run_plan(c, bits, ssa, sl, precision=prec, open_qubits=open_q, force_kernel=lambda st: 1)
    kinds = p.tn_plan_step_times()[1]
    if prec == "bf16x3":
        assert sum(1 for k in kinds if k == 2) >= 1
    err = rel_l2(got, sv.correlated_amplitudes(c, bits, open_q))
    print(f"correlated batches 20q, 3 open, {prec}: rel-L2 {err:.2e}, tensor-core steps {sum(1 for k in kinds if k == 2)}")
    assert err <= tol


def test_open_qubit_slices_sum_to_the_contraction(case20):
    torch, tn = require_cuda()
    c, bits, ssa, sl = case20
    open_q = [0, 19]
    total, p = run_plan(c, bits, ssa, sl, precision="fp32", open_qubits=open_q)
    ns = 1 << len(sl)
    part = torch.zeros(2 * ns * len(bits) * 4, dtype=torch.float64, device="cuda")
    p.tn_contract_slices(np.arange(ns), part, "fp32", stream=torch.cuda.current_stream())
    torch.cuda.synchronize()
    s = part.cpu().numpy().view(np.complex128).reshape(ns, -1).sum(axis=0)
    assert rel_l2(s, total) <= 1e-6


def test_perfect_samples_match_oracle_exactly(case20):
    torch, tn = require_cuda()
    c, bits, ssa, sl = case20
    open_q = [1, 6, 12, 18]
    amps, p = run_plan(c, bits, ssa, sl, precision="fp32", open_qubits=open_q)
    k = len(bits)
    rng = np.random.default_rng(17)
    u = rng.random(k)
    d_amps = torch.from_numpy(amps.view(np.float64).copy()).cuda()
    d_u = torch.from_numpy(u).cuda()
    picks = torch.empty(k, dtype=torch.int64, device="cuda")
    tn.tn_sample_completions(d_amps, k, len(open_q), d_u, picks)
    got = picks.cpu().numpy()
    assert np.array_equal(got, sample_completions(amps, len(open_q), u))
    # the drawn completions follow the batches' distributions: their mean
    # probability within the batch exceeds the uniform 1/16 (Porter-Thomas
    # batches: E[p_x | drawn] = 2/16 roughly)
    pr = np.abs(amps.reshape(k, 16)) ** 2
    pr /= pr.sum(axis=1, keepdims=True)
    assert pr[np.arange(k), got].mean() > 1.5 / 16


def test_pipeline_with_open_qubits(case20):
    torch, tn = require_cuda()
    from paper_2212_04749_gb300.pipeline import contract_batches
    c, bits, ssa, sl = case20
    open_q = [4, 5]
    ws = torch.empty(4 << 30, dtype=torch.uint8, device="cuda")
    batches = [bits[:200], bits[200:]]
    got = dict(contract_batches(c, batches, ssa, sl, "fp32", ws, open_qubits=open_q))
    for i, b in enumerate(batches):
        assert rel_l2(got[i], sv.correlated_amplitudes(c, b, open_q)) <= 1e-5
